"""Alg. 2 with the Budget rule: the particle count changes between rounds within one run.

A run created for N_cap particles and set to N < N_cap computes exactly what a run created
for N computes (particle n draws from counter n), and the Budget driver's rounds grow N and
T as the rule says while the estimates converge to the closed form.
"""
import numpy as np
from mcse import pooled
import pytest

from paper_2408_12057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
oais = pytest.importorskip("paper_2408_12057_gb300.oais")


def final(r):
    logw, ell, x = r.particles()
    return logw.cpu().numpy().copy(), x.cpu().numpy().copy()


@pytest.mark.parametrize("contraction,move", [(oais.CONTRACT_FP32, oais.MALA),
                                              (oais.CONTRACT_BF16_TC_STREAM, oais.HMC)])
def test_set_particles_equals_smaller_run(contraction, move):
    pr = W.linreg(n=200, d=8, seed=3)
    T = 6
    beta = W.linear_schedule(T) ** 2
    eps = oais.default_step_sizes(pr, beta, move)
    big = oais.OAIS(pr, move, 1024, beta, eps=eps, seed=8, leapfrog=3, contraction=contraction)
    big.set_particles(300)
    rb = big.round(T)
    small = oais.OAIS(pr, move, 300, beta, eps=eps, seed=8, leapfrog=3, contraction=contraction)
    rs = small.round(T)
    lb, xb = final(big)
    ls, xs = final(small)
    assert lb.shape == ls.shape == (300,)
    assert np.array_equal(lb, ls) and np.array_equal(xb, xs)
    assert rb["logZ"] == rs["logZ"]
    big.close()
    small.close()


@pytest.mark.parametrize("asmc", [False, True])
def test_budget_rounds_linreg(asmc):
    from test_oracle_closed_forms import linreg_logZ_woodbury
    pr = W.linreg(n=400, d=8, seed=11)
    Xt = torch.from_numpy(np.ascontiguousarray(pr.X, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()
    lz = linreg_logZ_woodbury(Xt.astype(np.float16).astype(np.float64), pr.y.astype(np.float64), pr.ref_scale, pr.p0)
    out = oais.run_rounds(pr, oais.HMC, 1024, 32, 6, 8192, 1024, asmc=asmc, leapfrog=5, adapt=True,
                          contraction=oais.CONTRACT_BF16_TC_STREAM)
    Ns = [N for N, _, _ in out]
    Ts = [T for _, T, _ in out]
    assert Ns[:3] == [1024, 1408, 2048] and Ts[:3] == [32, 45, 64]
    N, T, res = out[-1]
    assert np.isfinite(res["logZ"])
    # the last three rounds (N >= 2944 particles each) pooled: within 3 standard errors
    last = [r for _, _, r in out[-3:]]
    z, se = pooled([r["logZ"] for r in last], [r["se"] for r in last])
    assert abs(z - lz) < 3 * se, (out, lz)
