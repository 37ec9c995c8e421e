"""The fp32 CUDA-core lock-step ASMC (Alg. 1 with the ESS trigger of eq. sample_size_IS and
systematic resampling, Sec. 2.1.3) against the FP64 oracle, particle by particle.

The fp32 families keep states and log L in fp32 and log w in fp64 (log g formed in fp32), so a
Metropolis-Hastings decision whose oracle margin |log u - log alpha| is below the fp32 error of
log alpha (1e-3 is generous) may go either way, and one flipped decision changes that
particle's later weights and with them the ancestors of every later event.  So each case takes
the first run seed (searched on the oracle alone, from 100 up) whose decisions all clear that
bound and whose ESS stays 1e-4 N away from the threshold nu N at every step; on such a seed the
two sides must make the same decisions everywhere: the same steps resample, the same
ancestors, and weights, log-likelihoods, states and moments within the fp32 tolerances of the
single-step bar (1e-5 relative on log w, log L, log g_hat and the ESS; 1e-4 on states, which
carry T K rounded updates).  Sizes span several CTAs of 128 particles with a ragged last one.
"""
import numpy as np
import pytest

import oracle as o
from paper_2408_12057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
oais = pytest.importorskip("paper_2408_12057_gb300.oais")

TIE = 1e-3
NU = 0.5


def _tg(pr):
    return o.Target(pr.kind, pr.X, pr.y, pr.ref_scale, pr.p0)


def case(name):
    if name == "gmm_d16_k8_rwmh2":
        # the mixture workload's family (d = 16, 8 components, reference N(0, 25 I)), two
        # random-walk moves per step with the 0.1 / 1 / 10 proposal cycle
        pr = W.gmm()
        return pr, oais.RWMH, o.RWMH, 1000, W.linear_schedule(16) ** 3, 1.0, dict(moves=2, cycle=True)
    if name == "logreg_d32_mala":
        pr = W.logistic(n=300, d=32, seed=5)
        beta = W.linear_schedule(16) ** 2
        return pr, oais.MALA, o.MALA, 700, beta, oais.default_step_sizes(pr, beta, oais.MALA), dict()
    raise KeyError(name)


def clean_seed(pr, omove, N, beta, eps, kw):
    for seed in range(100, 400):
        r = o.asmc(_tg(pr), omove, N, beta, eps, seed, ess_frac=NU, **kw)
        ess_gap = np.min(np.abs(r["ess"][:-1] - NU * N)) / N
        if r["margin"].min() > TIE and ess_gap > 1e-4 and r["n_resample"] > 0:
            return seed, r
    pytest.fail("no seed without near-tie decisions in [100, 400)")


@pytest.mark.parametrize("name", ["gmm_d16_k8_rwmh2", "logreg_d32_mala"])
def test_fp32_lockstep_asmc_matches_oracle(name):
    pr, move, omove, N, beta, eps, kw = case(name)
    seed, r = clean_seed(pr, omove, N, beta, eps, kw)
    run = oais.OAIS(pr, move, N, beta, eps=eps, seed=seed, contraction=oais.CONTRACT_FP32, **kw)
    res = run.asmc_round(NU, len(beta) - 1)
    logw, ell, x = run.particles()
    ess, rs, anc = run.resampling()
    st = run.stats()
    g = dict(logw=logw.cpu().numpy().copy(), ell=ell.cpu().numpy().copy(),
             x=x.cpu().numpy().T.astype(np.float64).copy())
    run.close()
    # the same resampling decisions and the same ancestors of the last event
    assert res["n_resample"] == r["n_resample"]
    np.testing.assert_array_equal(rs, r["resampled"])
    np.testing.assert_array_equal(anc, r["ancestors"])
    np.testing.assert_allclose(ess, r["ess"], rtol=1e-5)
    # particle by particle
    np.testing.assert_allclose(g["logw"], r["logw"], rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(g["ell"], r["ell"], rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(g["x"], r["x"], rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(st["log_ghat"], r["log_ghat"], rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(st["accept"], r["accept"], rtol=0, atol=1e-12)
    assert res["logZ"] == pytest.approx(r["logZ"], rel=1e-5, abs=1e-4)
