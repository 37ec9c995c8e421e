"""The tensor-core (tcgen05, BF16) form of the logistic sweep against the FP64 oracle.

The tensor-core form rounds X once to bf16 (X~) and samples the posterior of X~, so
the oracle runs on X~ (exactly representable in fp64).  Particle states and residuals
are split into two bf16 terms, so the contractions keep fp32 accuracy and the same
tolerances as the FP32 CUDA-core form apply (see test_gpu_parity.py): log L and log w
to 1e-5 relative, states to 1e-4, near-tie MH decisions below 1e-3 explain any
disagreement.
"""
import numpy as np
import pytest

import oracle as o
from paper_2408_12057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
oais = pytest.importorskip("paper_2408_12057_gb300.oais")

REL, ABS, XREL, TIE = 1e-5, 1e-4, 1e-4, 1e-3


def bf16_round(X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def oracle_target(pr):
    return o.Target(pr.kind, bf16_round(pr.X), pr.y, pr.ref_scale, pr.p0)


def run(pr, N, beta, eps, seed, contraction):
    r = oais.OAIS(pr, oais.MALA, N, beta, eps=eps, seed=seed, contraction=contraction)
    res = r.round(len(beta) - 1)
    logw, ell, x = r.particles()
    out = dict(res=res, logw=logw.cpu().numpy().copy(), ell=ell.cpu().numpy().copy(),
               x=x.cpu().numpy().T.astype(np.float64).copy(), elbo_t=r.elbo_terms(), **r.stats())
    r.close()
    return out


def agree(g_logw, g_ell, g_x, r_logw, r_ell, r_x, r_margin):
    close = lambda a, b, rt, at: np.abs(a - b) <= at + rt * np.abs(b)
    ok = (close(g_logw, r_logw, REL, ABS) & close(g_ell, r_ell, REL, ABS)
          & np.all(close(g_x, r_x, XREL, XREL), axis=-1))
    bad = ~ok & (r_margin > TIE)
    assert not bad.any(), (f"{int(bad.sum())} particles disagree without a near-tie decision, "
                           f"e.g. {np.flatnonzero(bad)[:5]}: logw {g_logw[bad][:3]} vs {r_logw[bad][:3]}")
    return ok


@pytest.mark.parametrize("n,d,N,T", [(500, 16, 300, 6), (2000, 32, 300, 4), (64, 5, 129, 3), (2000, 32, 256, 1)])
def test_tc_matches_oracle_on_bf16_data(n, d, N, T):
    pr = W.logistic(n=n, d=d, seed=n + d)
    beta = W.linear_schedule(T) ** 3
    eps = oais.default_step_sizes(pr, beta, oais.MALA)
    g = run(pr, N, beta, eps, 31, oais.CONTRACT_BF16_TC)
    r = o.asmc(oracle_target(pr), o.MALA, N, beta, eps, 31)
    ok = agree(g["logw"], g["ell"], g["x"], r["logw"], r["ell"], r["x"], r["margin"])
    assert ok.mean() >= 0.9
    if ok.all():
        np.testing.assert_allclose(g["log_ghat"], r["log_ghat"], rtol=1e-5, atol=1e-4)
        np.testing.assert_allclose(g["accept"], r["accept"], rtol=0, atol=1e-12)
        # ELBO terms sum_n W_{t-1}^n log g_t^n (fp32 offsets and sums on this path)
        np.testing.assert_allclose(g["elbo_t"], r["elbo_t"], rtol=1e-4, atol=1e-3)
        assert g["res"]["kl"] >= -1e-3 * T


def test_tc_importance_sampling_invariant_full_size():
    pr = W.logistic()
    N = 1 << 16
    g = run(pr, N, [0.0, 1.0], 0.01, 77, oais.CONTRACT_BF16_TC)
    lw = torch.from_numpy(g["logw"])
    assert g["log_ghat"][0, 0] == pytest.approx(np.log(N), rel=1e-14)
    assert g["log_ghat"][0, 1] == pytest.approx(torch.logsumexp(lw, 0).item(), rel=1e-12)
    assert g["res"]["logZ"] == pytest.approx(torch.logsumexp(lw, 0).item() - np.log(N), rel=1e-12)
    tg = oracle_target(pr)
    for n in [0, 1, 127, 128, 255, 256, N // 2 + 3, N - 1]:
        r = o.asmc(tg, o.MALA, 1, [0.0, 1.0], 0.01, seed=77, n_offset=n)
        assert g["logw"][n] == pytest.approx(r["logw"][0], rel=REL, abs=ABS)


def test_tc_full_size_sampled():
    pr = W.logistic()
    N, T = 1 << 16, 256
    beta = W.linear_schedule(T) ** 4
    eps = oais.default_step_sizes(pr, beta, oais.MALA)
    g = run(pr, N, beta, eps, 12057, oais.CONTRACT_BF16_TC)
    assert np.isfinite(g["logw"]).all() and np.isfinite(g["log_ghat"]).all()
    tg = oracle_target(pr)
    idx = np.concatenate([[0, 127, 128, 255, 256, N - 1], np.random.default_rng(1).integers(0, N, 10)])
    rs = [o.asmc(tg, o.MALA, 1, beta, eps, seed=12057, n_offset=int(n)) for n in idx]
    ok = agree(g["logw"][idx], g["ell"][idx], g["x"][idx], np.array([r["logw"][0] for r in rs]),
               np.array([r["ell"][0] for r in rs]), np.stack([r["x"][0] for r in rs]),
               np.array([r["margin"][0] for r in rs]))
    assert ok.mean() >= 0.75


def test_tc_agrees_with_fp32_form_on_bf16_data():
    # the FP32 CUDA-core form given X~ as its data samples the same posterior with the same
    # random numbers: both GPU paths agree particle by particle
    pr = W.logistic(n=1000, d=32, seed=4)
    prq = W.Problem(pr.kind, bf16_round(pr.X).astype(np.float32), pr.y, pr.ref_scale, pr.p0)
    beta = W.linear_schedule(8) ** 3
    eps = oais.default_step_sizes(pr, beta, oais.MALA)
    a = run(pr, 2048, beta, eps, 5, oais.CONTRACT_BF16_TC)
    b = run(prq, 2048, beta, eps, 5, oais.CONTRACT_FP32)
    ok = (np.abs(a["logw"] - b["logw"]) <= ABS + REL * np.abs(b["logw"]))
    assert ok.mean() >= 0.95


def test_tc_context_resampling_rounds_and_potential_use_the_streamed_kernel():
    # a resident-form context keeps the streamed form's image and state: its resampling rounds
    # and its potential are those of a streamed-form context, bit for bit
    pr = W.logistic(n=700, d=20, seed=8)
    N, T = 512, 12
    beta = W.linear_schedule(T) ** 2
    eps = oais.default_step_sizes(pr, beta, oais.MALA)
    out = []
    gen = torch.Generator(device="cuda").manual_seed(4)
    x = torch.randn(pr.d, 64, dtype=torch.float32, device="cuda", generator=gen) * 0.3
    for c in (oais.CONTRACT_BF16_TC, oais.CONTRACT_BF16_TC_STREAM):
        r = oais.OAIS(pr, oais.MALA, N, beta, eps=eps, seed=3, contraction=c)
        res = r.asmc_round(0.5, T)
        logw, ell, _ = r.particles()
        pot_ell, pot_g = r.potential(x)
        out.append((res, logw.cpu().numpy().copy(), ell.cpu().numpy().copy(), pot_ell.cpu().numpy().copy(),
                    pot_g.cpu().numpy().copy()))
        r.close()
    (ra, la, ea, pa, ga), (rb, lb, eb, pb, gb) = out
    assert ra["n_resample"] == rb["n_resample"] and ra["n_resample"] > 0
    assert ra["logZ"] == rb["logZ"]
    assert np.array_equal(la, lb) and np.array_equal(ea, eb)
    assert np.array_equal(pa, pb) and np.array_equal(ga, gb)
