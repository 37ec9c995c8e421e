"""The online conditional-ESS comparator on the GPU (zja.cu + the lock-step ASMC kernels)
against the oracle's: the schedule found step by step, the estimate, the particles, and the
identity that every step but the last holds CESS_t / N = g_hat_1^2 / (g_hat_0 g_hat_2) at the
target (the device line search sums in fp32, so a candidate within ~1e-6 of the target may
fall on the other side: schedules are compared to the grid's resolution)."""
import numpy as np
import pytest

import oracle as o
from paper_2408_12057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
oais = pytest.importorskip("paper_2408_12057_gb300.oais")


def _tg(pr):
    return o.Target(pr.kind, pr.X, pr.y, pr.ref_scale, pr.p0)


def gpu_zja(pr, move, N, beta_ref, eps_ref, c, seed, ess_frac=0.0, T_max=400, **kw):
    r = oais.OAIS(pr, move, N, beta_ref, T_max=T_max, eps=eps_ref, seed=seed, **kw)
    res = r.zja_round(c, 8, ess_frac)
    st = r.stats()
    logw, ell, x = r.particles()
    out = dict(res=res, logw=logw.cpu().numpy().copy(), ell=ell.cpu().numpy().copy(),
               x=x.cpu().numpy().T.astype(np.float64).copy(), elbo_t=r.elbo_terms(), **st)
    out["next_T"] = r.schedule()[0].size - 1
    r.close()
    return out


@pytest.mark.parametrize("ess_frac", [0.0, 0.5])
def test_gauss_zja_matches_oracle(ess_frac):
    pr = W.gauss_conj(d=4, seed=2)
    N, c = 500, 0.9
    beta_ref = np.linspace(0.0, 1.0, 11)
    eps_ref = np.geomspace(0.5, 0.2, 10)
    g = gpu_zja(pr, oais.MALA, N, beta_ref, eps_ref, c, 17, ess_frac=ess_frac, moves=2)
    r = o.zja(_tg(pr), o.MALA, N, 400, beta_ref, eps_ref, c, 17, moves=2, ess_frac=ess_frac)
    T = g["res"]["T"]
    assert T == r["T"] and g["beta"].size == T + 1 and g["next_T"] == 8
    np.testing.assert_allclose(g["beta"], r["beta"], rtol=0, atol=1e-5)
    # CESS at the target on every step but the last (the fp32 sums: ~1e-5)
    cess = np.exp(2 * g["log_ghat"][:, 1] - g["log_ghat"][:, 0] - g["log_ghat"][:, 2])
    assert np.all(cess[:-1] >= c * (1 - 1e-4)) and np.all(cess[:-1] <= c * (1 + 2e-3))
    if np.array_equal(g["beta"], r["beta"]):
        np.testing.assert_allclose(g["logw"], r["logw"], rtol=1e-9, atol=1e-9)
        assert g["res"]["logZ"] == pytest.approx(r["logZ"], rel=1e-9, abs=1e-6)
    else:
        assert g["res"]["logZ"] == pytest.approx(r["logZ"], rel=1e-4, abs=1e-3)
    assert g["res"]["n_resample"] == r["n_resample"]


def test_unid_zja_runs_and_holds_the_target():
    # most reference draws are outside the support: they are lost at the first positive step
    # whatever its size, so the target is relative to the weight share inside the support, and
    # from then on the live particles carry the run
    pr = W.unid(m=1000, k=100)
    N, c = 2000, 0.8
    g = gpu_zja(pr, oais.RWMH, N, np.linspace(0.0, 1.0, 11), 0.05, c, 23, ess_frac=0.5, moves=2, T_max=2000)
    r = o.zja(_tg(pr), o.RWMH, N, 2000, np.linspace(0.0, 1.0, 11), 0.05, c, 23, moves=2, ess_frac=0.5)
    assert np.isfinite(g["res"]["logZ"]) and g["beta"][-1] == 1.0
    assert abs(g["res"]["T"] - r["T"]) <= max(2, r["T"] // 50)
    assert g["res"]["logZ"] == pytest.approx(r["logZ"], abs=0.5)
