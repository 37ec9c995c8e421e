"""Pins for the oracle's online conditional-ESS comparator (Zhou, Johansen & Aston 2016, the
paper's section on the connection to online CESS optimisation):

- the line search alone, against CESS / N = (sum W g)^2 / (sum W g^2) computed here in numpy:
  the chosen step meets the target (relative to the weight share inside the likelihood's
  support) and a step one part in a million longer does not;
- inside a run, the per-step moments recorded by the sampler give CESS_t / N =
  g_hat_1^2 / (g_hat_0 g_hat_2) at the target for every step but the last (the paper's identity
  D_hat_t = log N - log CESS_t ties the search to the moments Alg. 3 uses);
- on the conjugate Gaussian path with a strict target, log Z_hat against the closed form.
"""
import numpy as np
import pytest

import oracle as o
from paper_2408_12057_gb300 import workloads as W


def _tg(pr):
    return o.Target(pr.kind, pr.X, pr.y, pr.ref_scale, pr.p0)


def cess_frac(logw, ell, delta):
    keep = np.isfinite(logw)
    lw, l = logw[keep], ell[keep]
    W = np.exp(lw - lw.max())
    W /= W.sum()
    with np.errstate(over="ignore"):
        v = delta * l
        v = np.where(np.isfinite(l), v, -np.inf)
        m = v[np.isfinite(v)].max()
        g = np.exp(v - m)
    return (W @ g) ** 2 / (W @ (g * g))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_line_search_meets_the_target_at_grid_resolution(seed):
    rng = np.random.default_rng(seed)
    N = 300
    logw = rng.normal(0.0, 1.5, N)
    ell = -np.abs(rng.normal(50.0, 30.0, N))
    logw[:7] = -np.inf                       # zero weights
    ell[7:11] = -np.inf                      # states outside the support
    for beta_prev, c in [(0.0, 0.9), (0.3, 0.5), (0.97, 0.99), (0.0, 0.999999)]:
        b = o.zja_next_beta(logw, ell, beta_prev, c)
        delta = b - beta_prev
        assert beta_prev < b <= 1.0
        # weighted states outside the support are lost at any positive step: the target is
        # relative to the weight share A inside it (the limit of CESS / N as the step -> 0+)
        A = cess_frac(logw, ell, 1e-300)
        if b < 1.0:
            # met at the step, missed one part in a million further (the refined bracket is a
            # few 1e-8 of the step wide)
            assert cess_frac(logw, ell, delta) >= c * A * (1 - 1e-12)
            assert cess_frac(logw, ell, delta * (1 + 1e-6)) < c * A
        else:
            assert cess_frac(logw, ell, 1.0 - beta_prev) >= c * A * (1 - 1e-12)


def test_run_moments_hold_cess_at_target():
    pr = W.logistic(n=150, d=4, seed=3)
    c = 0.8
    r = o.zja(_tg(pr), o.MALA, 400, 500, np.linspace(0, 1, 5), 0.2, c, 11, ess_frac=0.5)
    lg = r["log_ghat"]
    cess = np.exp(2 * lg[:, 1] - lg[:, 0] - lg[:, 2])
    T = r["T"]
    assert T > 5 and r["beta"][-1] == 1.0 and np.all(np.diff(r["beta"]) > 0)
    assert np.all(cess[:-1] >= c * (1 - 1e-9)) and np.all(cess[:-1] <= c * (1 + 1e-3))
    assert cess[-1] >= c * (1 - 1e-9)
    assert r["n_resample"] > 0


def test_gaussian_logZ_against_closed_form():
    pr = W.gauss_conj(d=4, seed=2)
    tg = _tg(pr)
    d, s2, m = pr.d, pr.p0 ** 2, float((pr.X ** 2).sum())
    exact = d / 2 * np.log(s2 / (s2 + 1)) - m / (2 * (s2 + 1))
    z = np.array([o.zja(tg, o.MALA, 2000, 2000, np.linspace(0, 1, 11), 0.4, 0.995, 100 + r, moves=2)["logZ"]
                  for r in range(5)])
    assert abs(z.mean() - exact) < 4 * z.std(ddof=1) / np.sqrt(len(z)) + 0.02, (z, exact)
