"""Pins for the oracle's ELBO by-product (section on the KL divergence of a schedule:
log Z = ELBO + KL, ELBO estimated by sum_t sum_n W_{t-1}^n log g_t^n with normalised
weights W).  Reading: the printed estimator's W are the normalised weights of Alg. 1, so
the printed 1/N factor does not apply (with it the estimate would vanish as N grows).

- one step from the reference: W_0 is uniform and log g_1 = (beta_1 - beta_0) log L(X_0),
  so the term is the plain mean over the initial draws, recomputed here from the counter
  random numbers and the likelihood written out;
- Jensen, per step and per realisation: log sum_n W g >= sum_n W log g, i.e. every term lies
  below log g_hat_{t,1} - log g_hat_{t,0}, and the KL estimate log Z_hat - ELBO is >= 0;
- exact transitions on the conjugate Gaussian path (each move an independent draw from
  pi_beta): the weights are independent of the current draws, so the term of step t is an
  unbiased estimate of (beta_t - beta_{t-1}) E_{pi_beta_{t-1}}[log L], a closed form.
"""
import numpy as np
import pytest

import oracle as o
from paper_2408_12057_gb300 import workloads as W


def _tg(pr):
    return o.Target(pr.kind, pr.X, pr.y, pr.ref_scale, pr.p0)


def test_single_step_term_is_mean_log_likelihood_of_the_initial_draws():
    pr = W.gauss_conj(d=5, sigma=0.7, seed=3)
    tg = _tg(pr)
    N, seed, tag = 257, 11, 4
    beta = np.array([0.0, 0.35])
    r = o.asmc(tg, o.MALA, N, beta, 0.3, seed, tag=tag)
    mu, s2 = pr.X, pr.p0 ** 2
    x0 = np.stack([pr.ref_scale * o.normals(seed, n, 0, 0, tag, pr.d) for n in range(N)])
    ell0 = -0.5 * np.sum((x0 - mu) ** 2, axis=1) / s2
    assert r["elbo_t"][0] == pytest.approx(0.35 * ell0.mean(), rel=1e-12, abs=1e-12)
    assert r["elbo"] == pytest.approx(r["elbo_t"].sum(), rel=1e-15)


@pytest.mark.parametrize("case", ["gauss_mala", "logreg_mala_resampling", "linreg_hmc"])
def test_terms_obey_jensen_per_step(case):
    if case == "gauss_mala":
        pr, move, kw, ess = W.gauss_conj(d=4, seed=5), o.MALA, {}, 0.0
    elif case == "logreg_mala_resampling":
        pr, move, kw, ess = W.logistic(n=120, d=5, seed=6), o.MALA, {}, 0.5
    else:
        pr, move, kw, ess = W.linreg(n=60, d=4, seed=7), o.HMC, {"leapfrog": 3}, 0.0
    T = 24
    beta = W.linear_schedule(T) ** 3
    r = o.asmc(_tg(pr), move, 400, beta, 0.2, 9, ess_frac=ess, **kw)
    lg = r["log_ghat"]
    bound = lg[:, 1] - lg[:, 0]
    assert np.all(r["elbo_t"] <= bound + 1e-10 * (1.0 + np.abs(bound)))
    assert r["kl"] >= -1e-9 * (1.0 + abs(r["logZ"]))
    if ess > 0.0:
        assert r["n_resample"] > 0


def test_exact_transitions_gaussian_closed_form():
    pr = W.gauss_conj(d=3, sigma=0.8, seed=4)
    tg = _tg(pr)
    mu, s2, d = pr.X, pr.p0 ** 2, pr.d
    T, N = 6, 40000
    beta = W.linear_schedule(T)
    r = o.asmc(tg, o.EXACT, N, beta, 0.0, 21)

    def moments(b):
        # pi_b = N(m, v I) with precision 1 + b / s2 (reference N(0, I)) and m = v b mu / s2
        v = 1.0 / (1.0 + b / s2)
        m = v * b * mu / s2
        mean = -(np.sum((m - mu) ** 2) + d * v) / (2 * s2)
        var = np.sum(2 * v * v + 4 * v * (m - mu) ** 2) / (4 * s2 * s2)
        return mean, var

    ess = np.concatenate([[N], r["ess"][:-1]])   # ESS of W_{t-1}
    for t in range(1, T + 1):
        mean, var = moments(beta[t - 1])
        db = beta[t] - beta[t - 1]
        se = db * np.sqrt(var / ess[t - 1])
        assert abs(r["elbo_t"][t - 1] - db * mean) < 5 * se + 1e-12, t
    assert r["kl"] >= 0.0
