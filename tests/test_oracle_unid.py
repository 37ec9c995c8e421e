"""Pins for the oracle's unidentifiable-product family (the paper's GPU workload "Unid": X, Y ~
Uniform(0, b), K | X, Y ~ Binomial(m, X Y), state z under N(0, I) with X = b Phi(z_1),
Y = b Phi(z_2)):

- log L against scipy's binomial log-pmf at p = X Y, -inf outside (0, 1);
- the mode constant log Binom(k; m, k/m) against 50-digit arithmetic (mpmath), at the
  paper's m = 10^11, k = 10^10 and at small counts;
- the gradient against central differences;
- log Z by AIS against the one-dimensional quadrature
  Z = (1 / (b^2 (m + 1))) int_0^b I_{min(b x, 1)}(k + 1, m - k + 1) / x dx
  (integrating y through p = x y turns the binomial pmf into a regularised incomplete beta),
  and the paper-size value ln(ln(b^2 / q) / (b^2 (m + 1))) ~ -28.00 that it tends to.
"""
import mpmath
import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle as o
from paper_2408_12057_gb300 import workloads as W


def _tg(pr):
    return o.Target(pr.kind, pr.X, pr.y, pr.ref_scale, pr.p0)


def logZ_quadrature(m, k, b):
    q = k / m
    f = lambda x: special.betainc(k + 1, m - k + 1, min(b * x, 1.0)) / x
    val, _ = integrate.quad(f, 0.0, b, points=[q / b, 1.0 / b], limit=500, epsabs=0, epsrel=1e-12)
    return np.log(val) - 2 * np.log(b) - np.log(m + 1)


def test_log_likelihood_is_the_binomial_log_pmf():
    pr = W.unid(m=1000, k=100)
    tg = _tg(pr)
    rng = np.random.default_rng(0)
    seen_in, seen_out = 0, 0
    for _ in range(200):
        z = rng.normal(-1.8, 0.8, size=2)
        p = pr.p0 ** 2 * stats.norm.cdf(z[0]) * stats.norm.cdf(z[1])
        v = tg.log_lik(z)
        if 0.0 < p < 1.0:
            assert v == pytest.approx(stats.binom.logpmf(100, 1000, p), rel=1e-10, abs=1e-10)
            seen_in += 1
        else:
            assert v == -np.inf
            seen_out += 1
    assert seen_in > 20 and seen_out > 20


@pytest.mark.parametrize("m,k", [(1e11, 1e10), (1e11, 3e10), (5e7, 2e6), (1000, 100), (40, 3)])
def test_mode_constant_against_multiprecision(m, k):
    mpmath.mp.dps = 50
    M, K = mpmath.mpf(m), mpmath.mpf(k)
    q = K / M
    ref = (mpmath.loggamma(M + 1) - mpmath.loggamma(K + 1) - mpmath.loggamma(M - K + 1)
           + K * mpmath.log(q) + (M - K) * mpmath.log(1 - q))
    assert o.binom_mode_logpmf(m, k) == pytest.approx(float(ref), rel=1e-12, abs=1e-9)


@pytest.mark.parametrize("m,k", [(1000, 100), (1e11, 1e10)])
def test_gradient_against_central_differences(m, k):
    tg = _tg(W.unid(m=m, k=k))
    # points near the ridge p = k / m (for the large counts the finite differences need the
    # curvature scale: h ~ 1e-9 there)
    q = k / m
    z2 = stats.norm.ppf(q / 100.0 / stats.norm.cdf(-1.0))
    for z in [np.array([-1.0, z2]), np.array([-1.0, z2 + (0.3 if m < 1e6 else 3e-6)])]:
        v, g = tg.log_lik(z, grad=True)
        h = 1e-6 if m < 1e6 else 1e-9
        for i in range(2):
            e = np.zeros(2)
            e[i] = h
            fd = (tg.log_lik(z + e) - tg.log_lik(z - e)) / (2 * h)
            assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-5 * (1 + abs(fd)))


def test_logZ_against_quadrature():
    pr = W.unid(m=1000, k=100)
    tg = _tg(pr)
    lz = logZ_quadrature(1000.0, 100.0, pr.p0)
    T = 400
    beta = np.linspace(0.0, 1.0, T + 1) ** 4
    z = np.array([o.asmc(tg, o.RWMH, 4000, beta, 0.02, 300 + r, moves=2)["logZ"] for r in range(6)])
    assert abs(z.mean() - lz) < 4 * z.std(ddof=1) / np.sqrt(len(z)) + 0.02, (z, lz)


def test_paper_size_logZ_closed_form():
    # m = 10^11: I_{b x}(k + 1, m - k + 1) is a step at b x = q to within ~1e-6 in x, so the
    # quadrature tends to ln(ln(b^2 / q) / (b^2 (m + 1)))
    m, k, b = 1e11, 1e10, 10.0
    q = k / m
    approx = np.log(np.log(b * b / q) / (b * b * (m + 1)))
    assert approx == pytest.approx(-28.00095, abs=1e-4)
    assert logZ_quadrature(1e6, 1e5, b) == pytest.approx(np.log(np.log(b * b / q) / (b * b * (1e6 + 1))), abs=2e-3)


def test_infeasible_start_weights_vanish():
    # under the reference most draws have X Y >= 1: their log-likelihood is -inf, their weight
    # becomes 0 at the first positive step and stays 0; the estimate is finite
    pr = W.unid(m=1000, k=100)
    r = o.asmc(_tg(pr), o.RWMH, 500, np.linspace(0.0, 1.0, 11), 0.05, 7)
    assert np.isfinite(r["logZ"])
    frac_dead = np.mean(r["logw"] == -np.inf)
    assert 0.8 < frac_dead < 1.0
    assert r["elbo_t"][0] == -np.inf and r["kl"] == np.inf
