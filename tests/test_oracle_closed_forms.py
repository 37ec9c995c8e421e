"""Pins for the oracle's MCMC kernels and estimators against closed forms and
quadrature: each kernel must leave pi_beta invariant for Z_hat to be unbiased,
so a wrong acceptance ratio or drift shows up as a biased log Z."""
import numpy as np
import pytest
from scipy import special, stats

import oracle as o
from paper_2408_12057_gb300 import workloads as W


def _tg(pr):
    return o.Target(pr.kind, pr.X, pr.y, pr.ref_scale, pr.p0)


def linreg_logZ(X, y, tau, sigma):
    """log Z = log N(y; 0, sigma^2 I + tau^2 X X^T) (a library density)."""
    n = X.shape[0]
    return stats.multivariate_normal(np.zeros(n), sigma ** 2 * np.eye(n) + tau ** 2 * X @ X.T).logpdf(y)


def linreg_logZ_woodbury(X, y, tau, sigma):
    """The same quantity through the d x d form (used at full size)."""
    n, d = X.shape
    XtX, Xty = X.T @ X, X.T @ y
    A = np.eye(d) / tau ** 2 + XtX / sigma ** 2
    _, logdet = np.linalg.slogdet(np.eye(d) + (tau ** 2 / sigma ** 2) * XtX)
    m = np.linalg.solve(A, Xty / sigma ** 2)
    return (-0.5 * n * np.log(2 * np.pi) - n * np.log(sigma) - 0.5 * logdet
            - y @ y / (2 * sigma ** 2) + Xty @ m / (2 * sigma ** 2))


def linreg_grad_closed(X, y, tau, sigma):
    n, d = X.shape
    A = np.eye(d) / tau ** 2 + X.T @ X / sigma ** 2
    S = np.linalg.inv(A)
    m = S @ X.T @ y / sigma ** 2
    g_tau = (m @ m + np.trace(S)) / tau ** 2 - d
    r = y - X @ m
    g_sig = (r @ r + np.trace(S @ X.T @ X)) / sigma ** 2 - n
    return np.array([g_tau, g_sig])


def test_linreg_closed_forms_agree():
    pr = W.linreg(n=30, d=4)
    X, y = pr.X.astype(np.float64), pr.y.astype(np.float64)
    a = linreg_logZ(X, y, pr.ref_scale, pr.p0)
    assert linreg_logZ_woodbury(X, y, pr.ref_scale, pr.p0) == pytest.approx(a, rel=1e-11)
    # gradient in (log tau, log sigma) against finite differences of the library form
    h = 1e-5
    fd = [(linreg_logZ(X, y, pr.ref_scale * np.exp(h), pr.p0) - linreg_logZ(X, y, pr.ref_scale * np.exp(-h), pr.p0)) / (2 * h),
          (linreg_logZ(X, y, pr.ref_scale, pr.p0 * np.exp(h)) - linreg_logZ(X, y, pr.ref_scale, pr.p0 * np.exp(-h))) / (2 * h)]
    assert np.allclose(linreg_grad_closed(X, y, pr.ref_scale, pr.p0), fd, rtol=1e-6, atol=1e-6)


def _replicates(tg, move, N, beta, eps, R, seed0, **kw):
    out = [o.asmc(tg, move, N, beta, eps, seed=seed0 + r, **kw) for r in range(R)]
    z = np.array([r["logZ"] for r in out])
    return z, out


def test_hmc_linreg_logZ_and_fisher_gradient():
    pr = W.linreg(n=40, d=3, seed=11)
    tg = _tg(pr)
    X, y = pr.X.astype(np.float64), pr.y.astype(np.float64)
    T = 200
    beta = W.linear_schedule(T) ** 4
    eps = 0.3 / np.sqrt(1 + beta[1:] * X.shape[0] / pr.p0 ** 2)
    z, outs = _replicates(tg, o.HMC, 1000, beta, eps, 6, 100, leapfrog=5)
    exact = linreg_logZ(X, y, pr.ref_scale, pr.p0)
    assert abs(z.mean() - exact) < 4 * z.std(ddof=1) / np.sqrt(len(z)) + 0.01
    g = np.array([o.fisher_grad(tg, r["logw"], r["x"]) for r in outs])
    gc = linreg_grad_closed(X, y, pr.ref_scale, pr.p0)
    se = g.std(axis=0, ddof=1) / np.sqrt(len(g))
    assert np.all(np.abs(g.mean(axis=0) - gc) < 4 * se + 0.05 * np.abs(gc) + 0.05)


def test_mala_gauss_logZ_and_fisher_gradient():
    pr = W.gauss_conj(d=4, seed=2)
    tg = _tg(pr)
    T = 100
    beta = W.linear_schedule(T) ** 2
    eps = 0.9 / np.sqrt(1 + beta[1:] / pr.p0 ** 2)
    z, outs = _replicates(tg, o.MALA, 2000, beta, eps, 6, 300, moves=2)
    d, s2, m = pr.d, pr.p0 ** 2, float((pr.X ** 2).sum())
    exact = d / 2 * np.log(s2 / (s2 + 1)) - m / (2 * (s2 + 1))
    assert abs(z.mean() - exact) < 4 * z.std(ddof=1) / np.sqrt(len(z)) + 0.01
    # d log Z / d log s (prior scale) and d log Z / d log sigma_L, closed form with s = 1
    gc = np.array([-d / (s2 + 1) + m / (s2 + 1) ** 2, d / (s2 + 1) + m * s2 / (s2 + 1) ** 2])
    g = np.array([o.fisher_grad(tg, r["logw"], r["x"]) for r in outs])
    se = g.std(axis=0, ddof=1) / np.sqrt(len(g))
    assert np.all(np.abs(g.mean(axis=0) - gc) < 4 * se + 0.02 * np.abs(gc) + 0.02)


def test_mala_logistic_d2_against_quadrature():
    pr = W.logistic(n=60, d=2, seed=5)
    tg = _tg(pr)
    X, yv = pr.X.astype(np.float64), pr.y.astype(np.float64)
    # brute-force 2-D quadrature of Z = int N(x; 0, I) L(x) dx on a fine grid
    g = np.linspace(-7, 7, 1401)
    xx, yy = np.meshgrid(g, g, indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel()], 1)
    z = pts @ X.T
    loglik = (yv * z - np.logaddexp(0, z)).sum(1)
    logprior = -0.5 * (pts ** 2).sum(1) - np.log(2 * np.pi)
    h = g[1] - g[0]
    logZ_quad = special.logsumexp(loglik + logprior) + 2 * np.log(h)
    T = 100
    beta = W.linear_schedule(T) ** 3
    eps = 0.9 / np.sqrt(1 + beta[1:] * X.shape[0] / 4)
    zs, _ = _replicates(tg, o.MALA, 2000, beta, eps, 6, 500, moves=2)
    assert abs(zs.mean() - logZ_quad) < 4 * zs.std(ddof=1) / np.sqrt(len(zs)) + 0.01


def test_rwmh_gmm_normalised_target():
    # reading of the mixture workload: L = p / eta with p a normalised mixture, so log Z = 0
    pr = W.gmm(d=2, K=4, seed=9)
    tg = _tg(pr)
    T = 200
    beta = W.linear_schedule(T) ** 3
    zs, _ = _replicates(tg, o.RWMH, 2000, beta, 0.0, 6, 700, moves=3, cycle=True)
    assert abs(zs.mean()) < 4 * zs.std(ddof=1) / np.sqrt(len(zs)) + 0.01


@pytest.mark.parametrize("move,eps,kw", [
    (o.RWMH, 0.9, dict(moves=2)),
    (o.MALA, 0.7, dict(moves=2)),
    (o.HMC, 0.4, dict(leapfrog=3)),    # eps * omega * L ~ pi/2: a quarter period
])
def test_kernels_leave_pi_beta_invariant(move, eps, kw):
    # fixed temperature b after the first step: the particles must settle on pi_b,
    # which for the conjugate Gaussian is N(m_b, v_b I) with 1/v_b = 1 + b/sigma^2,
    # m_b = (b/sigma^2) mu v_b.  A wrong acceptance ratio moves these moments.
    pr = W.gauss_conj(d=3, sigma=0.8, seed=4)
    tg = _tg(pr)
    b = 0.6
    beta = np.array([0.0] + [b] * 60)
    r = o.asmc(tg, move, 20000, beta, eps, seed=5, **kw)
    v = 1.0 / (1.0 + b / pr.p0 ** 2)
    mean = (b / pr.p0 ** 2) * pr.X * v
    x = r["x"]
    n = x.shape[0]
    assert np.all(np.abs(x.mean(0) - mean) < 4.5 * np.sqrt(v / n))
    assert np.all(np.abs(x.var(0) - v) < 4.5 * v * np.sqrt(2.0 / n))
