"""Pins for the oracle's targets: each log-likelihood against a library density
(scipy.stats), each gradient against central finite differences."""
import numpy as np
import pytest
from scipy import special, stats

import oracle as o
from paper_2408_12057_gb300 import workloads as W


def _tg(pr):
    return o.Target(pr.kind, pr.X, pr.y, pr.ref_scale, pr.p0)


def _points(d, k=5, scale=1.0, seed=0):
    return np.random.default_rng(seed).normal(0, scale, size=(k, d))


def test_gauss_matches_scipy():
    pr = W.gauss_conj()
    tg = _tg(pr)
    for x in _points(pr.d):
        ref = stats.multivariate_normal(pr.X, pr.p0 ** 2 * np.eye(pr.d)).logpdf(x)
        ref += 0.5 * pr.d * np.log(2 * np.pi * pr.p0 ** 2)   # L is the unnormalised kernel
        assert tg.log_lik(x) == pytest.approx(ref, rel=1e-12, abs=1e-12)
        assert tg.log_ref(x) == pytest.approx(stats.multivariate_normal(np.zeros(pr.d)).logpdf(x),
                                              rel=1e-12)


def test_logistic_matches_scipy():
    pr = W.logistic(n=300, d=7)
    tg = _tg(pr)
    X = pr.X.astype(np.float64)
    for x in _points(pr.d, scale=0.5):
        p = special.expit(X @ x)
        ref = stats.bernoulli.logpmf(pr.y.astype(int), p).sum()
        assert tg.log_lik(x) == pytest.approx(ref, rel=1e-10)


def test_logistic_extreme_logits_stay_finite():
    X = np.array([[1.0], [-1.0]])
    tg = o.Target(o.LOGREG, X, np.array([1.0, 0.0]))
    v, g = tg.log_lik(np.array([800.0]), grad=True)
    assert np.isfinite(v) and np.isfinite(g).all()
    assert v == pytest.approx(0.0, abs=1e-300)


def test_gmm_matches_scipy():
    pr = W.gmm(d=4, K=3)
    tg = _tg(pr)
    for x in _points(pr.d, scale=6.0):
        comp = [stats.multivariate_normal(m, pr.p0 * np.eye(pr.d)).logpdf(x) for m in pr.X]
        logp = special.logsumexp(comp) - np.log(len(comp))
        logeta = stats.multivariate_normal(np.zeros(pr.d), pr.ref_scale ** 2 * np.eye(pr.d)).logpdf(x)
        assert tg.log_lik(x) == pytest.approx(logp - logeta, rel=1e-11)


def test_linreg_matches_scipy():
    pr = W.linreg(n=40, d=5)
    tg = _tg(pr)
    X = pr.X.astype(np.float64)
    for x in _points(pr.d):
        ref = stats.norm(X @ x, pr.p0).logpdf(pr.y).sum()
        assert tg.log_lik(x) == pytest.approx(ref, rel=1e-11)


@pytest.mark.parametrize("make", [
    lambda: W.gauss_conj(d=6),
    lambda: W.logistic(n=120, d=5),
    lambda: W.gmm(d=3, K=4),
    lambda: W.linreg(n=30, d=4),
])
def test_gradient_by_finite_differences(make):
    pr = make()
    tg = _tg(pr)
    h = 1e-6
    for x in _points(pr.d, k=3, scale=0.7, seed=3):
        _, g = tg.log_lik(x, grad=True)
        fd = np.zeros(pr.d)
        for i in range(pr.d):
            e = np.zeros(pr.d)
            e[i] = h
            fd[i] = (tg.log_lik(x + e) - tg.log_lik(x - e)) / (2 * h)
        assert np.allclose(g, fd, rtol=1e-5, atol=1e-5 * (1 + np.abs(fd).max()))
