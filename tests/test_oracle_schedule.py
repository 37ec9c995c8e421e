"""Pins for the oracle's OptimiseSchedule (Alg. 3) and its monotone interpolant."""
import numpy as np
import pytest
from scipy import integrate, interpolate, optimize

import oracle as o
from paper_2408_12057_gb300 import workloads as W


@pytest.mark.parametrize("seed", range(5))
def test_pchip_matches_scipy(seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(2, 40))
    x = np.cumsum(rng.uniform(0.01, 1.0, K))
    y = np.cumsum(rng.uniform(0.0, 1.0, K)) * (rng.uniform() < 0.8) + rng.normal(0, 0.3, K) * (seed == 4)
    f = o.pchip(x, y)
    ref = interpolate.PchipInterpolator(x, y)
    q = np.linspace(x[0], x[-1], 301)
    assert np.allclose(f(q), ref(q), rtol=1e-12, atol=1e-12)
    assert np.allclose(f(x), y, rtol=0, atol=1e-14)


def _ghat_from_D(D):
    # statistics whose D_hat equals D exactly: log g0 = log g1 = 0, log g2 = D
    g = np.zeros((len(D), 3))
    g[:, 2] = D
    return g


def test_constant_local_barrier_gives_uniform_schedule():
    # Gaussian mean shift: lambda is constant, so phi*(u) = u (Sec. 4.4, Gaussian paths)
    T, Tn, lam = 37, 50, 1.7
    beta = np.linspace(0, 1, T + 1) ** 2
    D = (lam * np.diff(beta)) ** 2
    bn, D_hat, Lam = o.optimise_schedule(beta, _ghat_from_D(D), Tn)
    assert np.allclose(D_hat, D, rtol=1e-12)
    assert Lam[-1] == pytest.approx(lam, rel=1e-12)
    assert np.allclose(bn, np.linspace(0, 1, Tn + 1), atol=1e-12)


def test_schedule_inverts_closed_form_barrier():
    # with exact D from the conjugate Gaussian, Alg. 3 approximates beta* = Lambda^-1(Lambda u)
    pr = W.gauss_conj()
    d, s2, m = pr.d, pr.p0 ** 2, float((pr.X ** 2).sum())
    A = lambda b: d / 2 * np.log(s2 / (s2 + b)) - b * m / (2 * (s2 + b))
    lam = lambda b: np.sqrt((d / 2) / (s2 + b) ** 2 + m * s2 / (s2 + b) ** 3)
    Lcum = lambda b: integrate.quad(lam, 0, b, epsabs=1e-13)[0]
    Ltot = Lcum(1.0)
    T = 2000
    beta = np.linspace(0, 1, T + 1)
    D = np.array([A(2 * beta[t] - beta[t - 1]) - 2 * A(beta[t]) + A(beta[t - 1]) for t in range(1, T + 1)])
    Tn = 16
    bn, _, Lam = o.optimise_schedule(beta, _ghat_from_D(D), Tn)
    assert Lam[-1] == pytest.approx(Ltot, rel=1e-3)
    for tp in range(1, Tn):
        star = optimize.brentq(lambda b: Lcum(b) - Ltot * tp / Tn, 0, 1, xtol=1e-14)
        assert bn[tp] == pytest.approx(star, abs=2e-4)
    assert bn[0] == 0.0 and bn[-1] == 1.0 and np.all(np.diff(bn) > 0)


def test_degenerate_statistics():
    beta = np.linspace(0, 1, 6)
    # all D_hat zero -> uniform schedule
    bn, _, Lam = o.optimise_schedule(beta, np.zeros((5, 3)), 8)
    assert Lam[-1] == 0 and np.allclose(bn, np.linspace(0, 1, 9))
    # a zero in the middle and a rounding negative: clamped, duplicate knot dropped, still monotone
    D = np.array([0.1, 0.0, -1e-17, 0.3, 0.2])
    bn, D_hat, _ = o.optimise_schedule(beta, _ghat_from_D(D), 20)
    assert np.all(D_hat >= 0) and np.all(np.diff(bn) >= 0)
    assert bn[0] == 0.0 and bn[-1] == 1.0
    # T = 1 (Alg. 2's first round, B = (0, 1)): two knots, linear new schedule
    bn, _, _ = o.optimise_schedule(np.array([0.0, 1.0]), _ghat_from_D(np.array([2.0])), 4)
    assert np.allclose(bn, [0, 0.25, 0.5, 0.75, 1.0])


def test_oais_rounds_approach_optimal_schedule():
    # Alg. 2 with the exact kernel: the round-k schedule approaches Lambda^-1(Lambda u)
    pr = W.gauss_conj()
    tg = o.Target(pr.kind, pr.X, None, pr.ref_scale, pr.p0)
    d, s2, m = pr.d, pr.p0 ** 2, float((pr.X ** 2).sum())
    lam = lambda b: np.sqrt((d / 2) / (s2 + b) ** 2 + m * s2 / (s2 + b) ** 3)
    Lcum = lambda b: integrate.quad(lam, 0, b, epsabs=1e-13)[0]
    Ltot = Lcum(1.0)
    beta = np.array([0.0, 1.0])
    for k, T in enumerate([1, 8, 32, 64, 64]):
        if k > 0:
            beta, _, _ = o.optimise_schedule(beta, ghat, T)
        r = o.asmc(tg, o.EXACT, 4096, beta, 0.0, seed=70 + k)
        ghat = r["log_ghat"]
    star = np.array([optimize.brentq(lambda b: Lcum(b) - Ltot * u, 0, 1) for u in
                     np.linspace(0, 1, 65)[1:-1]])
    assert np.max(np.abs(beta[1:-1] - star)) < 0.01
