"""Pins for the oracle's Alg. 1 (ASMC/AIS), its moment statistics and resampling.

Closed forms used (linear-path exponential family, appendix on MCMC kernels
with linear path): for eta = N(0, s^2 I) and L(x) = exp(-|x-mu|^2/(2 sig^2)),
A(beta) = log Z_beta = (d/2) log(sig^2/(sig^2 + beta s^2)) - beta m/(2(sig^2 + beta s^2))
with m = |mu|^2 (s = 1 below), D(beta, beta') = A(2beta'-beta) - 2A(beta') + A(beta),
delta = A''.  With an exact draw from pi_{beta_t} as the forward kernel the
performance-model assumptions hold exactly, so Thm 1(a) gives the exact
relative variance (exp(D(B_T)) - 1)/N of the AIS estimator.
"""
import os

import numpy as np
import pytest
from scipy import integrate

import oracle as o
from paper_2408_12057_gb300 import workloads as W


def _tg(pr):
    return o.Target(pr.kind, pr.X, pr.y, pr.ref_scale, pr.p0)


def A_gauss(pr, b):
    d, s2, m = pr.d, pr.p0 ** 2, float((pr.X ** 2).sum())
    return d / 2 * np.log(s2 / (s2 + b)) - b * m / (2 * (s2 + b))


def D_gauss(pr, beta):
    return np.array([A_gauss(pr, 2 * beta[t] - beta[t - 1]) - 2 * A_gauss(pr, beta[t])
                     + A_gauss(pr, beta[t - 1]) for t in range(1, len(beta))])


def Lambda_gauss(pr):
    d, s2, m = pr.d, pr.p0 ** 2, float((pr.X ** 2).sum())
    delta = lambda b: (d / 2) / (s2 + b) ** 2 + m * s2 / (s2 + b) ** 3
    return integrate.quad(lambda b: np.sqrt(delta(b)), 0.0, 1.0, epsabs=1e-12)[0]


def test_delta_is_second_derivative_of_A():
    # the closed forms used below are consistent with each other
    pr = W.gauss_conj()
    d, s2, m = pr.d, pr.p0 ** 2, float((pr.X ** 2).sum())
    h = 1e-4
    for b in [0.05, 0.1, 0.7]:
        fd = (A_gauss(pr, b + h) - 2 * A_gauss(pr, b) + A_gauss(pr, b - h)) / h ** 2
        exact = (d / 2) / (s2 + b) ** 2 + m * s2 / (s2 + b) ** 3
        assert fd == pytest.approx(exact, rel=1e-5)


def test_one_step_schedule_is_importance_sampling():
    # B = (0, 1): log Z_hat = LSE_n log L(X_0^n) - log N with X_0^n the reference draws
    pr = W.logistic(n=200, d=6)
    tg = _tg(pr)
    N, seed = 300, 99
    r = o.asmc(tg, o.MALA, N, [0.0, 1.0], 0.1, seed=seed, tag=4)
    X0 = np.stack([pr.ref_scale * o.normals(seed, n, 0, 0, 4, pr.d) for n in range(N)])
    ell0 = np.array([tg.log_lik(x) for x in X0])
    assert np.array_equal(r["logw"], ell0)
    assert r["logZ"] == o.logsumexp(ell0) - np.log(N)
    # the moments of step 1 use w_0 = 1: log g_hat_{1,i} = LSE(i * ell0)
    for i in range(3):
        assert r["log_ghat"][0, i] == pytest.approx(o.logsumexp(i * ell0), rel=1e-14, abs=1e-12)


def test_exact_kernel_logZ_and_discrepancies():
    pr = W.gauss_conj()
    tg = _tg(pr)
    T = 64
    beta = W.linear_schedule(T)
    r = o.asmc(tg, o.EXACT, 8192, beta, 0.0, seed=11)
    # log Z: with D(B_T) ~ 1 and N = 8192 the SE of log Z_hat is ~ sqrt((e^D - 1)/N) ~ 0.015
    Dex = D_gauss(pr, beta)
    se = np.sqrt(np.expm1(Dex.sum()) / 8192)
    assert abs(r["logZ"] - A_gauss(pr, 1.0)) < 4 * se
    _, D_hat, Lam = o.optimise_schedule(beta, r["log_ghat"], T)
    # D_hat_t is consistent for D(beta_{t-1}, beta_t) (eq. CESS)
    assert np.all(D_hat >= 0)
    rel = D_hat / Dex
    assert np.all(np.abs(rel - 1) < 0.2)
    assert abs(rel.mean() - 1) < 0.03
    # Lambda_hat_T approximates sum_t sqrt(D_t) (Cor. 1(b))
    assert Lam[-1] == pytest.approx(np.sqrt(Dex).sum(), rel=0.02)


def test_global_barrier_dense_limit():
    pr = W.gauss_conj()
    tg = _tg(pr)
    T = 400
    beta = W.linear_schedule(T)
    r = o.asmc(tg, o.EXACT, 4096, beta, 0.0, seed=12)
    _, _, Lam = o.optimise_schedule(beta, r["log_ghat"], T)
    assert Lam[-1] == pytest.approx(Lambda_gauss(pr), rel=0.02)


def test_printed_isotropic_normal_barrier():
    gold = dict(l.split() for l in open(os.path.join(os.path.dirname(__file__), "golden",
                                                     "annealed_mvn_barrier.txt"))
                if l.strip() and not l.startswith("#"))
    d, tau, tau0 = int(gold["d"]), float(gold["tau"]), float(gold["tau0"])
    pr = W.annealed_mvn(d=d, tau=tau, tau0=tau0)
    closed = np.sqrt(d / 2) * np.log(tau / tau0)
    assert round(closed, 1) == float(gold["Lambda_hat"])
    # Lambda_PT ~ Lambda / sqrt(pi) in high dimension (PT duality section)
    assert round(closed / np.sqrt(np.pi), 1) == float(gold["Lambda_PT_hat"])
    T = 300
    beta = W.linear_schedule(T)
    for move, kw in [(o.EXACT, {}), (o.RWMH, dict(moves=10))]:
        r = o.asmc(_tg(pr), move, 4096, beta, 0.4, seed=21, **kw)
        _, _, Lam = o.optimise_schedule(beta, r["log_ghat"], T)
        assert abs(Lam[-1] - float(gold["Lambda_hat"])) < 0.05 + 0.05 * closed


def test_high_dimensional_scaling():
    # product of d identical factors: Lambda^(d) = sqrt(d) Lambda^(1) (Sec. 4.3)
    T = 200
    beta = W.linear_schedule(T)
    lams = []
    for d in (1, 16):
        pr = W.annealed_mvn(d=d)
        r = o.asmc(_tg(pr), o.EXACT, 8192, beta, 0.0, seed=31)
        lams.append(o.optimise_schedule(beta, r["log_ghat"], T)[2][-1])
    assert lams[1] / lams[0] == pytest.approx(4.0, rel=0.05)


@pytest.mark.slow
def test_variance_identity_and_unbiasedness():
    pr = W.gauss_conj(d=4, seed=5)
    tg = _tg(pr)
    T, N, R = 32, 128, 600
    # schedule close to optimal for this target: beta = Lambda^-1(Lambda u) from the closed form
    grid = np.linspace(0, 1, 4001)
    lam = np.sqrt(np.gradient(np.gradient([A_gauss(pr, b) for b in grid], grid), grid))
    cum = np.concatenate([[0], np.cumsum(0.5 * (lam[1:] + lam[:-1]) * np.diff(grid))])
    beta = np.interp(np.linspace(0, cum[-1], T + 1), cum, grid)
    beta[0], beta[-1] = 0.0, 1.0
    D_total = D_gauss(pr, beta).sum()
    ratio = np.array([np.exp(o.asmc(tg, o.EXACT, N, beta, 0.0, seed=500 + r)["logZ"]
                             - A_gauss(pr, 1.0)) for r in range(R)])
    # unbiasedness (Prop. 1)
    assert abs(ratio.mean() - 1) < 4 * ratio.std() / np.sqrt(R)
    # Thm 1(a) for AIS: Var[Z_hat/Z] = (exp(D(B_T)) - 1)/N
    pred = np.expm1(D_total) / N
    c = ratio - ratio.mean()
    v = (c ** 2).mean()
    se_v = np.sqrt(((c ** 4).mean() - v ** 2) / R)
    assert abs(v - pred) < 4 * se_v


@pytest.mark.slow
def test_sir_unbiased():
    # SIR (resample every step): Z_hat stays unbiased (Prop. 1).  Thm 1(a)'s product formula
    # is not tested here: after resampling, duplicated particles share their next
    # incremental weight, so particle independence (Assumption 3) cannot hold exactly.
    pr = W.gauss_conj(d=4, seed=5)
    tg = _tg(pr)
    T, N, R = 16, 64, 400
    beta = W.linear_schedule(T)
    ratio = []
    for r in range(R):
        out = o.asmc(tg, o.EXACT, N, beta, 0.0, seed=900 + r, ess_frac=1.0 + 1e-9)
        assert out["n_resample"] == T - 1
        ratio.append(np.exp(out["logZ"] - A_gauss(pr, 1.0)))
    ratio = np.array(ratio)
    assert abs(ratio.mean() - 1) < 4 * ratio.std() / np.sqrt(R)


def test_adaptive_resampling_logZ():
    # ASMC with ESS-triggered resampling (nu = 1/2) on the GMM (reading: L = p/eta, Z = 1)
    pr = W.gmm(d=2, K=3, seed=3)
    tg = _tg(pr)
    T = 100
    beta = W.linear_schedule(T) ** 3
    zs, nres = [], []
    for r in range(8):
        out = o.asmc(tg, o.RWMH, 2000, beta, 0.0, seed=40 + r, moves=4, cycle=True, ess_frac=0.5)
        zs.append(out["logZ"])
        nres.append(out["n_resample"])
        fired = out["resampled"].astype(bool)
        fired[-1] = False                      # t = T closes the last segment regardless
        assert np.all(out["ess"][fired] < 0.5 * 2000)
        assert np.all(out["ess"][~fired][:-1] >= 0.5 * 2000)
    assert min(nres) > 0
    zs = np.array(zs)
    assert abs(zs.mean()) < 4 * zs.std(ddof=1) / np.sqrt(len(zs)) + 0.02


def test_systematic_resampling_offspring_counts():
    rng = np.random.default_rng(0)
    for N in (1, 2, 7, 64, 1000):
        logw = rng.normal(0, 3, size=N)
        W_ = np.exp(logw - o.logsumexp(logw))
        C = np.cumsum(W_)
        for U in (1e-6, 0.37, 0.999999):
            anc = o.systematic_resample(logw, U)
            assert np.all(np.diff(anc) >= 0) and anc.min() >= 0 and anc.max() < N
            # brute force: a^n = min{m : C_m > (n+U)/N}
            brute = np.array([min(N - 1, int(np.argmax(C > (n + U) / N)) if np.any(C > (n + U) / N)
                                  else N - 1) for n in range(N)])
            assert np.array_equal(anc, brute)
            # offspring count of m: ceil(N C_m - U) - ceil(N C_{m-1} - U), total N
            cnt = np.bincount(anc, minlength=N)
            Cm = np.concatenate([[0.0], C])
            closed = np.ceil(N * Cm[1:] - U) - np.ceil(N * Cm[:-1] - U)
            closed[-1] += N - closed.sum()   # C_N = 1 up to rounding
            assert cnt.sum() == N
            assert np.array_equal(cnt, closed.astype(int))


def test_cess_identity_and_nonnegativity():
    pr = W.logistic(n=200, d=4)
    beta = W.linear_schedule(20) ** 2
    r = o.asmc(_tg(pr), o.MALA, 500, beta, 0.2, seed=3)
    g = r["log_ghat"]
    N = 500
    cess = N * np.exp(2 * g[:, 1] - g[:, 2] - g[:, 0])
    _, D_hat, _ = o.optimise_schedule(beta, g, 20)
    assert np.all(D_hat >= 0)
    assert np.all((cess >= 1 - 1e-9) & (cess <= N * (1 + 1e-12)))
    assert np.allclose(D_hat, np.log(N) - np.log(cess), atol=1e-9)


def test_weights_follow_pre_move_state():
    # AIS log-weight after T = 2 is (beta_1 - beta_0) log L(X_0) + (beta_2 - beta_1) log L(X_1),
    # X_1 the state after step 1's move (same counters in a one-step run to beta_1).
    pr = W.gauss_conj(d=3)
    tg = _tg(pr)
    beta = [0.0, 0.3, 1.0]
    N, seed = 6, 8
    full = o.asmc(tg, o.RWMH, N, beta, 0.3, seed=seed)
    first = o.asmc(tg, o.RWMH, N, beta[:2], 0.3, seed=seed)
    X0 = np.stack([o.normals(seed, n, 0, 0, 0, 3) for n in range(N)])
    ell0 = np.array([tg.log_lik(x) for x in X0])
    ell1 = np.array([tg.log_lik(x) for x in first["x"]])
    expect = (0.0 + (beta[1] - beta[0]) * ell0) + (beta[2] - beta[1]) * ell1
    assert np.array_equal(full["logw"], expect)
    assert not np.array_equal(first["x"], X0)   # the move did something
