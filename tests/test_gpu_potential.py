"""The potential entry point (log L and its hand-written gradient kernel), its autograd
wrapper, and the Fisher-identity gradient of log Z, against the FP64 oracle and closed forms."""
import numpy as np
import pytest

import oracle as o
from paper_2408_12057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
oais = pytest.importorskip("paper_2408_12057_gb300.oais")


def _tg(pr):
    return o.Target(pr.kind, pr.X, pr.y, pr.ref_scale, pr.p0)


@pytest.mark.parametrize("make,move", [
    (lambda: W.logistic(), oais.MALA),
    (lambda: W.linreg(n=500, d=16, seed=2), oais.HMC),
    (lambda: W.gmm(), oais.RWMH),
    (lambda: W.gauss_conj(), oais.MALA),
    (lambda: W.logistic(n=77, d=3, seed=9), oais.MALA),
])
def test_potential_matches_oracle(make, move):
    pr = make()
    run = oais.OAIS(pr, move, 16, W.linear_schedule(2))
    dt = torch.float64 if pr.kind == W.GAUSS else torch.float32
    N = 1000
    g = torch.Generator().manual_seed(3)
    x = (torch.randn(pr.d, N, generator=g, dtype=torch.float64) * (0.3 if pr.kind != W.GMM else 5.0)).to(dt)
    ell, grad = run.potential(x.cuda())
    ell, grad = ell.cpu().numpy(), grad.cpu().numpy().astype(np.float64)
    tg = _tg(pr)
    rel = 1e-12 if pr.kind == W.GAUSS else 1e-5
    for n in range(0, N, 37):
        v, gv = tg.log_lik(x[:, n].double().numpy(), grad=True)
        assert ell[n] == pytest.approx(v, rel=rel, abs=1e-4 if pr.kind != W.GAUSS else 1e-12)
        scale = 1 + np.abs(gv).max()
        np.testing.assert_allclose(grad[:, n], gv, rtol=0, atol=(1e-10 if pr.kind == W.GAUSS else 2e-5) * scale)
    run.close()


def test_autograd_wrapper_gradcheck_fp64_family():
    pr = W.gauss_conj(d=6, seed=1)
    run = oais.OAIS(pr, oais.MALA, 16, W.linear_schedule(2))
    LogLik = oais.log_likelihood_function()
    x = torch.randn(9, pr.d, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda v: LogLik.apply(v, run), (x,), eps=1e-6, atol=1e-7)
    run.close()


def test_autograd_wrapper_logistic_backward():
    pr = W.logistic(n=300, d=8, seed=4)
    run = oais.OAIS(pr, oais.MALA, 16, W.linear_schedule(2))
    LogLik = oais.log_likelihood_function()
    x = (torch.randn(50, pr.d, device="cuda") * 0.3).requires_grad_(True)
    w = torch.rand(50, device="cuda", dtype=torch.float32)
    (LogLik.apply(x, run) * w).sum().backward()
    tg = _tg(pr)
    for n in range(0, 50, 7):
        _, gv = tg.log_lik(x[n].detach().double().cpu().numpy(), grad=True)
        np.testing.assert_allclose(x.grad[n].cpu().numpy(), w[n].item() * gv, rtol=1e-4, atol=1e-4)
    run.close()


def test_fisher_gradient_matches_oracle_on_same_particles():
    pr = W.gauss_conj(d=4, seed=2)
    beta = W.linear_schedule(40) ** 2
    run = oais.OAIS(pr, oais.MALA, 3000, beta, eps=0.5, seed=3)
    run.round(40)
    g = run.grad_logZ()
    logw, ell, x = (t.cpu().numpy() for t in run.particles())
    ref = o.fisher_grad(_tg(pr), logw, x.T)
    np.testing.assert_allclose(g, ref, rtol=1e-9, atol=1e-9)
    run.close()


def test_fisher_gradient_linreg_closed_form():
    pr = W.linreg(n=40, d=3, seed=11)
    X, y = pr.X.astype(np.float64), pr.y.astype(np.float64)
    A = np.eye(3) / pr.ref_scale ** 2 + X.T @ X / pr.p0 ** 2
    S = np.linalg.inv(A)
    m = S @ X.T @ y / pr.p0 ** 2
    closed = np.array([(m @ m + np.trace(S)) / pr.ref_scale ** 2 - 3,
                       ((y - X @ m) @ (y - X @ m) + np.trace(S @ X.T @ X)) / pr.p0 ** 2 - 40])
    beta = W.linear_schedule(200) ** 4
    eps = oais.default_step_sizes(pr, beta, oais.HMC) * 0.6
    gs = []
    for rep in range(8):
        run = oais.OAIS(pr, oais.HMC, 1 << 15, beta, eps=eps, seed=40 + rep, leapfrog=5)
        run.round(200)
        gs.append(run.grad_logZ())
        run.close()
    gs = np.array(gs)
    se = gs.std(axis=0, ddof=1) / np.sqrt(len(gs))
    # within 3 standard errors of the mean over eight seeds
    assert np.all(np.abs(gs.mean(0) - closed) < 3 * se), (gs.mean(0), closed, se)
