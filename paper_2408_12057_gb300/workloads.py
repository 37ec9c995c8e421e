"""Seeded synthetic inputs for the five OAIS workloads.

This module only draws data (numpy PCG64, seed = 2408 + workload number); it
holds none of the sampler's arithmetic.  Both the CUDA path and the FP64
checker receive the same arrays from here.  The paper's own datasets are not
used: each workload is a synthetic stand-in with the shapes and value
distributions of the configuration it names.

  1 conjugate Gaussian, d=8: eta = N(0, I), L(x) = exp(-|x-mu|^2/(2*0.5^2)),
    mu ~ N(0, 4 I)
  2 Bayesian logistic regression: X 2000x32 iid N(0,1), w ~ N(0, I),
    y ~ Bernoulli(sigmoid(X w)), prior N(0, I_32)
  3 Gaussian mixture, d=16: 8 equal-weight components, means U[-10,10]^16,
    covariance 0.5 I, reference N(0, 25 I)
  4 Bayesian linear regression: X 50000x256 N(0,1), tau=1, sigma=0.3,
    w ~ N(0, tau^2 I), y = X w + sigma * eps
  5 64 logistic-regression posteriors, n ~ logU[500, 50000],
    d uniform in {8,16,32,64,128}, data as in 2
The annealed multivariate normal of the paper's model table (d=5, tau=5,
tau0=1, mu=0) is workload 1's family with mu = 0 and sigma^2 = 1/4.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GAUSS, LOGREG, GMM, LINREG, UNID = 0, 1, 2, 3, 4


def data_seed(cfg: int) -> int:
    return 2408 + int(cfg)


def run_seed(replicate: int = 0) -> int:
    return 12057 + int(replicate)


@dataclass
class Problem:
    """One target on the geometric path eta * L^beta, eta = N(0, ref_scale^2 I).

    kind   GAUSS / LOGREG / GMM / LINREG / UNID
    X      GAUSS: mu (d,); LOGREG/LINREG: design (n, d); GMM: means (K, d);
           UNID: (m, k) trials and successes (d = 2)
    y      LOGREG labels {0,1} / LINREG responses (n,), else None
    p0     GAUSS: likelihood sigma; GMM: component variance; LINREG: noise sigma;
           UNID: upper end b of the uniform priors
    """
    kind: int
    X: np.ndarray
    y: np.ndarray | None
    ref_scale: float
    p0: float
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        if self.kind == UNID:
            return 2
        return int(self.X.shape[0] if self.kind == GAUSS else self.X.shape[1])

    @property
    def n(self) -> int:
        return 0 if self.kind in (GAUSS, UNID) else int(self.X.shape[0])


def gauss_conj(d: int = 8, sigma: float = 0.5, mu_scale: float = 2.0, seed: int | None = None,
               mu: np.ndarray | None = None) -> Problem:
    rng = np.random.default_rng(data_seed(1) if seed is None else seed)
    if mu is None:
        mu = rng.normal(0.0, mu_scale, size=d)
    return Problem(GAUSS, np.asarray(mu, dtype=np.float64), None, 1.0, sigma,
                   name=f"gauss_conj_d{d}")


def unid(m: float = 1e11, k: float = 1e10, b: float = 10.0) -> Problem:
    """The unidentifiable product parameterisation (the paper's model appendix; its GPU
    experiments use m = 10^11 trials and k = 10^10 successes): X, Y ~ Uniform(0, b),
    K | X, Y ~ Binomial(m, X Y).  The state is z in R^2 under N(0, I) with X = b Phi(z_1),
    Y = b Phi(z_2); no data beyond (m, k)."""
    return Problem(UNID, np.array([float(m), float(k)]), None, 1.0, float(b),
                   name=f"unid_m{m:.0e}_k{k:.0e}")


def annealed_mvn(d: int = 5, tau: float = 5.0, tau0: float = 1.0) -> Problem:
    """The model table's annealed MVN: eta = N(0, 1/tau0), target N(0, 1/tau) per coordinate."""
    sigma = 1.0 / np.sqrt(tau - tau0)
    return Problem(GAUSS, np.zeros(d), None, 1.0 / np.sqrt(tau0), sigma, name=f"annealed_mvn_d{d}")


def logistic(n: int = 2000, d: int = 32, seed: int | None = None) -> Problem:
    rng = np.random.default_rng(data_seed(2) if seed is None else seed)
    X = rng.normal(0.0, 1.0, size=(n, d)).astype(np.float32)
    w = rng.normal(0.0, 1.0, size=d)
    z = X.astype(np.float64) @ w
    p = 1.0 / (1.0 + np.exp(-z))
    y = (rng.uniform(size=n) < p).astype(np.float32)
    return Problem(LOGREG, X, y, 1.0, 1.0, name=f"logreg_n{n}_d{d}", extra={"w_true": w})


def gmm(d: int = 16, K: int = 8, var: float = 0.5, ref_scale: float = 5.0,
        seed: int | None = None) -> Problem:
    rng = np.random.default_rng(data_seed(3) if seed is None else seed)
    means = rng.uniform(-10.0, 10.0, size=(K, d)).astype(np.float32)
    return Problem(GMM, means, None, ref_scale, var, name=f"gmm_d{d}_K{K}")


def linreg(n: int = 50000, d: int = 256, tau: float = 1.0, sigma: float = 0.3,
           seed: int | None = None) -> Problem:
    rng = np.random.default_rng(data_seed(4) if seed is None else seed)
    X = rng.normal(0.0, 1.0, size=(n, d)).astype(np.float32)
    w = rng.normal(0.0, tau, size=d)
    y = (X.astype(np.float64) @ w + sigma * rng.normal(size=n)).astype(np.float32)
    return Problem(LINREG, X, y, tau, sigma, name=f"linreg_n{n}_d{d}", extra={"w_true": w})


def batched_logistic(P: int = 64, n_lo: int = 500, n_hi: int = 50000,
                     dims=(8, 16, 32, 64, 128), seed: int | None = None) -> list[Problem]:
    rng = np.random.default_rng(data_seed(5) if seed is None else seed)
    out = []
    for p in range(P):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        d = int(rng.choice(dims))
        out.append(logistic(n=n, d=d, seed=int(rng.integers(1 << 31))))
    return out


def linear_schedule(T: int) -> np.ndarray:
    return np.linspace(0.0, 1.0, T + 1)
