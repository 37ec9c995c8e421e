"""FP64 CPU oracle for OAIS / ASMC (arXiv 2408.12057) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never loads it; the two share no code.  The arithmetic
lives in ``oais_oracle.c`` (plain C, double precision, no fast-math, no FMA
contraction) and is reached through ctypes.

Function map (paper passage each one follows):
  philox4x32_10        Philox4x32-10 of Salmon et al. (SC'11)
  normals / uniforms   counter layout and Box-Muller map (a reading; the paper
                       only asks for split random streams, App. E.3)
  log_lik              log L and its gradient for the four target families on
                       the geometric path gamma_beta = eta * L^beta (Sec. 2)
  asmc                 Alg. 1 (ASMC), AIS when ess_frac == 0, adaptive
                       resampling (eq. sample_size_IS) otherwise; with the
                       ELBO estimator's terms (log Z = ELBO + KL, section on
                       the KL divergence of a schedule)
  systematic_resample  Sec. 2.1.3
  optimise_schedule    Alg. 3 with D_hat of eq. CESS
  pchip                monotone interpolation used by Alg. 3
  fisher_grad          grad_theta log Z = E_pi[grad_theta log gamma] with the
                       weighted estimator of eq. estimator_pi_t
  zja                  the online conditional-ESS comparator (section on the
                       connection to online CESS optimisation)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oais_oracle.c")
_LIB = os.path.join(_HERE, "liboais_oracle.so")
_lock = threading.Lock()
_lib = None

GAUSS, LOGREG, GMM, LINREG, UNID = 0, 1, 2, 3, 4
RWMH, MALA, HMC, EXACT = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE semantics, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Target(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("d", ctypes.c_int), ("n", ctypes.c_int),
                ("X", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("ref_scale", ctypes.c_double), ("p0", ctypes.c_double)]


class _Move(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("moves", ctypes.c_int),
                ("leapfrog", ctypes.c_int), ("cycle", ctypes.c_int)]


class _Result(ctypes.Structure):
    _fields_ = [("logZ", ctypes.c_double), ("n_resample", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            u32, u64, i32, i64, f64 = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                       ctypes.c_long, ctypes.c_double)
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_u01.argtypes = [u32]
            lib.orc_u01.restype = f64
            lib.orc_normals.argtypes = [u64, u32, u32, u32, u32, i32, P]
            lib.orc_mh_uniform.argtypes = [u64, u32, u32, u32, u32]
            lib.orc_mh_uniform.restype = f64
            lib.orc_resample_uniform.argtypes = [u64, u32, u32]
            lib.orc_resample_uniform.restype = f64
            lib.orc_log_ref.argtypes = [P, P]
            lib.orc_log_ref.restype = f64
            lib.orc_log_lik.argtypes = [P, P, P]
            lib.orc_log_lik.restype = f64
            lib.orc_binom_mode_logpmf.argtypes = [f64, f64]
            lib.orc_binom_mode_logpmf.restype = f64
            lib.orc_logsumexp.argtypes = [P, i64]
            lib.orc_logsumexp.restype = f64
            lib.orc_systematic_resample.argtypes = [i64, P, f64, P]
            lib.orc_asmc.argtypes = [P, P, i64, i32, P, P, u64, u32, i64, f64,
                                     P, P, P, P, P, P, P, P, P, P, P]
            lib.orc_asmc.restype = i32
            lib.orc_zja.argtypes = [P, P, i64, i32, P, P, i32, f64, f64, u64, u32,
                                    P, P, P, P, P, P, P, P, P, P]
            lib.orc_zja.restype = i32
            lib.orc_zja_next_beta.argtypes = [i64, P, P, f64, f64, i32, i32]
            lib.orc_zja_next_beta.restype = f64
            lib.orc_pchip_slopes.argtypes = [i32, P, P, P]
            lib.orc_pchip_eval.argtypes = [i32, P, P, P, f64]
            lib.orc_pchip_eval.restype = f64
            lib.orc_optimise_schedule.argtypes = [i32, P, P, i32, P, P, P]
            lib.orc_optimise_schedule.restype = i32
            lib.orc_fisher_grad.argtypes = [P, i64, P, P, P]
            lib.orc_fisher_grad.restype = i32
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Target:
    """A target family on the geometric path with reference eta = N(0, ref_scale^2 I).

    kind GAUSS : L(x) = exp(-|x - mu|^2 / (2 p0^2)),           X = mu (d,)
    kind LOGREG: L(x) = prod_r Bern(y_r | sigmoid(X_r . x)),    X (n, d), y (n,)
    kind GMM   : L(x) = p(x) / eta(x), p = mean_k N(mu_k, p0 I), X = means (K, d)
    kind LINREG: L(x) = prod_r N(y_r; X_r . x, p0^2),           X (n, d), y (n,)
    kind UNID  : L(z) = Binom(k; m, p0^2 Phi(z_1) Phi(z_2)),     X = (m, k), d = 2, ref_scale 1
    """

    def __init__(self, kind, X, y=None, ref_scale=1.0, p0=1.0):
        self.kind = int(kind)
        self.X = _f64(X)
        if self.kind == GAUSS:
            self.d, self.n = self.X.shape[0], 0
        elif self.kind == UNID:
            self.d, self.n = 2, 0
        else:
            self.n, self.d = self.X.shape
        self.y = None if y is None else _f64(y)
        self.ref_scale = float(ref_scale)
        self.p0 = float(p0)
        self._c = _Target(self.kind, self.d, self.n, self.X.ctypes.data,
                          None if self.y is None else self.y.ctypes.data,
                          self.ref_scale, self.p0)

    def log_lik(self, x, grad=False):
        lib = _load()
        x = _f64(x)
        g = np.zeros(self.d) if grad else None
        v = lib.orc_log_lik(ctypes.byref(self._c), _ptr(x), _ptr(g))
        return (v, g) if grad else v

    def log_ref(self, x):
        return _load().orc_log_ref(ctypes.byref(self._c), _ptr(_f64(x)))


def binom_mode_logpmf(m, k):
    """log Binom(k; m, k/m): log-gamma below a million counts, Stirling's series above."""
    return _load().orc_binom_mode_logpmf(float(m), float(k))


def philox4x32_10(ctr, key):
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(r):
    return _load().orc_u01(int(r))


def normals(seed, n, t, k, tag, d):
    z = np.zeros(d)
    _load().orc_normals(seed, n, t, k, tag, d, _ptr(z))
    return z


def mh_uniform(seed, n, t, k, tag):
    return _load().orc_mh_uniform(seed, n, t, k, tag)


def resample_uniform(seed, t, tag):
    return _load().orc_resample_uniform(seed, t, tag)


def logsumexp(a):
    a = _f64(a)
    return _load().orc_logsumexp(_ptr(a), a.size)


def systematic_resample(logw, U):
    logw = _f64(logw)
    anc = np.zeros(logw.size, dtype=np.int64)
    _load().orc_systematic_resample(logw.size, _ptr(logw), float(U), _ptr(anc))
    return anc


def asmc(target: Target, move_kind, N, beta, eps, seed, tag=0, moves=1, leapfrog=1,
         cycle=False, ess_frac=0.0, n_offset=0):
    """Alg. 1.  Returns a dict with logZ, log_ghat (T,3), accept (T,), ess (T,),
    logw (N,), x (N,d), ell (N,), margin (N,), resampled (T,), n_resample, ancestors (N,) of
    the last intermediate resampling event (-1 if there was none), and the ELBO
    estimator's terms elbo_t (T,) = sum_n W_{t-1}^n log g_t^n with their sum elbo and
    kl = logZ - elbo (log Z = ELBO + KL, section on the KL divergence of a schedule).
    Particle n draws from counter n_offset + n (AIS particles are independent, so a
    subset of a large run can be recomputed on its own)."""
    lib = _load()
    beta = _f64(beta)
    T = beta.size - 1
    eps = _f64(np.broadcast_to(np.asarray(eps, dtype=np.float64), (T,)))
    mv = _Move(int(move_kind), int(moves), int(leapfrog), int(bool(cycle)))
    res = _Result()
    out = dict(log_ghat=np.zeros((T, 3)), accept=np.zeros(T), ess=np.zeros(T),
               logw=np.zeros(N), x=np.zeros((N, target.d)), ell=np.zeros(N),
               margin=np.zeros(N), resampled=np.zeros(T, dtype=np.int64), elbo_t=np.zeros(T),
               ancestors=np.full(N, -1, dtype=np.int64))
    rc = lib.orc_asmc(ctypes.byref(target._c), ctypes.byref(mv), int(N), int(T), _ptr(beta),
                      _ptr(eps), int(seed), int(tag), int(n_offset), float(ess_frac), ctypes.byref(res),
                      _ptr(out["log_ghat"]), _ptr(out["accept"]), _ptr(out["ess"]),
                      _ptr(out["logw"]), _ptr(out["x"]), _ptr(out["ell"]), _ptr(out["margin"]),
                      _ptr(out["resampled"]), _ptr(out["elbo_t"]), _ptr(out["ancestors"]))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    out["logZ"] = res.logZ
    out["n_resample"] = res.n_resample
    out["elbo"] = float(out["elbo_t"].sum())
    out["kl"] = out["logZ"] - out["elbo"]
    return out


def zja(target: Target, move_kind, N, T_max, beta_ref, eps_ref, cess_frac, seed, tag=0, moves=1,
        leapfrog=1, cycle=False, ess_frac=0.0):
    """The online conditional-ESS comparator (section on the connection to online CESS
    optimisation): the schedule is found step by step so that CESS / N = cess_frac (line search
    of four passes over 32 candidates), step sizes interpolated from (beta_ref, eps_ref); then
    the steps of Alg. 1.  Returns a dict with logZ, T, beta (T+1,), eps (T,), log_ghat (T,3),
    elbo_t (T,), logw, x, ell, margin, n_resample."""
    lib = _load()
    beta_ref = _f64(beta_ref)
    T_ref = beta_ref.size - 1
    eps_ref = _f64(np.broadcast_to(np.asarray(eps_ref, dtype=np.float64), (T_ref,)))
    mv = _Move(int(move_kind), int(moves), int(leapfrog), int(bool(cycle)))
    res = _Result()
    Tout = ctypes.c_int()
    out = dict(beta=np.zeros(T_max + 1), eps=np.zeros(T_max), log_ghat=np.zeros((T_max, 3)),
               logw=np.zeros(N), x=np.zeros((N, target.d)), ell=np.zeros(N), margin=np.zeros(N),
               elbo_t=np.zeros(T_max))
    rc = lib.orc_zja(ctypes.byref(target._c), ctypes.byref(mv), int(N), int(T_max), _ptr(beta_ref),
                     _ptr(eps_ref), int(T_ref), float(cess_frac), float(ess_frac), int(seed), int(tag),
                     ctypes.byref(res), ctypes.byref(Tout), _ptr(out["beta"]), _ptr(out["eps"]),
                     _ptr(out["log_ghat"]), _ptr(out["logw"]), _ptr(out["x"]), _ptr(out["ell"]),
                     _ptr(out["margin"]), _ptr(out["elbo_t"]))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    T = Tout.value
    out.update(beta=out["beta"][:T + 1], eps=out["eps"][:T], log_ghat=out["log_ghat"][:T],
               elbo_t=out["elbo_t"][:T], T=T, logZ=res.logZ, n_resample=res.n_resample)
    return out


def zja_next_beta(logw, ell, beta_prev, cess_frac, t=1, T_max=1 << 30):
    """The line search alone: beta_t from the particles' log-weights and log-likelihoods."""
    logw, ell = _f64(logw), _f64(ell)
    return _load().orc_zja_next_beta(logw.size, _ptr(logw), _ptr(ell), float(beta_prev), float(cess_frac),
                                     int(t), int(T_max))


def pchip(xk, yk):
    """Return a callable monotone cubic Hermite interpolant through (xk, yk)."""
    lib = _load()
    xk, yk = _f64(xk), _f64(yk)
    dk = np.zeros_like(xk)
    lib.orc_pchip_slopes(xk.size, _ptr(xk), _ptr(yk), _ptr(dk))

    def f(x):
        x = np.atleast_1d(_f64(x))
        return np.array([lib.orc_pchip_eval(xk.size, _ptr(xk), _ptr(yk), _ptr(dk), float(v))
                         for v in x])
    return f


def optimise_schedule(beta, log_ghat, Tn):
    """Alg. 3.  Returns (beta_new (Tn+1,), D_hat (T,), Lambda_hat (T+1,))."""
    lib = _load()
    beta, log_ghat = _f64(beta), _f64(log_ghat)
    T = beta.size - 1
    bn, D, L = np.zeros(Tn + 1), np.zeros(T), np.zeros(T + 1)
    lib.orc_optimise_schedule(T, _ptr(beta), _ptr(log_ghat), int(Tn), _ptr(bn), _ptr(D), _ptr(L))
    return bn, D, L


def fisher_grad(target: Target, logw, x):
    """(d/dlog s, d/dlog p0) of log Z by the weighted-particle estimator."""
    lib = _load()
    logw, x = _f64(logw), _f64(x)
    g = np.zeros(2)
    lib.orc_fisher_grad(ctypes.byref(target._c), logw.size, _ptr(logw), _ptr(x), _ptr(g))
    return g
