"""ctypes binding of the OAIS C ABI (include/oais.h).

Argument marshalling only: every step of the sampler runs in liboais.so's CUDA
kernels.  PyTorch provides the device workspace (a uint8 tensor) and the CUDA
stream (the current torch stream).  There is no CPU fallback: if the library
cannot be built or loaded, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

GAUSS, LOGREG, GMM, LINREG, UNID = 0, 1, 2, 3, 4
RWMH, MALA, HMC = 0, 1, 2
DT_F64, DT_F32 = 0, 1
CONTRACT_FP32, CONTRACT_BF16_TC, CONTRACT_BF16_TC_STREAM, CONTRACT_FP8_TC_STREAM = 0, 1, 2, 3
FAULT_NONE, FAULT_NAN_DATA, FAULT_WITHHOLD_HANDOFF = 0, 1, 2

STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
          4: "non-finite value", 5: "device wait timed out", 6: "unsupported configuration"}


class OAISError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Target(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("d", ctypes.c_int32), ("n", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("X", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("ref_scale", ctypes.c_double), ("p0", ctypes.c_double),
                ("on_device", ctypes.c_int32), ("contraction", ctypes.c_int32)]


class _Move(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("moves", ctypes.c_int32), ("leapfrog", ctypes.c_int32),
                ("cycle", ctypes.c_int32), ("adapt", ctypes.c_int32)]


class _RoundResult(ctypes.Structure):
    _fields_ = [("logZ", ctypes.c_double), ("se", ctypes.c_double), ("Lambda_hat", ctypes.c_double),
                ("ess", ctypes.c_double), ("sweep_ms", ctypes.c_double), ("T", ctypes.c_int32),
                ("round", ctypes.c_int32), ("n_resample", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("elbo", ctypes.c_double), ("kl", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load liboais.so (building it with nvcc first if it is stale or missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            P, i32, i64, u32, u64, f64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                              ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                              ctypes.c_size_t)
            sig = {
                "oais_workspace_bytes": ([P, P, i64, i32, P], i32),
                "oais_init": ([P, P, P, i64, P, i32, i32, P, u64, P, sz, P], i32),
                "oais_round": ([P, i32, P], i32),
                "oasmc_round": ([P, i32, f64, P], i32),
                "oais_zja_round": ([P, f64, f64, i32, P], i32),
                "oais_get_resampling": ([P, P, P, P], i32),
                "asmc_run": ([P, P, i64, P, i32, P, f64, u64, P, P, P, P, P], i32),
                "oais_logZ": ([P, P, P], i32),
                "oais_get_stats": ([P, P, P, P, P, P], i32),
                "oais_get_elbo": ([P, P, P], i32),
                "oais_get_schedule": ([P, P, P, P], i32),
                "oais_set_schedule": ([P, P, P, i32], i32),
                "oais_particles": ([P, P, P, P], i32),
                "oais_grad_logZ": ([P, P], i32),
                "oais_set_shard": ([P, i64, i64], i32),
                "oais_state_bytes": ([P, P], i32),
                "oais_save_state": ([P, P, sz], i32),
                "oais_load_state": ([P, P, sz], i32),
                "oais_round_local": ([P, P, P, P, P], i32),
                "oais_round_commit": ([P, i32, P, P, P, P], i32),
                "oais_potential": ([P, P, i64, P, P, P], i32),
                "oais_destroy": ([P], None),
                "oais_last_error": ([P], ctypes.c_char_p),
                "oais_status_string": ([i32], ctypes.c_char_p),
                "oais_optimise_schedule": ([i32, P, P, i32, P, P, P], i32),
                "oais_sweep_blocks": ([i64], i32),
                "oais_step_partial_bytes": ([], i32),
                "oais_ctx_sweep": ([P, i32, P, P, u64, u32, i64, i64, P, P, P, P, P, P], i32),
                "oais_merge_stats": ([P, i32, i32, i64, i32, P, P, P], i32),
                "oais_logsumexp_scratch_bytes": ([i64], sz),
                "oais_logsumexp": ([P, i64, P, P, P], i32),
                "oais_batch_init": ([P, i32, P, P, i64, P, i32, i32, P, u64, P, P, P], i32),
                "oais_batch_round": ([P, i32, P], i32),
                "oais_batch_autotune": ([P, i32, P], i32),
                "oais_batch_tile_shape": ([P, i32, P, P], i32),
                "oais_batch_set_tile_shape": ([P, i32, i32, i32], i32),
                "oais_batch_context": ([P, i32, P], i32),
                "oais_batch_last_error": ([P], ctypes.c_char_p),
                "oais_batch_destroy": ([P], None),
                "oais_set_problem": ([P, i32], i32),
                "oais_budget": ([i64, i32, i64, i32, P, P], i32),
                "oais_set_particles": ([P, i64], i32),
                "oais_merge_shard_stats": ([i32, i32, P, P, P, P, P, P], i32),
                "oais_default_step_sizes": ([P, i32, P, i32, P], i32),
                "oais_arm_fault": ([P, i32, f64], i32),
                "oais_set_exact_data": ([P, i32], i32),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(st, ctx=None):
    if st != 0:
        msg = lib().oais_last_error(ctx)
        raise OAISError(st, msg.decode() if msg else "")


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def optimise_schedule(beta, log_ghat, T_next):
    """Alg. 3 on the host (library code, no device work): (beta_next, D_hat, Lambda_hat)."""
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    lg = np.ascontiguousarray(log_ghat, dtype=np.float64)
    T = beta.size - 1
    bn, D, L = np.zeros(T_next + 1), np.zeros(T), np.zeros(T + 1)
    _check(lib().oais_optimise_schedule(T, _np_ptr(beta), _np_ptr(lg), int(T_next), _np_ptr(bn),
                                        _np_ptr(D), _np_ptr(L)))
    return bn, D, L


def _host_target(problem, contraction=CONTRACT_FP32):
    """(_Target, keep-alive arrays) describing a workloads.Problem with host data."""
    kind = problem.kind
    dtype = DT_F64 if kind in (GAUSS, UNID) else DT_F32
    npdt = np.float64 if dtype == DT_F64 else np.float32
    X = np.ascontiguousarray(problem.X, dtype=npdt)
    y = None if problem.y is None else np.ascontiguousarray(problem.y, dtype=npdt)
    tg = _Target(kind, problem.d, problem.n, dtype, X.ctypes.data, None if y is None else y.ctypes.data,
                 problem.ref_scale, problem.p0, 0, int(contraction))
    return tg, (X, y)


def default_step_sizes(problem, beta, move_kind):
    """The library's starting rule for per-step sizes (oais_default_step_sizes): the reference
    scale shrunk by the tempered curvature of the likelihood and by the kernel's dimension
    scaling; returns eps [T] for the schedule beta [T+1]."""
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    T = beta.size - 1
    tg, keep = _host_target(problem)
    eps = np.zeros(T)
    _check(lib().oais_default_step_sizes(ctypes.byref(tg), int(move_kind), _np_ptr(beta), T, _np_ptr(eps)))
    del keep
    return eps


class OAIS:
    """One OAIS run (Alg. 2) over a target of paper_2408_12057_gb300.workloads.Problem."""

    def __init__(self, problem, move_kind, N, beta, T_max=None, eps=None, seed=12057, moves=1,
                 leapfrog=5, cycle=False, adapt=False, data_on_device=True, stream=None,
                 contraction=CONTRACT_FP32, exact_data=False):
        import torch
        self._torch = torch
        self.problem = problem
        self.N = int(N)
        beta = np.ascontiguousarray(beta, dtype=np.float64)
        T = beta.size - 1
        self.T_max = int(T_max if T_max is not None else T)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        kind = problem.kind
        dtype = DT_F64 if kind in (GAUSS, UNID) else DT_F32
        npdt = np.float64 if dtype == DT_F64 else np.float32
        X = np.ascontiguousarray(problem.X, dtype=npdt)
        y = None if problem.y is None else np.ascontiguousarray(problem.y, dtype=npdt)
        if data_on_device:
            self._X = torch.from_numpy(X).cuda()
            self._y = None if y is None else torch.from_numpy(y).cuda()
            Xp, yp = self._X.data_ptr(), (None if y is None else self._y.data_ptr())
        else:
            self._X, self._y = X, y
            Xp, yp = X.ctypes.data, (None if y is None else y.ctypes.data)
        self._tg = _Target(kind, problem.d, problem.n, dtype, Xp, yp, problem.ref_scale, problem.p0,
                           1 if data_on_device else 0, int(contraction))
        self._mv = _Move(int(move_kind), int(moves), int(leapfrog), int(bool(cycle)), int(bool(adapt)))
        L = lib()
        nbytes = ctypes.c_size_t()
        _check(L.oais_workspace_bytes(ctypes.byref(self._tg), ctypes.byref(self._mv), self.N,
                                      self.T_max, ctypes.byref(nbytes)))
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
        eps_arr = None if eps is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(eps, dtype=np.float64), (T,)))
        self._ctx = ctypes.c_void_p()
        _check(L.oais_init(ctypes.byref(self._ctx), ctypes.byref(self._tg), ctypes.byref(self._mv),
                           self.N, _np_ptr(beta), T, self.T_max,
                           None if eps_arr is None else _np_ptr(eps_arr), int(seed),
                           _dptr(self.workspace), self.workspace.numel(), _stream_ptr(self.stream)))
        if exact_data:
            self.set_exact_data(True)

    def close(self):
        if getattr(self, "_borrowed", False):
            return
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().oais_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def set_particles(self, N):
        """Active particle count of the next rounds (at most the count the run was created with)."""
        _check(lib().oais_set_particles(self._ctx, int(N)), self._ctx)
        self.N = int(N)

    def set_exact_data(self, on=True):
        """Tensor-core forms: reweight each round's final particles from the rounded data X~ to X
        (oais_set_exact_data), so that log Z_hat estimates log Z of X."""
        _check(lib().oais_set_exact_data(self._ctx, int(bool(on))), self._ctx)

    def arm_fault(self, kind, wait_seconds=0.0):
        """Test support: arm a host-side fault for the next round (oais_arm_fault):
        FAULT_NAN_DATA (the round returns a non-finite error) or FAULT_WITHHOLD_HANDOFF (a
        persistent tensor-core sweep's bounded hand-off waits give up after wait_seconds)."""
        _check(lib().oais_arm_fault(self._ctx, int(kind), float(wait_seconds)), self._ctx)

    def set_problem(self, p):
        """Problem index p in the random-number tag (round | p << 16), as problem p of a batch."""
        _check(lib().oais_set_problem(self._ctx, int(p)), self._ctx)

    __del__ = close

    def round(self, T_next=None):
        """Run one round; returns a dict with logZ, se, Lambda_hat, ess, sweep_ms, T, round."""
        if T_next is None:
            T_next = self.schedule()[0].size - 1
        r = _RoundResult()
        _check(lib().oais_round(self._ctx, int(T_next), ctypes.byref(r)), self._ctx)
        return {f: getattr(r, f) for f, _ in _RoundResult._fields_ if f != "pad"}

    def asmc_round(self, ess_frac=0.5, T_next=None):
        """One optimised-ASMC round with adaptive resampling (ESS < ess_frac * N)."""
        if T_next is None:
            T_next = self.schedule()[0].size - 1
        r = _RoundResult()
        _check(lib().oasmc_round(self._ctx, int(T_next), float(ess_frac), ctypes.byref(r)), self._ctx)
        return {f: getattr(r, f) for f, _ in _RoundResult._fields_ if f != "pad"}

    def zja_round(self, cess_frac, T_next=None, ess_frac=0.0):
        """One run of the online conditional-ESS comparator (the schedule found step by step
        so that CESS / N = cess_frac); the schedule that ran is then ``stats()["beta"]``."""
        if T_next is None:
            T_next = self.schedule()[0].size - 1
        r = _RoundResult()
        _check(lib().oais_zja_round(self._ctx, float(cess_frac), float(ess_frac), int(T_next), ctypes.byref(r)),
               self._ctx)
        return {f: getattr(r, f) for f, _ in _RoundResult._fields_ if f != "pad"}

    def resampling(self):
        """(ess [T], resampled [T], ancestors of the last event [N]) of the last ASMC round."""
        T = self.stats()["D_hat"].size
        ess, rs, anc = np.zeros(T), np.zeros(T, dtype=np.int32), np.zeros(self.N, dtype=np.int64)
        _check(lib().oais_get_resampling(self._ctx, _np_ptr(ess), _np_ptr(rs), _np_ptr(anc)), self._ctx)
        return ess, rs, anc

    def logZ(self):
        z, s = ctypes.c_double(), ctypes.c_double()
        _check(lib().oais_logZ(self._ctx, ctypes.byref(z), ctypes.byref(s)), self._ctx)
        return z.value, s.value

    def stats(self):
        T = ctypes.c_int32()
        _check(lib().oais_get_stats(self._ctx, None, None, None, None, ctypes.byref(T)), self._ctx)
        T = T.value
        lg, D, b, a = np.zeros((T, 3)), np.zeros(T), np.zeros(T + 1), np.zeros(T)
        _check(lib().oais_get_stats(self._ctx, _np_ptr(lg), _np_ptr(D), _np_ptr(b), _np_ptr(a), None),
               self._ctx)
        return {"log_ghat": lg, "D_hat": D, "beta": b, "accept": a}

    def elbo_terms(self):
        """Per-step ELBO terms sum_n W_{t-1}^n log g_t^n of the last round (their sum is the
        round result's ``elbo``, and ``kl`` = logZ - elbo)."""
        T = ctypes.c_int32()
        _check(lib().oais_get_elbo(self._ctx, None, ctypes.byref(T)), self._ctx)
        e = np.zeros(T.value)
        _check(lib().oais_get_elbo(self._ctx, _np_ptr(e), None), self._ctx)
        return e

    def schedule(self):
        T = ctypes.c_int32()
        _check(lib().oais_get_schedule(self._ctx, None, None, ctypes.byref(T)), self._ctx)
        b, e = np.zeros(T.value + 1), np.zeros(T.value)
        _check(lib().oais_get_schedule(self._ctx, _np_ptr(b), _np_ptr(e), None), self._ctx)
        return b, e

    def set_schedule(self, beta, eps=None):
        beta = np.ascontiguousarray(beta, dtype=np.float64)
        T = beta.size - 1
        e = None if eps is None else np.ascontiguousarray(np.broadcast_to(
            np.asarray(eps, dtype=np.float64), (T,)))
        _check(lib().oais_set_schedule(self._ctx, _np_ptr(beta), None if e is None else _np_ptr(e), T),
               self._ctx)

    # ---- checkpoint / resume between rounds ----
    def save_state(self) -> bytes:
        n = ctypes.c_size_t()
        _check(lib().oais_state_bytes(self._ctx, ctypes.byref(n)), self._ctx)
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().oais_save_state(self._ctx, buf, n.value), self._ctx)
        return buf.raw

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().oais_load_state(self._ctx, buf, len(blob)), self._ctx)

    # ---- sharding across processes (one exchange of 4T + 2 doubles per round) ----
    def set_shard(self, n_offset, N_total):
        """This run's particles are [n_offset, n_offset + N) of a run of N_total."""
        _check(lib().oais_set_shard(self._ctx, int(n_offset), int(N_total)), self._ctx)

    def round_local(self):
        """Sweep this shard: dict(log_ghat [T,3], accepted [T], lse [2]) for the exchange."""
        T = self.schedule()[0].size - 1
        lg, acc, lse, Tc = np.zeros((T, 3)), np.zeros(T), np.zeros(2), ctypes.c_int32()
        _check(lib().oais_round_local(self._ctx, _np_ptr(lg), _np_ptr(acc), _np_ptr(lse), ctypes.byref(Tc)),
               self._ctx)
        return {"log_ghat": lg, "accepted": acc, "lse": lse}

    def round_commit(self, T_next, merged):
        """Install the statistics merged over all shards; returns the round result."""
        r = _RoundResult()
        lg = np.ascontiguousarray(merged["log_ghat"], dtype=np.float64)
        acc = np.ascontiguousarray(merged["accepted"], dtype=np.float64)
        lse = np.ascontiguousarray(merged["lse"], dtype=np.float64)
        _check(lib().oais_round_commit(self._ctx, int(T_next), _np_ptr(lg), _np_ptr(acc), _np_ptr(lse),
                                       ctypes.byref(r)), self._ctx)
        return {f: getattr(r, f) for f, _ in _RoundResult._fields_ if f != "pad"}

    def grad_logZ(self):
        """Fisher-identity estimate of d log Z / d(log ref_scale, log p0) from the last round."""
        g = np.zeros(2)
        _check(lib().oais_grad_logZ(self._ctx, _np_ptr(g)), self._ctx)
        return g

    def potential(self, x, grad=True, stream=None):
        """log L and grad log L at states x [d, N] (CUDA tensor of the family's dtype)."""
        torch = self._torch
        x = x.contiguous()
        N = x.shape[1]
        ell = torch.empty(N, dtype=torch.float64, device=x.device)
        g = torch.empty_like(x) if grad else None
        _check(lib().oais_potential(self._ctx, _dptr(x), N, _dptr(ell), None if g is None else _dptr(g),
                                    _stream_ptr(stream)), self._ctx)
        return (ell, g) if grad else ell

    def particles(self):
        """(logw [N], ell [N], x [d, N]) torch views of the final particles of the last round."""
        torch = self._torch
        pl, pe, px = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().oais_particles(self._ctx, ctypes.byref(pl), ctypes.byref(pe), ctypes.byref(px)),
               self._ctx)
        base = self.workspace.data_ptr()
        N, d = self.N, self.problem.d

        def view(ptr, dtype, count):
            esz = torch.empty(0, dtype=dtype).element_size()
            off = ptr - base
            return self.workspace[off:off + count * esz].view(dtype)

        xdt = torch.float64 if self.problem.kind in (GAUSS, UNID) else torch.float32
        return (view(pl.value, torch.float64, N), view(pe.value, torch.float64, N),
                view(px.value, xdt, d * N).view(d, N))

    # ---- kernel-level calls (device tensors) ----
    def sweep(self, beta_dev, eps_dev, seed, tag, n_offset, N, logw, ell, x, partials, status,
              stream=None):
        T = beta_dev.numel() - 1
        _check(lib().oais_ctx_sweep(self._ctx, T, _dptr(beta_dev), _dptr(eps_dev), int(seed), int(tag),
                                    int(n_offset), int(N), _dptr(logw), _dptr(ell), _dptr(x),
                                    _dptr(partials), _dptr(status), _stream_ptr(stream)), self._ctx)


def merge_shard_stats(parts):
    """Merge per-shard round statistics in rank order (oais_merge_shard_stats): the moments and
    the final weight sums combine by log-sum-exp over shards, acceptance counts add."""
    P = len(parts)
    T = int(np.asarray(parts[0]["log_ghat"]).shape[0])
    lg = np.ascontiguousarray(np.stack([p["log_ghat"] for p in parts]), dtype=np.float64)
    acc = np.ascontiguousarray(np.stack([p["accepted"] for p in parts]), dtype=np.float64)
    lse = np.ascontiguousarray(np.stack([p["lse"] for p in parts]), dtype=np.float64)
    lg_o, acc_o, lse_o = np.zeros((T, 3)), np.zeros(T), np.zeros(2)
    _check(lib().oais_merge_shard_stats(P, T, _np_ptr(lg), _np_ptr(acc), _np_ptr(lse), _np_ptr(lg_o),
                                        _np_ptr(acc_o), _np_ptr(lse_o)))
    return {"log_ghat": lg_o, "accepted": acc_o, "lse": lse_o}


def exchange_stats(local, group=None, device=None):
    """All-gather one shard's statistics (4T + 2 doubles) over a torch.distributed group and
    merge them.  Works with gloo (CPU tensors) and NCCL (pass device=cuda)."""
    import torch
    import torch.distributed as dist
    T = local["log_ghat"].shape[0]
    flat = np.concatenate([local["log_ghat"].ravel(), local["accepted"], local["lse"]])
    t = torch.from_numpy(flat)
    if device is not None:
        t = t.to(device)
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(bufs, t, group=group)
    parts = []
    for b in bufs:
        v = b.cpu().numpy()
        parts.append({"log_ghat": v[:3 * T].reshape(T, 3), "accepted": v[3 * T:4 * T], "lse": v[4 * T:]})
    return merge_shard_stats(parts)


def distributed_round(run, T_next, group=None, device=None):
    """One OAIS round of a run sharded over the ranks of `group` (each rank one OAIS shard)."""
    merged = exchange_stats(run.round_local(), group=group, device=device)
    return run.round_commit(T_next, merged)


def sweep_blocks(N):
    return lib().oais_sweep_blocks(int(N))


def step_partial_bytes():
    return lib().oais_step_partial_bytes()


def merge_stats(partials, nblocks, T, N, moves, stream=None):
    import torch
    lg = torch.empty((T, 3), dtype=torch.float64, device="cuda")
    acc = torch.empty(T, dtype=torch.float64, device="cuda")
    _check(lib().oais_merge_stats(_dptr(partials), int(nblocks), int(T), int(N), int(moves), _dptr(lg),
                                  _dptr(acc), _stream_ptr(stream)))
    return lg, acc


def logsumexp(a, stream=None):
    """(log sum exp a, log sum exp 2a) of a float64 CUDA tensor, as a 2-element CUDA tensor."""
    import torch
    n = a.numel()
    scratch = torch.empty(lib().oais_logsumexp_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    _check(lib().oais_logsumexp(_dptr(a), n, _dptr(out), _dptr(scratch), _stream_ptr(stream)))
    return out


def log_likelihood_function():
    """torch.autograd.Function whose forward is log L(x) for a batch of states and whose
    backward applies the hand-written gradient kernel (both from one oais_potential call).

    Usage: LogLik = log_likelihood_function(); ell = LogLik.apply(x, run) with x [N, d]."""
    import torch

    class LogLikelihood(torch.autograd.Function):
        @staticmethod
        def forward(fctx, x, run):
            ell, g = run.potential(x.detach().t().contiguous(), grad=True)
            fctx.save_for_backward(g)
            return ell.to(x.dtype)

        @staticmethod
        def backward(fctx, grad_out):
            (g,) = fctx.saved_tensors
            return (grad_out.to(g.dtype)[:, None] * g.t()), None

    return LogLikelihood


def budget(N, T, N_cap, T_cap):
    """Alg. 2's Budget: (N, T) times sqrt(2) while N fits N_cap, then T doubles (oais_budget)."""
    Nn, Tn = ctypes.c_int64(), ctypes.c_int32()
    _check(lib().oais_budget(int(N), int(T), int(N_cap), int(T_cap), ctypes.byref(Nn), ctypes.byref(Tn)))
    return Nn.value, Tn.value


def run_rounds(problem, move_kind, N0, T0, rounds, N_cap, T_cap, asmc=False, ess_frac=0.5, **kw):
    """Alg. 2 with Budget: `rounds` rounds starting from N0 particles on the linear schedule of
    length T0; each round's particle count and schedule length come from budget().  One run
    holds N_cap particles' worth of memory.  Returns [(N, T, result)] per round."""
    beta0 = np.linspace(0.0, 1.0, int(T0) + 1)
    r = OAIS(problem, move_kind, int(N_cap), beta0, T_max=int(T_cap), **kw)
    r.set_particles(N0)
    N, T, out = int(N0), int(T0), []
    try:
        for _ in range(int(rounds)):
            Nn, Tn = budget(N, T, N_cap, T_cap)
            res = r.asmc_round(ess_frac, Tn) if asmc else r.round(Tn)
            out.append((N, T, res))
            r.set_particles(Nn)
            N, T = Nn, Tn
    finally:
        r.close()
    return out


class OAISBatch:
    """P independent OAIS runs of one family whose sweeps share one persistent tensor-core
    launch per round (captured as a CUDA graph).  problems: list of workloads.Problem (LOGREG
    with MALA, or LINREG with MALA or HMC; d <= 128).  eps: [P][T] step sizes or None (the
    starting rule default_step_sizes per problem).  batch.problem(p) gives an OAIS view of
    problem p (logZ, stats, schedule, particles, ...)."""

    def __init__(self, problems, move_kind, N, beta, T_max=None, eps=None, seed=12057, moves=1, leapfrog=5,
                 stream=None):
        import torch
        self._torch = torch
        self.problems = list(problems)
        P = len(self.problems)
        self.N = int(N)
        beta = np.ascontiguousarray(beta, dtype=np.float64)
        T = beta.size - 1
        self.T_max = int(T_max if T_max is not None else T)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._keep = []
        tgs = (_Target * P)()
        for p, pr in enumerate(self.problems):
            X = torch.from_numpy(np.ascontiguousarray(pr.X, dtype=np.float32)).cuda()
            y = torch.from_numpy(np.ascontiguousarray(pr.y, dtype=np.float32)).cuda()
            self._keep += [X, y]
            tgs[p] = _Target(pr.kind, pr.d, pr.n, DT_F32, X.data_ptr(), y.data_ptr(), pr.ref_scale, pr.p0, 1,
                             CONTRACT_BF16_TC_STREAM)
        self._mv = _Move(int(move_kind), int(moves), int(leapfrog), 0, 0)
        L = lib()
        self.workspaces = []
        ptrs, sizes = (ctypes.c_void_p * P)(), (ctypes.c_size_t * P)()
        for p in range(P):
            nb = ctypes.c_size_t()
            _check(L.oais_workspace_bytes(ctypes.byref(tgs[p]), ctypes.byref(self._mv), self.N, self.T_max,
                                          ctypes.byref(nb)))
            w = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
            self.workspaces.append(w)
            ptrs[p], sizes[p] = w.data_ptr(), nb.value
        if eps is None:
            eps = np.stack([default_step_sizes(pr, beta, move_kind) for pr in self.problems])
        eps = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.float64), (P, T)))
        self._b = ctypes.c_void_p()
        st = L.oais_batch_init(ctypes.byref(self._b), P, tgs, ctypes.byref(self._mv), self.N, _np_ptr(beta), T,
                               self.T_max, _np_ptr(eps), int(seed), ptrs, sizes, _stream_ptr(self.stream))
        if st != 0:
            raise OAISError(st, L.oais_batch_last_error(None).decode())
        self._views = []
        for p, pr in enumerate(self.problems):
            c = ctypes.c_void_p()
            self._check(L.oais_batch_context(self._b, p, ctypes.byref(c)))
            v = OAIS.__new__(OAIS)
            v._torch, v.problem, v.N, v.T_max, v.stream = torch, pr, self.N, self.T_max, self.stream
            v._ctx, v.workspace, v._borrowed = c, self.workspaces[p], True
            self._views.append(v)

    def _check(self, st):
        if st != 0:
            raise OAISError(st, lib().oais_batch_last_error(self._b).decode())

    def round(self, T_next=None):
        """One round of every problem; returns a list of per-problem result dicts."""
        P = len(self.problems)
        if T_next is None:
            T_next = self._views[0].schedule()[0].size - 1
        res = (_RoundResult * P)()
        self._check(lib().oais_batch_round(self._b, int(T_next), res))
        return [{f: getattr(r, f) for f, _ in _RoundResult._fields_ if f != "pad"} for r in res]

    def autotune(self, T_probe=4):
        """Time the tile shapes (rows per X chunk, ring depth) per width class (d_pad 16/32/64/128)
        and keep the fastest; returns the chosen depths (tile_shape gives the whole shape)."""
        chosen = (ctypes.c_int32 * 4)()
        self._check(lib().oais_batch_autotune(self._b, int(T_probe), chosen))
        return list(chosen)

    def tile_shape(self, width_class):
        """(rows per X chunk, ring depth) of a width class (0: d_pad 16 ... 3: d_pad 128); (0, 0) if absent."""
        ch, st = ctypes.c_int32(), ctypes.c_int32()
        self._check(lib().oais_batch_tile_shape(self._b, int(width_class), ctypes.byref(ch), ctypes.byref(st)))
        return ch.value, st.value

    def set_tile_shape(self, width_class, chunk_rows=0, stages=0):
        """Pin a width class's tile shape (0: the default chunk of 64 rows, the deepest ring)."""
        self._check(lib().oais_batch_set_tile_shape(self._b, int(width_class), int(chunk_rows), int(stages)))

    def problem(self, p):
        return self._views[p]

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            lib().oais_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    __del__ = close
