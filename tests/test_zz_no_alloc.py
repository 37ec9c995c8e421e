"""oais_logsumexp_noalloc, the allocation-free log-sum-exp, called through the C ABI.

Some callers cannot allocate device memory (inside a capture that must not allocate,
under an allocator that owns all device memory, in a fixed-budget loop); this entry
point keeps its scratch in a fixed device array inside the library.  It must give the
same result as oais_logsumexp, which takes caller scratch, on consecutive calls -- the
shared array keeps the previous call's contents, which must not leak into the next.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
oais = pytest.importorskip("paper_2408_12057_gb300.oais")

MAX_N = 16777216


def _noalloc():
    f = oais.lib().oais_logsumexp_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    return f


def _call(f, a):
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    st = f(ctypes.c_void_p(a.data_ptr()), a.numel(), ctypes.c_void_p(out.data_ptr()),
           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_scratch_entry_point_on_consecutive_calls():
    f = _noalloc()
    g = torch.Generator(device="cuda").manual_seed(7)
    # a large call first, then a smaller one: stale records of the first must not leak
    for n, scale in [(3_000_000, 40.0), (1_000, 3.0), (4096 * 7 + 5, 700.0)]:
        a = torch.randn(n, dtype=torch.float64, device="cuda", generator=g) * scale
        got = _call(f, a)
        ref = oais.logsumexp(a).cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


def _torch_ref(a):
    return np.array([torch.logsumexp(a, 0).item(), torch.logsumexp(2.0 * a, 0).item()])


def test_noalloc_matches_torch_up_to_its_limits():
    # the largest n the array covers (every one of its 4096 records written), a final record of
    # one element, and inputs with -inf entries (zero weights); each checked against
    # torch.logsumexp directly and against oais_logsumexp
    f = _noalloc()
    g = torch.Generator(device="cuda").manual_seed(11)
    for n in [MAX_N, 4096 * 9 + 1, 4097, 1]:
        a = torch.randn(n, dtype=torch.float64, device="cuda", generator=g) * 25.0
        if n > 1:
            a[::3] = float("-inf")
        got = _call(f, a)
        np.testing.assert_allclose(got, _torch_ref(a), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(got, oais.logsumexp(a).cpu().numpy(), rtol=1e-13, atol=1e-13)
        del a
    torch.cuda.empty_cache()


def test_noalloc_all_minus_infinity_gives_minus_infinity():
    # every weight zero: both sums are empty, log 0 = -inf (not NaN), on two calls in a row
    # and after a finite call has left its records in the array
    f = _noalloc()
    for n in [5, 4096 * 3 + 1]:
        a = torch.full((n,), float("-inf"), dtype=torch.float64, device="cuda")
        got = _call(f, a)
        assert np.all(got == -np.inf), got
        b = torch.linspace(-3.0, 2.0, n, dtype=torch.float64, device="cuda")
        np.testing.assert_allclose(_call(f, b), _torch_ref(b), rtol=1e-12, atol=1e-12)


def test_noalloc_rejects_sizes_beyond_its_array():
    f = _noalloc()
    a = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    # the size check happens before any launch, so a too-large n with a tiny buffer is safe
    st = f(ctypes.c_void_p(a.data_ptr()), MAX_N + 1, ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1
    assert b"MAX_N" in oais.lib().oais_last_error(None)
    st = f(ctypes.c_void_p(a.data_ptr()), 0, ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1
