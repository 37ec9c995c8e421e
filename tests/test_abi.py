"""The C ABI on a machine without a GPU: the library builds, loads, exports every
symbol include/oais.h declares, validates arguments, and its host-only
OptimiseSchedule (Alg. 3) agrees with the oracle's independent implementation."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as o
from paper_2408_12057_gb300 import oais, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b((?:oais|asmc)_\w+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for core in ("oais_init", "oais_round", "oais_logZ", "oais_destroy", "oais_last_error"):
        assert core in names


@pytest.mark.parametrize("name", declared_functions())
def test_library_exports_declared_symbol(name):
    L = ctypes.CDLL(oais._build.build())
    assert hasattr(L, name), name


def test_optimise_schedule_matches_oracle():
    rng = np.random.default_rng(3)
    for T, Tn in [(1, 5), (7, 7), (64, 128), (300, 50)]:
        beta = np.concatenate([[0.0], np.sort(rng.uniform(0, 1, T - 1)), [1.0]])
        lg = np.zeros((T, 3))
        lg[:, 0] = rng.normal(0, 1, T)
        lg[:, 1] = lg[:, 0] + rng.normal(0, 1, T)
        D = rng.exponential(0.1, T) * (rng.uniform(size=T) > 0.1)
        lg[:, 2] = D + 2 * lg[:, 1] - lg[:, 0]
        a = oais.optimise_schedule(beta, lg, Tn)
        b = o.optimise_schedule(beta, lg, Tn)
        for x, y in zip(a, b):
            np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-14)


def test_validation_errors_need_no_gpu():
    L = oais.lib()
    pr = W.logistic(n=10, d=3)
    X = np.ascontiguousarray(pr.X, dtype=np.float32)
    y = np.ascontiguousarray(pr.y, dtype=np.float32)
    tg = oais._Target(oais.LOGREG, 3, 10, oais.DT_F32, X.ctypes.data, y.ctypes.data, 1.0, 1.0, 0)
    mv = oais._Move(oais.MALA, 1, 1, 0, 0)
    ctx = ctypes.c_void_p()
    bad = np.array([0.0, 0.7, 0.5, 1.0])      # not increasing
    st = L.oais_init(ctypes.byref(ctx), ctypes.byref(tg), ctypes.byref(mv), 100, bad.ctypes.data, 3, 3,
                     None, 1, None, 0, None)
    assert st == 1 and b"schedule" in L.oais_last_error(None)
    good = np.linspace(0, 1, 4)
    st = L.oais_init(ctypes.byref(ctx), ctypes.byref(tg), ctypes.byref(mv), 0, good.ctypes.data, 3, 3,
                     None, 1, None, 0, None)
    assert st == 1
    wide = oais._Target(oais.LOGREG, 300, 10, oais.DT_F32, X.ctypes.data, y.ctypes.data, 1.0, 1.0, 0)
    nbytes = ctypes.c_size_t()
    assert L.oais_workspace_bytes(ctypes.byref(wide), ctypes.byref(mv), 100, 4, ctypes.byref(nbytes)) == 6
    assert L.oais_workspace_bytes(ctypes.byref(tg), ctypes.byref(mv), 100, 4, ctypes.byref(nbytes)) == 0
    assert nbytes.value > 0
    assert L.oais_status_string(4) == b"non-finite log-weight or log-likelihood"


def test_budget_rule():
    # Alg. 2's Budget: (N, T) x sqrt(2) while N fits the cap, then T doubles with N kept
    from paper_2408_12057_gb300 import oais
    N, T, seen = 1024, 64, []
    for _ in range(8):
        N2, T2 = oais.budget(N, T, 4096, 4096)
        seen.append((N2, T2))
        if N < 4096:
            assert N2 % 128 == 0 and (N2 == 4096 or abs(N2 / N - 2 ** 0.5) < 0.1)
            assert abs(T2 / T - 2 ** 0.5) < 0.05
        else:
            assert N2 == N and T2 == min(2 * T, 4096)
        N, T = N2, T2
    assert seen == [(1408, 91), (2048, 129), (2944, 182), (4096, 257), (4096, 514), (4096, 1028),
                    (4096, 2056), (4096, 4096)]
    with pytest.raises(Exception):
        oais.budget(0, 10, 100, 100)


def test_batch_tile_shape_calls_validate_without_a_gpu():
    L = oais.lib()
    ch, st = ctypes.c_int32(7), ctypes.c_int32(7)
    assert L.oais_batch_tile_shape(None, 0, ctypes.byref(ch), ctypes.byref(st)) == 1   # OAIS_EINVAL
    assert L.oais_batch_set_tile_shape(None, 0, 32, 0) == 1
