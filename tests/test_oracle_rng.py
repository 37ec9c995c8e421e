"""Pins for the oracle's random numbers: Philox4x32-10 known answers (SC'11 /
Random123), the exactness of the uniform map and the law of the normals."""
import os

import numpy as np
import pytest
from scipy import stats

import oracle as o

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(v, 16) for v in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    assert list(o.philox4x32_10(ctr, key)) == expect


def test_uniform_map_is_open_interval_and_exact():
    # u = ((r >> 9) + 0.5) 2^-23 is exactly representable in fp32 and never 0 or 1
    for r in [0, 1, 511, 512, 0x7FFFFFFF, 0xFFFFFFFF]:
        u = o.u01(r)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u
    assert o.u01(0) == 0.5 / 2 ** 23
    assert o.u01(0xFFFFFFFF) == 1.0 - 0.5 / 2 ** 23


def test_normals_law():
    z = np.concatenate([o.normals(7, n, 3, 1, 0, 16) for n in range(4000)])
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 4 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_normals_streams_differ_by_counter():
    a = o.normals(1, 5, 2, 0, 0, 8)
    assert not np.allclose(a, o.normals(1, 6, 2, 0, 0, 8))   # particle
    assert not np.allclose(a, o.normals(1, 5, 3, 0, 0, 8))   # step
    assert not np.allclose(a, o.normals(1, 5, 2, 1, 0, 8))   # move
    assert not np.allclose(a, o.normals(1, 5, 2, 0, 1, 8))   # round tag
    assert not np.allclose(a, o.normals(2, 5, 2, 0, 0, 8))   # seed
    # the first d components do not depend on how many are asked for
    assert np.array_equal(o.normals(1, 5, 2, 0, 0, 13)[:8], a)


def test_mh_uniform_law():
    u = np.array([o.mh_uniform(3, n, 1, 0, 0) for n in range(5000)])
    assert stats.kstest(u, "uniform").pvalue > 1e-4
