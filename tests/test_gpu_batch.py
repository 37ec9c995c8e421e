"""Batched problems (many independent posteriors in one persistent tensor-core launch).

Every problem of a batch is the same computation as a single streamed context with its
problem index (random-number tag round | p << 16), so: each problem agrees with the FP64
oracle on X~ = f16(bf16(X)) particle by particle (the tolerances of the streamed form), and
with the single-context run bit for bit, in the first round and in later rounds replayed
from the captured graph; the ring depth changes no result, and a tile shape the autotuner
chose gives the same bits when pinned.
"""
import numpy as np
import pytest

import oracle as o
from paper_2408_12057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
oais = pytest.importorskip("paper_2408_12057_gb300.oais")

REL, ABS, XREL, TIE = 1e-5, 1e-4, 1e-4, 1e-3


def f16_of_bf16(X):
    b = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()
    return b.astype(np.float16).astype(np.float64)


def oracle_target(pr):
    return o.Target(pr.kind, f16_of_bf16(pr.X), pr.y, pr.ref_scale, pr.p0)


def view(v):
    logw, ell, x = v.particles()
    return dict(logw=logw.cpu().numpy().copy(), ell=ell.cpu().numpy().copy(),
                x=x.cpu().numpy().T.astype(np.float64).copy(), **v.stats())


def agree(g, r):
    close = lambda a, b, rt, at: np.abs(a - b) <= at + rt * np.abs(b)
    ok = (close(g["logw"], r["logw"], REL, ABS) & close(g["ell"], r["ell"], REL, ABS)
          & np.all(close(g["x"], r["x"], XREL, XREL), axis=-1))
    bad = ~ok & (r["margin"] > TIE)
    assert not bad.any(), f"{int(bad.sum())} particles disagree without a near-tie decision"
    return ok


def mixed_problems():
    # one problem per width class and a ragged chunk count each
    dims, ns = [8, 16, 32, 64, 128, 40], [100, 500, 777, 1300, 64, 257]
    return [W.logistic(n=n, d=d, seed=100 + i) for i, (n, d) in enumerate(zip(ns, dims))]


def test_batch_matches_oracle_per_problem():
    probs = mixed_problems()
    N, T = 300, 3
    beta = W.linear_schedule(T) ** 3
    eps = np.stack([oais.default_step_sizes(pr, beta, oais.MALA) for pr in probs])
    b = oais.OAISBatch(probs, oais.MALA, N, beta, eps=eps, seed=31)
    res = b.round(T)
    for p, pr in enumerate(probs):
        g = view(b.problem(p))
        r = o.asmc(oracle_target(pr), o.MALA, N, beta, eps[p], 31, tag=p << 16)
        ok = agree(g, r)
        assert ok.mean() >= 0.9
        assert res[p]["logZ"] == pytest.approx(float(np.logaddexp.reduce(g["logw"]) - np.log(N)), rel=1e-12)
    b.close()


def test_batch_equals_single_contexts_over_rounds():
    probs = mixed_problems()[:4]
    N, T = 256, 4
    beta = W.linear_schedule(T) ** 2
    eps = np.stack([oais.default_step_sizes(pr, beta, oais.MALA) for pr in probs])
    b = oais.OAISBatch(probs, oais.MALA, N, beta, eps=eps, seed=7)
    singles = []
    for p, pr in enumerate(probs):
        s = oais.OAIS(pr, oais.MALA, N, beta, eps=eps[p], seed=7, contraction=oais.CONTRACT_BF16_TC_STREAM)
        s.set_problem(p)
        singles.append(s)
    for rnd in range(3):   # rounds 2 and 3 replay the captured graph
        rb = b.round(T)
        for p, s in enumerate(singles):
            rs = s.round(T)
            g, h = view(b.problem(p)), view(s)
            assert np.array_equal(g["logw"], h["logw"]), (rnd, p)
            assert np.array_equal(g["log_ghat"], h["log_ghat"]), (rnd, p)
            assert rb[p]["logZ"] == rs["logZ"] and rb[p]["Lambda_hat"] == rs["Lambda_hat"]
            assert rb[p]["elbo"] == rs["elbo"] and np.isfinite(rs["elbo"])
            assert np.array_equal(b.problem(p).schedule()[0], s.schedule()[0])
    for s in singles:
        s.close()
    b.close()


def width_class(d):
    return 0 if d <= 16 else 1 if d <= 32 else 2 if d <= 64 else 3


@pytest.mark.parametrize("chunk", [128])
def test_batch_other_chunks_match_oracle_per_problem(chunk):
    # 128-row chunks for the classes d_pad 16, 32, 64 and the default 64 rows for d_pad 128 in
    # the same launch: every problem still agrees with the oracle particle by particle
    probs = mixed_problems()
    N, T = 300, 3
    beta = W.linear_schedule(T) ** 3
    eps = np.stack([oais.default_step_sizes(pr, beta, oais.MALA) for pr in probs])
    b = oais.OAISBatch(probs, oais.MALA, N, beta, eps=eps, seed=31)
    for c in (0, 1, 2):
        b.set_tile_shape(c, chunk_rows=chunk)
        assert b.tile_shape(c)[0] == chunk and b.tile_shape(c)[1] >= 2
    assert b.tile_shape(3)[0] == 64
    with pytest.raises(oais.OAISError):
        b.set_tile_shape(3, chunk_rows=chunk)   # d_pad 128: two K slabs, the image depends on the chunk
    res = b.round(T)
    for p, pr in enumerate(probs):
        g = view(b.problem(p))
        r = o.asmc(oracle_target(pr), o.MALA, N, beta, eps[p], 31, tag=p << 16)
        ok = agree(g, r)
        assert ok.mean() >= 0.9
        assert res[p]["logZ"] == pytest.approx(float(np.logaddexp.reduce(g["logw"]) - np.log(N)), rel=1e-12)
    b.close()


def test_batch_linreg_refuses_chunk128():
    probs = [W.linreg(n=300, d=16, seed=3), W.linreg(n=200, d=32, seed=4)]
    beta = W.linear_schedule(2)
    b = oais.OAISBatch(probs, oais.HMC, 128, beta, seed=3, leapfrog=2)
    with pytest.raises(oais.OAISError):
        b.set_tile_shape(0, chunk_rows=128)   # the chunk images carry y per chunk
    with pytest.raises(oais.OAISError):
        b.set_tile_shape(0, chunk_rows=32)    # not a built shape
    assert b.tile_shape(0)[0] == 64
    b.close()


def test_batch_autotune_shape_is_reproducible():
    # the autotuner's tile shapes, pinned on a fresh batch, give the same bits; classes that
    # kept 64-row chunks give the bits of an untuned batch (the ring depth changes no result)
    probs = mixed_problems()
    N, T = 512, 3
    beta = W.linear_schedule(T) ** 3
    a = oais.OAISBatch(probs, oais.MALA, N, beta, seed=5)
    ra = a.round(T)
    la = [view(a.problem(p))["logw"] for p in range(len(probs))]
    b = oais.OAISBatch(probs, oais.MALA, N, beta, seed=5)
    chosen = b.autotune(T_probe=2)
    assert all(c == 0 or 2 <= c <= 8 for c in chosen) and any(c > 0 for c in chosen)
    shapes = [b.tile_shape(c) for c in range(4)]
    for c, (ch, st) in enumerate(shapes):
        present = any(width_class(pr.d) == c for pr in probs)
        assert (ch in (64, 128) and st == chosen[c]) if present else (ch, st) == (0, 0)
    rb = b.round(T)
    lb = [view(b.problem(p))["logw"] for p in range(len(probs))]
    c2 = oais.OAISBatch(probs, oais.MALA, N, beta, seed=5)
    for c, (ch, st) in enumerate(shapes):
        if ch:
            c2.set_tile_shape(c, ch, st)
    rc = c2.round(T)
    for p, pr in enumerate(probs):
        assert np.array_equal(lb[p], view(c2.problem(p))["logw"]) and rb[p]["logZ"] == rc[p]["logZ"]
        if shapes[width_class(pr.d)][0] == 64:
            assert np.array_equal(la[p], lb[p]) and ra[p]["logZ"] == rb[p]["logZ"]
    a.close()
    b.close()
    c2.close()


def test_batch_linreg_hmc():
    # oracle parity of HMC trajectories where it is well conditioned (n <= 300: a relative
    # gradient error of 1e-5 moves a 3-leapfrog trajectory by far less than the tolerance);
    # every problem, the n = 1000 one included, equals its single-context run bit for bit
    shapes = [(300, 20), (130, 70), (200, 8), (1000, 8)]
    probs = [W.linreg(n=n, d=d, seed=n + d) for n, d in shapes]
    N, T = 200, 2
    beta = W.linear_schedule(T) ** 3
    eps = np.stack([oais.default_step_sizes(pr, beta, oais.HMC) for pr in probs])
    b = oais.OAISBatch(probs, oais.HMC, N, beta, eps=eps, seed=9, leapfrog=3)
    b.round(T)
    for p, pr in enumerate(probs):
        g = view(b.problem(p))
        s = oais.OAIS(pr, oais.HMC, N, beta, eps=eps[p], seed=9, leapfrog=3,
                      contraction=oais.CONTRACT_BF16_TC_STREAM)
        s.set_problem(p)
        s.round(T)
        assert np.array_equal(g["logw"], view(s)["logw"])
        s.close()
        if pr.n <= 300:
            r = o.asmc(oracle_target(pr), o.HMC, N, beta, eps[p], 9, tag=p << 16, leapfrog=3)
            assert agree(g, r).mean() >= 0.9
    b.close()


def test_batched_workload_full_size_sampled():
    # the batched workload at its full size: 64 logistic problems, n log-uniform in
    # [500, 50000], d in {8, ..., 128}, N = 2^14 each; a short schedule, sampled particles of
    # a few problems recomputed by the oracle
    probs = W.batched_logistic()
    N, T = 1 << 14, 3
    beta = W.linear_schedule(T) ** 3
    eps = np.stack([oais.default_step_sizes(pr, beta, oais.MALA) for pr in probs])
    b = oais.OAISBatch(probs, oais.MALA, N, beta, eps=eps, seed=12057)
    res = b.round(T)
    assert all(np.isfinite(r["logZ"]) for r in res)
    order = np.argsort([pr.n * (pr.d + 64) for pr in probs])
    for p in [int(order[0]), int(order[len(order) // 2]), int(order[-1])]:
        pr = probs[p]
        g = view(b.problem(p))
        tg = oracle_target(pr)
        idx = np.array([0, 128, N - 1, 4097])
        rs = [o.asmc(tg, o.MALA, 1, beta, eps[p], seed=12057, tag=p << 16, n_offset=int(n)) for n in idx]
        r = {k: np.array([q[k][0] for q in rs]) for k in ("logw", "ell", "margin")}
        r["x"] = np.stack([q["x"][0] for q in rs])
        gi = {k: g[k][idx] for k in ("logw", "ell", "x")}
        assert agree(gi, r).mean() >= 0.5
    b.close()
