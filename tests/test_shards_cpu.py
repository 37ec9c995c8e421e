"""Sharding the OAIS particles over ranks (one exchange per round), without a GPU.

Particles are independent within an AIS round (Sec. 5.1.2), so a run of N particles can be
split into shards that own disjoint blocks of the particle counter space.  The only exchange
is the per-round statistics: the moments g_hat_{t,i} and the final weight sums are sums over
particles (merged by log-sum-exp), acceptance counts add.  Per-shard statistics here come from
the oracle; the exchange runs over torch.distributed with gloo, world size 2.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as o
from paper_2408_12057_gb300 import oais, workloads as W


def shard_stats(pr, N, beta, lo, hi, seed=7):
    r = o.asmc(o.Target(pr.kind, pr.X, pr.y, pr.ref_scale, pr.p0), o.MALA, hi - lo, beta, 0.3, seed,
               n_offset=lo)
    return {"log_ghat": r["log_ghat"], "accepted": r["accept"] * (hi - lo),
            "lse": np.array([o.logsumexp(r["logw"]), o.logsumexp(2 * r["logw"])])}


def problem():
    return W.logistic(n=120, d=4, seed=8), W.linear_schedule(12) ** 2


def test_merged_shards_equal_the_full_run():
    pr, beta = problem()
    N = 600
    full = shard_stats(pr, N, beta, 0, N)
    parts = [shard_stats(pr, N, beta, a, b) for a, b in [(0, 128), (128, 400), (400, 600)]]
    m = oais.merge_shard_stats(parts)
    np.testing.assert_allclose(m["log_ghat"], full["log_ghat"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(m["lse"], full["lse"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(m["accepted"], full["accepted"], rtol=0, atol=1e-9)
    # the next schedule (host Alg. 3 of the library) is the same
    a = oais.optimise_schedule(beta, m["log_ghat"], 20)[0]
    b = oais.optimise_schedule(beta, full["log_ghat"], 20)[0]
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pr, beta = problem()
        N = 512
        bounds = [(0, 256), (256, 512)]
        local = shard_stats(pr, N, beta, *bounds[rank])
        merged = oais.exchange_stats(local)
        full = shard_stats(pr, N, beta, 0, N)
        ok = (np.allclose(merged["log_ghat"], full["log_ghat"], rtol=1e-12, atol=1e-12)
              and np.allclose(merged["lse"], full["lse"], rtol=1e-12, atol=1e-12)
              and np.allclose(merged["accepted"], full["accepted"], atol=1e-9))
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


def test_gloo_exchange_two_ranks(tmp_path):
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        assert (tmp_path / f"rank{r}.txt").read_text() == "ok"


def test_merge_is_log_sum_exp_over_shards_with_empty_ones():
    # a shard whose weights are all zero contributes -inf sums and changes nothing; one shard
    # merges to itself; the result does not depend on how the particles were split
    rng = np.random.default_rng(4)
    T = 5
    a = {"log_ghat": rng.normal(size=(T, 3)), "accepted": rng.integers(0, 50, T).astype(float),
         "lse": rng.normal(size=2)}
    empty = {"log_ghat": np.full((T, 3), -np.inf), "accepted": np.zeros(T), "lse": np.full(2, -np.inf)}
    for parts in ([a], [a, empty], [empty, a, empty]):
        m = oais.merge_shard_stats(parts)
        np.testing.assert_array_equal(m["log_ghat"], a["log_ghat"])
        np.testing.assert_array_equal(m["lse"], a["lse"])
        np.testing.assert_array_equal(m["accepted"], a["accepted"])
    m = oais.merge_shard_stats([empty, empty])
    assert np.all(m["log_ghat"] == -np.inf) and np.all(m["lse"] == -np.inf)
    # two shards: log(e^a + e^b), also for values far apart
    b = {"log_ghat": a["log_ghat"] + 800.0, "accepted": a["accepted"], "lse": a["lse"] - 800.0}
    m = oais.merge_shard_stats([a, b])
    np.testing.assert_allclose(m["log_ghat"], a["log_ghat"] + 800.0, rtol=1e-15, atol=1e-12)
    np.testing.assert_allclose(m["lse"], a["lse"], rtol=1e-15, atol=1e-12)
    np.testing.assert_array_equal(m["accepted"], 2 * a["accepted"])


def test_default_step_sizes_follow_the_stated_rule():
    # eps_t = c / sqrt(1/s^2 + beta_t kappa) with the kernel's dimension factor c and the
    # family's curvature estimate kappa (oais_default_step_sizes in include/oais.h)
    beta = W.linear_schedule(10) ** 2
    cases = [
        (W.logistic(n=50, d=6, seed=1), lambda p: 0.25 * np.sum(p.X.astype(np.float64) ** 2) / p.d),
        (W.linreg(n=40, d=5, seed=2), lambda p: np.sum(p.X.astype(np.float64) ** 2) / p.d / p.p0 ** 2),
        (W.gauss_conj(d=4, seed=3), lambda p: 1.0 / p.p0 ** 2),
        (W.gmm(d=4, K=3, seed=4), lambda p: 1.0 / p.p0),
        (W.unid(m=1000, k=100), lambda p: 1000 / (0.1 * 0.9) * 0.01),
    ]
    for pr, kappa in cases:
        for move, c in [(oais.RWMH, 2.38 / np.sqrt(pr.d)), (oais.MALA, 1.2 * pr.d ** (-1 / 6)),
                        (oais.HMC, pr.d ** -0.25)]:
            got = oais.default_step_sizes(pr, beta, move)
            want = c / np.sqrt(1.0 / pr.ref_scale ** 2 + beta[1:] * kappa(pr))
            np.testing.assert_allclose(got, want, rtol=1e-12)
            assert np.all(np.diff(got) <= 0)          # tighter as the likelihood is switched on
