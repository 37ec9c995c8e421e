"""Two shard contexts on one GPU against one context holding all particles: the shards'
merged round equals the full round (same particles through their counters)."""
import numpy as np
import pytest

from paper_2408_12057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
oais = pytest.importorskip("paper_2408_12057_gb300.oais")


@pytest.mark.parametrize("contraction", [0, 1])
def test_two_shards_equal_one_run(contraction):
    pr = W.logistic(n=1000, d=32, seed=3)
    N, T = 4096, 16
    beta = W.linear_schedule(T) ** 3
    eps = oais.default_step_sizes(pr, beta, oais.MALA)
    full = oais.OAIS(pr, oais.MALA, N, beta, T_max=32, eps=eps, seed=9, contraction=contraction)
    shards = [oais.OAIS(pr, oais.MALA, N // 2, beta, T_max=32, eps=eps, seed=9, contraction=contraction)
              for _ in range(2)]
    for k, s in enumerate(shards):
        s.set_shard(k * N // 2, N)
    for rnd in range(2):
        rf = full.round(32 if rnd == 0 else 16)
        merged = oais.merge_shard_stats([s.round_local() for s in shards])
        rs = [s.round_commit(32 if rnd == 0 else 16, merged) for s in shards]
        for r in rs:
            assert r["logZ"] == pytest.approx(rf["logZ"], rel=1e-12, abs=1e-10)
            assert r["Lambda_hat"] == pytest.approx(rf["Lambda_hat"], rel=1e-10)
        np.testing.assert_allclose(shards[0].schedule()[0], full.schedule()[0], rtol=1e-10, atol=1e-13)
        np.testing.assert_allclose(shards[1].schedule()[1], full.schedule()[1], rtol=1e-10)
        # particles: shard k holds particles [k N/2, (k+1) N/2) of the full run -- bit for bit in
        # the first round; later rounds run a schedule merged in a different summation order
        # (equal to ~1e-15), so the weights agree to rounding
        lw = full.particles()[0].cpu().numpy()
        for k, s in enumerate(shards):
            mine = s.particles()[0].cpu().numpy()
            if rnd == 0:
                np.testing.assert_array_equal(mine, lw[k * N // 2:(k + 1) * N // 2])
            else:
                np.testing.assert_allclose(mine, lw[k * N // 2:(k + 1) * N // 2], rtol=1e-12, atol=1e-9)
    with pytest.raises(oais.OAISError):
        shards[0].round(16)        # a shard cannot run a round on its own statistics
    for r in shards + [full]:
        r.close()


def test_checkpoint_resume_is_bit_identical():
    pr = W.logistic(n=400, d=8, seed=2)
    beta = W.linear_schedule(16) ** 3
    eps = oais.default_step_sizes(pr, beta, oais.MALA)
    a = oais.OAIS(pr, oais.MALA, 1000, beta, T_max=64, eps=eps, seed=4, adapt=True)
    a.round(32)
    blob = a.save_state()
    z_a = [a.round(64)["logZ"], a.round(64)["logZ"]]
    b = oais.OAIS(pr, oais.MALA, 1000, W.linear_schedule(3), T_max=64, seed=99, adapt=True)
    b.round(3)
    b.load_state(blob)
    with pytest.raises(oais.OAISError):
        b.logZ()                   # the round run before the load belongs to another state
    z_b = [b.round(64)["logZ"], b.round(64)["logZ"]]
    assert z_a == z_b
    # a blob is checked like the setters' arguments: a zero step size or a shard block past
    # the counter space is rejected and leaves the context as it was
    T = 32
    hdr = len(blob) - 8 * (2 * T + 1)
    eps_at = hdr + 8 * (T + 1)
    bad = bytearray(blob)
    bad[eps_at:eps_at + 8] = np.float64(0.0).tobytes()
    before = b.schedule()
    with pytest.raises(oais.OAISError):
        b.load_state(bytes(bad))
    after = b.schedule()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    bad = bytearray(blob)
    bad[16:24] = np.int64(1 << 33).tobytes()           # N_total beyond 2^32
    with pytest.raises(oais.OAISError):
        b.load_state(bytes(bad))
    wrong = oais.OAIS(pr, oais.MALA, 999, beta, T_max=64)
    with pytest.raises(oais.OAISError):
        wrong.load_state(blob)
    for r in (a, b, wrong):
        r.close()
