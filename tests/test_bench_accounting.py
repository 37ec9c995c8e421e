"""The work counts behind the bench line's roofline fractions, checked against hand counts.

The mixture sweep's count is of the instructions a particle-step needs as written for the
instruction set (a packed fp32 pair or a wide multiply counts once); the logistic sweep's of
the contraction FLOP of one log L and gradient evaluation (X x and X^T r).
"""
import bench
from paper_2408_12057_gb300 import workloads as W


def test_mixture_instruction_count():
    d, K, moves = 16, 8, 2
    ops = bench.gmm_ops_per_particle_step(d, K, moves)
    # Philox4x32-10: 10 rounds of 2 wide multiplies and 2 three-input xors, 4 calls for the 16
    # normals and one for the MH uniform, per move
    assert ops["philox"] == moves * 5 * 10 * 4
    # per move: 17 uniforms (3 each), 16 normals (4 each), the packed proposal (2 per coordinate)
    assert ops["uniforms"] == moves * 17 * 3
    assert ops["box_muller"] == moves * 16 * 4
    assert ops["proposal"] == moves * 32
    # the density: K d / 2 packed differences + K d / 2 packed square-accumulates, 6 per
    # component (the exponent scaled to base 2, so one ex2), one log, |x|^2 in d / 2 packed
    # steps and 4 more
    assert ops["density"] == moves * (K * d + 6 * K + 1 + d // 2 + 4)
    assert ops["total"] == sum(v for k, v in ops.items() if k != "total") == 1138


def test_logistic_flop_count():
    pr = W.logistic()
    assert bench.algorithmic_flops_per_particle_step(pr) == 4.0 * 2000 * 32
