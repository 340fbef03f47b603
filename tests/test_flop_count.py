"""The roofline's arithmetic per stage and iteration: bench.py's constant is
the oracle's counted value on the benchmarked workload (oracle/flop_count.py),
and the counter itself is pinned by hand counts of single steps."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import flop_count


def test_bench_constant_is_the_oracle_count():
    import bench

    f, total, work = flop_count.measure(instances=(0, 1), per=24)
    # a smaller sample of the same workload: within 5 % of the stored value
    assert f == pytest.approx(bench.FLOP_PER_STAGE_ITER, rel=0.05)
    f_full, _, _ = flop_count.measure()
    assert f_full == pytest.approx(bench.FLOP_PER_STAGE_ITER, rel=1e-3)


def test_counter_matches_hand_counts():
    # the default build counts nothing; the counting build's one-iteration
    # solve of a single-interval TO is at least the hand count of its dense
    # factorisation steps (7x7 Cholesky n^3/3-ish, five solves 2 n^2 each)
    inst = W.push_l2_instance(0)
    inst["knots_per_segment"] = 1
    seqs = np.zeros((1, 1), np.uint8)
    f, total, work = oracle.flops_per_stage_iteration([inst], np.zeros(1, np.int32), seqs, np.ones(1, np.int32),
                                                      opts=oracle.default_opts(max_iters=1))
    assert work == 1
    chol7 = sum(2 * j + 1 + (6 - j) * (2 * j + 1) for j in range(7))
    assert total >= chol7 + 5 * 2 * 49
    assert total < 20000


def test_bench_bimanual_constant_is_the_oracle_count():
    import bench

    f, total, work = flop_count.measure_bimanual()
    assert f == pytest.approx(bench.BIM_FLOP_PER_STAGE_ITER, rel=1e-3)
