"""The roofline's arithmetic per stage and iteration: bench.py's constants
are the oracle's counted values on the benchmarked workloads
(oracle/flop_count.py); the C counter is pinned by hand counts of single
steps and, on whole solves, by the independent numpy restatement of the
method (oracle/timing.py), whose count on fixed-step orders is the same
number."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import flop_count
from oracle import timing as TM


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


@pytest.mark.parametrize("seed,order", [(0, (0, 4)), (0, (12, 2)), (1, (3, 3)), (1, (2, 11))])
def test_c_count_equals_the_numpy_count(seed, order):
    # two implementations of the same method and counting conventions: the
    # C build (row scales recomputed per row, sweep in place) and the numpy
    # oracle (dense factorisation, failed sweeps located by LAPACK's pivot)
    inst = W.push_l2_instance(seed)
    _, t_py, w_py = TM.flops_per_stage_iteration([inst], [(0, order)], None)
    _, t_c, w_c = oracle.flops_per_stage_iteration([inst], np.zeros(1, np.int32), np.array([list(order)], np.uint8),
                                                   np.array([2], np.int32))
    assert w_py == w_c
    assert t_py == t_c


def test_counting_leaves_the_solve_unchanged():
    inst = W.push_l2_instance(2)
    tm = flop_count.timing_bounds(inst, 2)["binding"]
    z0, _, r0 = TM.solve(inst, (4, 7), timing=tm)
    TM.count_flops(True)
    z1, _, r1 = TM.solve(inst, (4, 7), timing=tm)
    assert TM.count_flops(False) > 0
    np.testing.assert_array_equal(z0, z1)
    assert r0["iters"] == r1["iters"]


def test_bench_timing_constants_are_the_oracle_count():
    import bench

    # a quarter of the sample (two orders per instance): within 10 %
    f, _, _ = flop_count.measure_timing("binding", per=2)
    assert f == pytest.approx(bench.TIMING_FLOP_PER_STAGE_ITER["binding"], rel=0.10)
