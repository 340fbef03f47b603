"""Flops per stage and solver iteration of the method, measured by the
oracle's counting build -- TEST INFRASTRUCTURE (part of the oracle).

The evaluator's roofline divides the method's arithmetic by the kernel's
time; this script measures that arithmetic once, on a seeded sample of the
benchmarked workload (4-segment pushing orders, N = 80, cold start): the
counting build of the FP64 oracle solves each order and counts the
floating-point operations of the method's steps (see comet_oracle.c), and
the total is divided by the sum over the orders of iterations x intervals.
bench.py carries the printed values as FLOP_PER_STAGE_ITER and
BIM_FLOP_PER_STAGE_ITER (the bimanual task, on random 1..6-segment orders);
tests/test_flop_count.py re-measures them.

    python -m oracle.flop_count
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

SAMPLE_INSTANCES = (0, 1, 2, 3)
SAMPLE_ORDERS = 96  # per instance


def measure(instances=SAMPLE_INSTANCES, per=SAMPLE_ORDERS):
    """(flops per stage-iteration, total flops, stage-iterations) on the
    seeded sample: `per` uniformly drawn 4-segment orders of each instance."""
    insts = [W.push_l4_instance(s) for s in instances]
    seqs, idx = [], []
    for i, s in enumerate(instances):
        rng = np.random.default_rng(1000 + s)
        seqs.append(rng.integers(0, 12, (per, 4)))
        idx.append(np.full(per, i))
    seqs = np.concatenate(seqs).astype(np.uint8)
    idx = np.concatenate(idx).astype(np.int32)
    return oracle.flops_per_stage_iteration(insts, idx, seqs, np.full(len(idx), 4, np.int32))


def measure_bimanual(instances=tuple(range(8)), per=16):
    """The same for the bimanual task: `per` random orders of 1..6 segments
    of each instance (bench.py's bimanual leg draws the same kind)."""
    insts = [W.bimanual_instance(s) for s in instances]
    seqs, idx, lens = [], [], []
    for i, s in enumerate(instances):
        rng = np.random.default_rng(2000 + s)
        for _ in range(per):
            L = int(rng.integers(1, 7))
            q = np.zeros(6, np.uint16)
            q[:L] = rng.integers(0, 507, L)
            seqs.append(q)
            idx.append(i)
            lens.append(L)
    return oracle.bim_flops_per_stage_iteration(insts, np.array(idx, np.int32), seqs, np.array(lens, np.int32))


if __name__ == "__main__":
    f, total, work = measure()
    print(f"pushing: {f:.1f} flops per stage-iteration ({total} flops over {work} stage-iterations)")
    f, total, work = measure_bimanual()
    print(f"bimanual: {f:.1f} flops per stage-iteration ({total} flops over {work} stage-iterations)")
