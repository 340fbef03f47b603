"""Flops per stage and solver iteration of the method, measured by the
oracle's counting build -- TEST INFRASTRUCTURE (part of the oracle).

The evaluator's roofline divides the method's arithmetic by the kernel's
time; this script measures that arithmetic once, on a seeded sample of the
benchmarked workload (4-segment pushing orders, N = 80, cold start): the
counting build of the FP64 oracle solves each order and counts the
floating-point operations of the method's steps (see comet_oracle.c), and
the total is divided by the sum over the orders of iterations x intervals.
bench.py carries the printed values as FLOP_PER_STAGE_ITER,
BIM_FLOP_PER_STAGE_ITER (the bimanual task, on random 1..6-segment orders)
and TIMING_FLOP_PER_STAGE_ITER (timing optimisation under the bench's two
duration bounds, counted by the numpy oracle of oracle/timing.py with the
same conventions; on fixed-step orders its count equals the C build's);
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


def timing_bounds(inst, L):
    """The bench's two duration bounds for an L-segment order of `inst`:
    room (h in [dt/2, 2 dt], T twice the fixed schedule's length) and
    binding (h in [dt/5, 3 dt], T = 3/4 of it)."""
    dt, n = inst["dt"], inst["knots_per_segment"] * L
    return {"slack": dict(h_min=0.5 * dt, h_max=2.0 * dt, T=2.0 * n * dt),
            "binding": dict(h_min=0.2 * dt, h_max=3.0 * dt, T=0.75 * n * dt)}


def _timing_job(job):
    from oracle import timing as TM

    seed, modes, bound, max_iters = job
    inst = W.push_l2_instance(seed)
    f, total, work = TM.flops_per_stage_iteration([inst], [(0, modes)], timing_bounds(inst, len(modes))[bound],
                                                  max_iters=max_iters)
    return total, work


def measure_timing(bound, seeds=tuple(range(3, 11)), per=6, max_iters=1500, workers=None):
    """Timing optimisation: `per` uniformly drawn 2-segment orders of each
    push_l2 instance (the bench's 2-segment leg uses seeds 3..10) under the
    named bound, solved by the numpy oracle on a spawn pool (one BLAS thread
    per worker).  Returns (flops per stage-iteration, total, work)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    jobs = []
    for s in seeds:
        rng = np.random.default_rng(3000 + s)
        jobs += [(s, tuple(int(m) for m in rng.integers(0, 12, 2)), bound, max_iters) for _ in range(per)]
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        n = workers or max(1, min(16, os.cpu_count() or 1, len(jobs)))
        with ProcessPoolExecutor(n, mp_context=mp.get_context("spawn")) as ex:
            res = list(ex.map(_timing_job, jobs))
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    total = sum(r[0] for r in res)
    work = sum(r[1] for r in res)
    return total / max(work, 1), total, work


if __name__ == "__main__":
    f, total, work = measure()
    print(f"pushing: {f:.1f} flops per stage-iteration ({total} flops over {work} stage-iterations)")
    f, total, work = measure_bimanual()
    print(f"bimanual: {f:.1f} flops per stage-iteration ({total} flops over {work} stage-iterations)")
    for bound in ("slack", "binding"):
        f, total, work = measure_timing(bound)
        print(f"timing ({bound}): {f:.1f} flops per stage-iteration ({total} flops over {work} stage-iterations)")
