"""Process-pool jobs of the timing-optimisation parity test: oracle solves
and tight FP64 polishes (oracle/timing.py), one TO per job.  Kept apart from
the test module so that spawned workers import numpy and the oracle only."""
from __future__ import annotations

import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

import workloads as W
from oracle import timing as TM

N = 16
# tight FP64 polish: warm start at an answer, strong proximal term, no
# multipliers carried over (the exact local solution of the answer's basin)
POLISH = dict(eps_dual=1e-9, eps_primal=1e-11, eps_comp=1e-11, max_iters=2000, beta0=1e4, beta_max=1e8, rho0=1e-2,
              rho_min=1e-2)


def instance(i: int) -> dict:
    """push_l2 instances 0..3, then the straight push (goal 0.1 m ahead)."""
    return W.push_l2_instance(i) if i < 4 else W.push_l2_straight(0.1)


def solve(job):
    """job = (inst_index, modes, timing, max_iters, warm or None, extra opts);
    an inst_index of the form ("l4", seed) names a push_l4 instance (N = 20
    knots per segment) instead."""
    i, modes, timing, max_iters, warm, extra = job
    opts = dict(extra or {})
    if max_iters is not None:
        opts["max_iters"] = max_iters
    if isinstance(i, tuple):
        inst = W.push_l4_instance(i[1])
        n = int(inst["knots_per_segment"]) * len(modes)
    else:
        inst, n = instance(i), N
    z, lam, r = TM.solve(inst, tuple(modes), n, timing=timing, warm=warm, **opts)
    return z, lam, r


def run(jobs, workers=None):
    """Oracle jobs on a spawn pool with one BLAS thread per worker."""
    import multiprocessing as mp

    workers = workers or max(1, min(16, os.cpu_count() or 1, len(jobs)))
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(solve, jobs))
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def to_interleaved(tr: np.ndarray, Nmax: int = N, n: int | None = None) -> np.ndarray:
    """GPU record (x, y, theta, s, tau [Nmax+1]; f_n, f_t, sdot, h [Nmax])
    -> the oracle's interleaved z of an n-interval TO (n = Nmax unless
    given)."""
    n = Nmax if n is None else n
    x = tr[: 5 * (Nmax + 1)].reshape(5, Nmax + 1)
    u = tr[5 * (Nmax + 1): 5 * (Nmax + 1) + 4 * Nmax].reshape(4, Nmax)
    z = np.zeros(9 * n + 5)
    for k in range(n + 1):
        z[9 * k: 9 * k + 5] = x[:, k]
    for k in range(n):
        z[9 * k + 5: 9 * k + 9] = u[:, k]
    return z
