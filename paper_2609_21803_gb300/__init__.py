"""GB300-native CoMET hot path: thin Python binding of ``libcomet.so``.

Every entry point of ``include/comet.h`` is exposed under the same name and
only marshals arguments (ctypes); all computation runs in the CUDA library.
The library is built in-tree by ``paper_2609_21803_gb300.build.build()``
(nvcc, sm_103a).  Importing this package never falls back to another
implementation: if the library is missing, ``lib()`` raises.

Pointer arguments accept torch tensors (their ``data_ptr()``, host or CUDA),
numpy arrays (host), raw integer addresses or ``None``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

MAX_SEGMENTS = 16
TO_CONVERGED, TO_MAX_ITER, TO_INFEASIBLE, TO_FACTOR_FAIL, TO_NONFINITE = range(5)
OK = 0

_lock = threading.Lock()
_lib = None


class InstanceDesc(ctypes.Structure):
    _fields_ = [
        ("task", ctypes.c_int32), ("knots_per_segment", ctypes.c_int32),
        ("max_segments", ctypes.c_int32), ("n_modes", ctypes.c_int32),
        ("side_x", ctypes.c_double), ("side_y", ctypes.c_double), ("c_ls", ctypes.c_double),
        ("mu", ctypes.c_double), ("dt", ctypes.c_double), ("kappa", ctypes.c_double),
        ("start", ctypes.c_double * 3), ("goal", ctypes.c_double * 3),
        ("w_terminal", ctypes.c_double), ("w_control", ctypes.c_double),
        ("mass", ctypes.c_double), ("ground_mu", ctypes.c_double),
    ]


class SolverOpts(ctypes.Structure):
    _fields_ = [
        ("max_iters", ctypes.c_int32), ("ref_iters", ctypes.c_int32),
        ("eps_feas", ctypes.c_double), ("eps_primal", ctypes.c_double), ("eps_dual", ctypes.c_double),
        ("eps_comp", ctypes.c_double), ("merit_mu", ctypes.c_double),
        ("beta0", ctypes.c_double), ("beta_max", ctypes.c_double), ("beta_ref", ctypes.c_double),
        ("rho0", ctypes.c_double), ("rho_min", ctypes.c_double),
        ("precision_flags", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("refine_beta", ctypes.c_double),
    ]


class PlanOpts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("batch", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("k_ref", ctypes.c_int32), ("budget", ctypes.c_int64), ("ref_iters", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("radius", ctypes.c_int32), ("grammar", ctypes.c_int32)]


GRAMMAR_NONE, GRAMMAR_PUSH = 0, 1   # neighbourhood rules (comet_frontier_create_ex)
MODE_FREE = 12                      # free motion in the 13-mode pushing alphabet


class ModeSeq(ctypes.Structure):
    _fields_ = [("instance", ctypes.c_int32), ("len", ctypes.c_uint8),
                ("pad", ctypes.c_uint8 * 3), ("modes", ctypes.c_uint16 * MAX_SEGMENTS)]


class PlanResult(ctypes.Structure):
    _fields_ = [("best", ModeSeq), ("best_cost", ctypes.c_float), ("best_viol", ctypes.c_float),
                ("best_status", ctypes.c_int32), ("rounds_run", ctypes.c_int32), ("evaluations", ctypes.c_int64),
                ("explore_ms", ctypes.c_float), ("refine_ms", ctypes.c_float)]


class LaunchConfig(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("max_blocks_per_sm", ctypes.c_int32), ("unroll", ctypes.c_int32)]


class ProposalDesc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("rows_cap", ctypes.c_int32), ("dataset_cap", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("lambda_w", ctypes.c_double), ("warm_mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class AdamWOpts(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("weight_decay", ctypes.c_double)]


class GemmEpilogue(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k_splits", ctypes.c_int32), ("bias", ctypes.c_void_p),
                ("out_f32", ctypes.c_void_p), ("ld_f32", ctypes.c_int64),
                ("out_bf16", ctypes.c_void_p), ("ld_bf16", ctypes.c_int64),
                ("out_bf16_t", ctypes.c_void_p), ("ld_bf16_t", ctypes.c_int64),
                ("z_in", ctypes.c_void_p), ("ld_z", ctypes.c_int64)]


GEMM_STORE, GEMM_BIAS_GELU, GEMM_GELU_GRAD, GEMM_ATOMIC_ADD = 0, 1, 2, 3


class TimingOpts(ctypes.Structure):
    _fields_ = [("h_min", ctypes.c_double), ("h_max", ctypes.c_double), ("T_max", ctypes.c_double)]


class MctsOpts(ctypes.Structure):
    _fields_ = [("n_modes", ctypes.c_int32), ("l_max", ctypes.c_int32), ("grammar", ctypes.c_int32),
                ("reward", ctypes.c_int32), ("max_evals", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("c_uct", ctypes.c_double), ("eps_feas", ctypes.c_double), ("merit_mu", ctypes.c_double),
                ("max_ms", ctypes.c_double)]


class MctsStats(ctypes.Structure):
    _fields_ = [("evaluations", ctypes.c_int64), ("tree_nodes", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("exhausted", ctypes.c_int32), ("reserved", ctypes.c_int32), ("best", ctypes.c_double)]


MCTS_REWARD_FEASIBLE, MCTS_REWARD_MERIT = 0, 1

MODE_SEQ_DTYPE = np.dtype([("instance", "<i4"), ("len", "u1"), ("pad", "u1", (3,)), ("modes", "<u2", (MAX_SEGMENTS,))])
MODE_SEQ_BYTES = 40
assert MODE_SEQ_DTYPE.itemsize == ctypes.sizeof(ModeSeq) == MODE_SEQ_BYTES

# exported symbols of include/comet.h
EXPORTS = (
    "comet_default_opts", "comet_problem_create", "comet_problem_destroy", "comet_traj_stride",
    "comet_eval_modes", "comet_eval_modes_budget", "comet_eval_stats", "comet_eval_check",
    "comet_debug_stall_staging", "comet_mode_code",
    "comet_eval_modes_timed",
    "comet_last_error", "comet_eval_modes_noalloc", "comet_fp32_fma_peak", "comet_fp32_fma_peak_threads",
    "comet_frontier_create", "comet_frontier_destroy", "comet_frontier_add", "comet_expand",
    "comet_frontier_next", "comet_frontier_size", "comet_frontier_best", "comet_frontier_copy_next",
    "comet_frontier_save", "comet_frontier_load",
    "comet_default_plan_opts", "comet_plan",
    # include/comet_proposal.h
    "comet_default_proposal_desc", "comet_default_adamw_opts", "comet_proposal_create", "comet_proposal_destroy",
    "comet_proposal_dims", "comet_proposal_set_params", "comet_proposal_get_params", "comet_proposal_features",
    "comet_proposal_save", "comet_proposal_load",
    "comet_proposal_forward", "comet_proposal_train_batch", "comet_proposal_add_samples",
    "comet_proposal_dataset_size", "comet_proposal_dataset_rows", "comet_proposal_train", "comet_proposal_predict", "comet_proposal_prune",
    "comet_gemm_bf16", "comet_plan_learned",
    "comet_get_launch_config", "comet_set_launch_config", "comet_autotune", "comet_proposal_time_forward",
    "comet_plan_batch", "comet_plan_batch_learned", "comet_frontier_create_ex", "comet_sample_orders",
    # include/comet_mcts.h
    "comet_mcts_default_opts", "comet_mcts_create", "comet_mcts_destroy", "comet_mcts_ask", "comet_mcts_tell",
    "comet_mcts_get_stats", "comet_mcts_best", "comet_plan_mcts",
)


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False):
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"libcomet.so is not built ({path}); run paper_2609_21803_gb300.build.build()")
                path = _build.build()
            L = ctypes.CDLL(path)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            L.comet_default_opts.argtypes = [ctypes.POINTER(SolverOpts)]
            L.comet_problem_create.argtypes = [ctypes.POINTER(InstanceDesc), i32, ctypes.POINTER(SolverOpts), vp,
                                               ctypes.POINTER(vp)]
            L.comet_problem_destroy.argtypes = [vp]
            L.comet_traj_stride.argtypes = [vp]
            L.comet_traj_stride.restype = i64
            L.comet_eval_modes.argtypes = [vp, vp, i64, vp, vp, vp, vp]
            L.comet_eval_modes_budget.argtypes = [vp, vp, i64, vp, i32, vp, vp, vp]
            L.comet_eval_stats.argtypes = [vp, vp, vp, vp, vp]
            L.comet_eval_check.argtypes = [vp, vp]
            L.comet_debug_stall_staging.argtypes = [vp, i32]
            L.comet_eval_modes_timed.argtypes = [vp, ctypes.POINTER(TimingOpts), vp, i64, vp, i32, vp, vp, vp]
            L.comet_fp32_fma_peak.argtypes = [vp, i32, vp, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]
            L.comet_fp32_fma_peak_threads.argtypes = []
            L.comet_fp32_fma_peak_threads.restype = i32
            L.comet_eval_modes_noalloc.argtypes = [ctypes.POINTER(InstanceDesc), i32, ctypes.POINTER(SolverOpts), vp,
                                                   vp, i64, vp, vp, vp, vp]
            L.comet_frontier_create.argtypes = [vp, i32, i64, i32, i32, ctypes.POINTER(vp)]
            L.comet_frontier_create_ex.argtypes = [vp, i32, i64, i32, i32, i32, i32, ctypes.POINTER(vp)]
            L.comet_sample_orders.argtypes = [vp, i32, ctypes.c_uint64, i64, i64, i32, vp]
            L.comet_frontier_destroy.argtypes = [vp]
            L.comet_frontier_add.argtypes = [vp, vp, i64, vp, vp]
            L.comet_expand.argtypes = [vp, vp, i32]
            L.comet_frontier_next.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(i64)]
            L.comet_frontier_size.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32)]
            L.comet_frontier_copy_next.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
            L.comet_frontier_best.argtypes = [vp, i32, vp, vp]
            L.comet_frontier_save.argtypes = [vp, ctypes.c_char_p]
            L.comet_frontier_load.argtypes = [vp, ctypes.c_char_p]
            L.comet_default_plan_opts.argtypes = [ctypes.POINTER(PlanOpts)]
            L.comet_plan.argtypes = [vp, i32, vp, i64, ctypes.POINTER(PlanOpts), ctypes.POINTER(PlanResult), vp]
            L.comet_mode_code.argtypes = [ctypes.POINTER(ModeSeq), i32]
            L.comet_mode_code.restype = ctypes.c_uint64
            L.comet_last_error.restype = ctypes.c_char_p
            L.comet_default_proposal_desc.argtypes = [ctypes.POINTER(ProposalDesc)]
            L.comet_default_proposal_desc.restype = None
            L.comet_default_adamw_opts.argtypes = [ctypes.POINTER(AdamWOpts)]
            L.comet_default_adamw_opts.restype = None
            L.comet_proposal_create.argtypes = [vp, ctypes.POINTER(ProposalDesc), ctypes.POINTER(vp)]
            L.comet_proposal_destroy.argtypes = [vp]
            L.comet_proposal_dims.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                              ctypes.POINTER(i64)]
            L.comet_proposal_set_params.argtypes = [vp, vp]
            L.comet_proposal_get_params.argtypes = [vp, vp, vp]
            L.comet_proposal_save.argtypes = [vp, ctypes.c_char_p]
            L.comet_proposal_load.argtypes = [vp, ctypes.c_char_p]
            L.comet_proposal_features.argtypes = [vp, vp, i64, vp]
            L.comet_proposal_forward.argtypes = [vp, vp, i64, vp]
            L.comet_proposal_train_batch.argtypes = [vp, vp, vp, vp, i64, ctypes.POINTER(AdamWOpts),
                                                     ctypes.POINTER(ctypes.c_float)]
            L.comet_proposal_add_samples.argtypes = [vp, vp, i64, vp, vp, vp, vp]
            L.comet_proposal_dataset_size.argtypes = [vp, ctypes.POINTER(i64)]
            L.comet_proposal_dataset_rows.argtypes = [vp, i64, i64, vp, vp, vp]
            L.comet_proposal_train.argtypes = [vp, i64, i32, ctypes.POINTER(AdamWOpts), ctypes.c_uint64, vp]
            L.comet_proposal_predict.argtypes = [vp, vp, i64, vp, vp]
            L.comet_proposal_prune.argtypes = [vp, vp, i32, vp]
            L.comet_get_launch_config.argtypes = [vp, ctypes.POINTER(LaunchConfig)]
            L.comet_set_launch_config.argtypes = [vp, ctypes.POINTER(LaunchConfig)]
            L.comet_autotune.argtypes = [vp, vp, i64, i32, ctypes.POINTER(LaunchConfig), vp,
                                         ctypes.POINTER(i32)]
            L.comet_proposal_time_forward.argtypes = [vp, vp, i64, i32, ctypes.POINTER(ctypes.c_float)]
            L.comet_plan_batch.argtypes = [vp, i32, vp, vp, vp, ctypes.POINTER(PlanOpts), vp]
            L.comet_plan_batch_learned.argtypes = [vp, i32, vp, vp, vp, ctypes.POINTER(PlanOpts), vp, vp]
            L.comet_plan_learned.argtypes = [vp, i32, vp, i64, ctypes.POINTER(PlanOpts), vp,
                                             ctypes.POINTER(PlanResult), vp]
            L.comet_gemm_bf16.argtypes = [vp, i64, vp, i64, i64, i32, i32, ctypes.POINTER(GemmEpilogue), vp]
            L.comet_mcts_default_opts.argtypes = [ctypes.POINTER(MctsOpts)]
            L.comet_mcts_create.argtypes = [ctypes.POINTER(MctsOpts), ctypes.POINTER(vp)]
            L.comet_mcts_destroy.argtypes = [vp]
            L.comet_mcts_ask.argtypes = [vp, i32, i64, vp, ctypes.POINTER(i64)]
            L.comet_mcts_tell.argtypes = [vp, vp, vp, i64]
            L.comet_mcts_get_stats.argtypes = [vp, ctypes.POINTER(MctsStats)]
            L.comet_mcts_best.argtypes = [vp, i64, vp, vp, ctypes.POINTER(i64)]
            L.comet_plan_mcts.argtypes = [vp, i32, ctypes.POINTER(MctsOpts), i64, ctypes.POINTER(PlanOpts),
                                          ctypes.POINTER(PlanResult), vp]
            for name in EXPORTS:
                if name not in ("comet_traj_stride", "comet_mode_code", "comet_last_error",
                                "comet_default_proposal_desc", "comet_default_adamw_opts"):
                    getattr(L, name).restype = i32
            _lib = L
    return _lib


class CometError(RuntimeError):
    pass


def _check(rc: int):
    if rc != OK:
        raise CometError(f"comet status {rc}: {lib().comet_last_error().decode()}")


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


# ------------------------------------------------------------------ C ABI

def comet_default_opts() -> SolverOpts:
    o = SolverOpts()
    _check(lib().comet_default_opts(ctypes.byref(o)))
    return o


def make_instance_desc(d: dict) -> InstanceDesc:
    s = InstanceDesc()
    s.task = int(d.get("task", 0))
    s.knots_per_segment = int(d["knots_per_segment"])
    s.max_segments = int(d["max_segments"])
    s.n_modes = int(d.get("n_modes", 12))
    for f in ("side_x", "side_y", "c_ls", "mu", "dt", "w_terminal", "w_control"):
        setattr(s, f, float(d[f]))
    s.kappa = float(d.get("kappa", 1.0))
    for i in range(3):
        s.start[i] = float(d["start"][i])
        s.goal[i] = float(d["goal"][i])
    s.mass = float(d.get("mass", 0.0))
    s.ground_mu = float(d.get("ground_mu", 0.0))
    return s


def comet_problem_create(instances, opts=None, cuda_stream=None) -> int:
    """instances: list of dicts (or InstanceDesc); opts: SolverOpts, dict or
    None; cuda_stream: integer cudaStream_t handle or None.  Returns the
    problem handle (an integer address)."""
    descs = [x if isinstance(x, InstanceDesc) else make_instance_desc(x) for x in instances]
    arr = (InstanceDesc * len(descs))(*descs)
    o = None
    if opts is not None:
        if isinstance(opts, dict):
            oo = comet_default_opts()
            for k, v in opts.items():
                setattr(oo, k, v)
            opts = oo
        o = ctypes.byref(opts)
    h = ctypes.c_void_p()
    _check(lib().comet_problem_create(arr, len(descs), o, cuda_stream, ctypes.byref(h)))
    return h.value


def comet_problem_destroy(problem: int):
    _check(lib().comet_problem_destroy(problem))


def comet_traj_stride(problem: int) -> int:
    return int(lib().comet_traj_stride(problem))


def comet_eval_modes(problem, mode_seqs, n, warm_starts, out_cost, out_traj, out_status):
    _check(lib().comet_eval_modes(problem, _ptr(mode_seqs), int(n), _ptr(warm_starts), _ptr(out_cost),
                                  _ptr(out_traj), _ptr(out_status)))


def comet_eval_modes_budget(problem, mode_seqs, n, warm_starts, max_iters, out_cost, out_traj, out_status):
    _check(lib().comet_eval_modes_budget(problem, _ptr(mode_seqs), int(n), _ptr(warm_starts), int(max_iters),
                                         _ptr(out_cost), _ptr(out_traj), _ptr(out_status)))


def comet_eval_stats(problem, out_viol, out_merit, out_iters, out_stat):
    _check(lib().comet_eval_stats(problem, _ptr(out_viol), _ptr(out_merit), _ptr(out_iters), _ptr(out_stat)))


def comet_eval_check(problem) -> int:
    """The last evaluator launch's device flag (0 nothing, 1 malformed order,
    2 a bounded wait gave up); raises CometError (COMET_ERR_TIMEOUT) on 2."""
    flag = ctypes.c_int32(0)
    st = lib().comet_eval_check(problem, ctypes.byref(flag))
    if st != 0:
        _check(st)
    return int(flag.value)


def comet_debug_stall_staging(problem, on: bool):
    _check(lib().comet_debug_stall_staging(problem, int(bool(on))))


def comet_eval_modes_timed(problem, timing: dict, mode_seqs, n, warm_starts, max_iters, out_cost, out_traj,
                           out_status):
    """Timing optimisation (comet_eval_modes_timed); timing: {"h_min",
    "h_max", "T_max"}; every array device memory; trajectory records of
    9 N_max + 5 floats (x, y, theta, s, tau [N_max + 1], f_n, f_t, sdot, h
    [N_max])."""
    t = TimingOpts(float(timing["h_min"]), float(timing["h_max"]), float(timing["T_max"]))
    _check(lib().comet_eval_modes_timed(problem, ctypes.byref(t), _ptr(mode_seqs), int(n), _ptr(warm_starts),
                                        int(max_iters), _ptr(out_cost), _ptr(out_traj), _ptr(out_status)))


def comet_fp32_fma_peak(cuda_stream, iters: int, scratch) -> tuple[float, float]:
    """Measured FP32 FMA throughput (TFLOP/s) and the kernel time (ms);
    scratch: device buffer of comet_fp32_fma_peak_threads() floats."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().comet_fp32_fma_peak(cuda_stream, int(iters), _ptr(scratch), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def comet_fp32_fma_peak_threads() -> int:
    return int(lib().comet_fp32_fma_peak_threads())


def comet_eval_modes_noalloc(instances, opts, cuda_stream, mode_seqs, n, warm_starts, out_cost, out_traj,
                             out_status):
    """The allocation-free entry point: descriptors from the host, every
    array in device memory (see include/comet.h)."""
    descs = [x if isinstance(x, InstanceDesc) else make_instance_desc(x) for x in instances]
    arr = (InstanceDesc * len(descs))(*descs)
    o = None
    if opts is not None:
        if isinstance(opts, dict):
            oo = comet_default_opts()
            for k, v in opts.items():
                setattr(oo, k, v)
            opts = oo
        o = ctypes.byref(opts)
    _check(lib().comet_eval_modes_noalloc(arr, len(descs), o, cuda_stream, _ptr(mode_seqs), int(n),
                                          _ptr(warm_starts), _ptr(out_cost), _ptr(out_traj), _ptr(out_status)))


def comet_frontier_create(problem, instance: int, capacity: int, batch: int, k_max: int, radius: int = 1,
                          grammar: int = GRAMMAR_NONE) -> int:
    h = ctypes.c_void_p()
    _check(lib().comet_frontier_create_ex(problem, instance, capacity, batch, k_max, radius, grammar, ctypes.byref(h)))
    return h.value


def comet_frontier_destroy(frontier):
    _check(lib().comet_frontier_destroy(frontier))


def comet_frontier_add(frontier, seqs, n, cost, viol):
    _check(lib().comet_frontier_add(frontier, _ptr(seqs), int(n), _ptr(cost), _ptr(viol)))


def comet_expand(problem, frontier, k: int):
    _check(lib().comet_expand(problem, frontier, int(k)))


def comet_frontier_next(frontier):
    """(device address of the next batch, its size)."""
    p = ctypes.c_void_p()
    n = ctypes.c_int64()
    _check(lib().comet_frontier_next(frontier, ctypes.byref(p), ctypes.byref(n)))
    return p.value, n.value


def comet_frontier_copy_next(frontier, out, cap: int) -> int:
    n = ctypes.c_int64()
    _check(lib().comet_frontier_copy_next(frontier, _ptr(out), int(cap), ctypes.byref(n)))
    return n.value


def frontier_next_orders(frontier, cap: int):
    """The next batch as a list of mode tuples (host copy)."""
    buf = np.zeros(cap, dtype=MODE_SEQ_DTYPE)
    n = comet_frontier_copy_next(frontier, buf, cap)
    return [tuple(int(m) for m in r["modes"][: r["len"]]) for r in buf[:n]]


def comet_frontier_size(frontier):
    n = ctypes.c_int64()
    e = ctypes.c_int32()
    _check(lib().comet_frontier_size(frontier, ctypes.byref(n), ctypes.byref(e)))
    return n.value, e.value


def comet_frontier_save(frontier, path):
    """V's codes and merits and the pending batch to a checkpoint file."""
    _check(lib().comet_frontier_save(frontier, os.fsencode(path)))


def comet_frontier_load(frontier, path):
    """Resume a frontier of the same instance and rule from a checkpoint."""
    _check(lib().comet_frontier_load(frontier, os.fsencode(path)))


def comet_frontier_best(frontier, k: int):
    codes = np.zeros(k, dtype=np.uint64)
    merit = np.zeros(k, dtype=np.float32)
    _check(lib().comet_frontier_best(frontier, int(k), codes.ctypes.data, merit.ctypes.data))
    return codes, merit


def comet_default_plan_opts() -> PlanOpts:
    o = PlanOpts()
    _check(lib().comet_default_plan_opts(ctypes.byref(o)))
    return o


def comet_plan(problem, instance: int, seeds, n_seeds: int, opts=None, out_traj=None, proposal=None) -> dict:
    """Algorithm 1 on the device (see include/comet.h; with `proposal`,
    comet_plan_learned of include/comet_proposal.h); opts: PlanOpts, dict or
    None.  Returns the result as a dict."""
    if opts is None or isinstance(opts, dict):
        o = comet_default_plan_opts()
        for k, v in (opts or {}).items():
            setattr(o, k, v)
        opts = o
    r = PlanResult()
    if proposal is None:
        _check(lib().comet_plan(problem, int(instance), _ptr(seeds), int(n_seeds), ctypes.byref(opts),
                                ctypes.byref(r), _ptr(out_traj)))
    else:
        _check(lib().comet_plan_learned(problem, int(instance), _ptr(seeds), int(n_seeds), ctypes.byref(opts),
                                        proposal, ctypes.byref(r), _ptr(out_traj)))
    best = tuple(int(r.best.modes[i]) for i in range(r.best.len))
    return {"best": best, "best_cost": r.best_cost, "best_viol": r.best_viol, "best_status": r.best_status,
            "rounds_run": r.rounds_run, "evaluations": r.evaluations, "explore_ms": r.explore_ms,
            "refine_ms": r.refine_ms}


def comet_plan_batch(problem, instances, seeds_per_instance, opts=None, proposal=None) -> list:
    """Algorithm 1 for several instances at once (comet_plan_batch; with
    `proposal`, comet_plan_batch_learned of include/comet_proposal.h);
    seeds_per_instance: a list (one per instance) of lists of mode tuples."""
    if opts is None or isinstance(opts, dict):
        o = comet_default_plan_opts()
        for k, v in (opts or {}).items():
            setattr(o, k, v)
        opts = o
    inst = np.ascontiguousarray(instances, dtype=np.int32)
    offs = np.zeros(len(inst) + 1, np.int64)
    allseq, idx = [], []
    for i, seeds in enumerate(seeds_per_instance):
        allseq += list(seeds)
        idx += [int(inst[i])] * len(seeds)
        offs[i + 1] = offs[i] + len(seeds)
    packed = pack_mode_seqs(allseq, np.array(idx, np.int32))
    res = (PlanResult * len(inst))()
    if proposal is None:
        _check(lib().comet_plan_batch(problem, len(inst), inst.ctypes.data, packed.ctypes.data, offs.ctypes.data,
                                      ctypes.byref(opts), res))
    else:
        _check(lib().comet_plan_batch_learned(problem, len(inst), inst.ctypes.data, packed.ctypes.data,
                                              offs.ctypes.data, ctypes.byref(opts), proposal, res))
    out = []
    for r in res:
        out.append({"best": tuple(int(r.best.modes[i]) for i in range(r.best.len)), "best_cost": r.best_cost,
                    "best_viol": r.best_viol, "best_status": r.best_status, "rounds_run": r.rounds_run,
                    "evaluations": r.evaluations, "explore_ms": r.explore_ms, "refine_ms": r.refine_ms})
    return out


def comet_sample_orders(problem, instance: int, seed: int, first: int, n: int, grammar: int = GRAMMAR_NONE):
    """Orders first .. first + n - 1 of the uniform sample (comet_sample_orders),
    as a host array of packed records."""
    out = np.zeros(n, dtype=MODE_SEQ_DTYPE)
    _check(lib().comet_sample_orders(problem, instance, seed, first, n, grammar, out.ctypes.data))
    return out


def comet_mcts_default_opts(**over) -> MctsOpts:
    o = MctsOpts()
    _check(lib().comet_mcts_default_opts(ctypes.byref(o)))
    for k, v in over.items():
        setattr(o, k, v)
    return o


class Mcts:
    """The host tree search of include/comet_mcts.h (ask / tell)."""

    def __init__(self, **opts):
        self.opts = comet_mcts_default_opts(**opts)
        h = ctypes.c_void_p()
        _check(lib().comet_mcts_create(ctypes.byref(self.opts), ctypes.byref(h)))
        self.handle = h

    def ask(self, pool: int, instance: int = 0):
        """The next pool as a host array of packed records."""
        out = np.zeros(pool, dtype=MODE_SEQ_DTYPE)
        n = ctypes.c_int64()
        _check(lib().comet_mcts_ask(self.handle, instance, pool, out.ctypes.data, ctypes.byref(n)))
        return out[: n.value]

    def tell(self, cost, viol):
        c = np.ascontiguousarray(cost, dtype=np.float32)
        v = np.ascontiguousarray(viol, dtype=np.float32)
        _check(lib().comet_mcts_tell(self.handle, c.ctypes.data, v.ctypes.data, len(c)))

    def stats(self) -> dict:
        st = MctsStats()
        _check(lib().comet_mcts_get_stats(self.handle, ctypes.byref(st)))
        return {"evaluations": st.evaluations, "tree_nodes": st.tree_nodes, "pending": st.pending,
                "exhausted": bool(st.exhausted), "best": st.best}

    def best(self, k: int):
        codes = np.zeros(max(k, 1), np.uint64)
        merits = np.zeros(max(k, 1), np.float64)
        n = ctypes.c_int64()
        _check(lib().comet_mcts_best(self.handle, k, codes.ctypes.data, merits.ctypes.data, ctypes.byref(n)))
        return codes[: n.value], merits[: n.value]

    def close(self):
        if self.handle:
            lib().comet_mcts_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def comet_plan_mcts(problem, instance: int, mcts_opts=None, pool: int = 1024, opts=None, out_traj=None) -> dict:
    """MCTS plan for one instance (comet_plan_mcts); mcts_opts: MctsOpts,
    dict or None; opts: PlanOpts, dict or None (k_ref, ref_iters)."""
    if mcts_opts is None or isinstance(mcts_opts, dict):
        mcts_opts = comet_mcts_default_opts(**(mcts_opts or {}))
    if opts is None or isinstance(opts, dict):
        o = comet_default_plan_opts()
        for k, v in (opts or {}).items():
            setattr(o, k, v)
        opts = o
    r = PlanResult()
    _check(lib().comet_plan_mcts(problem, int(instance), ctypes.byref(mcts_opts), int(pool), ctypes.byref(opts),
                                 ctypes.byref(r), _ptr(out_traj)))
    return {"best": tuple(int(r.best.modes[i]) for i in range(r.best.len)), "best_cost": r.best_cost,
            "best_viol": r.best_viol, "best_status": r.best_status, "rounds_run": r.rounds_run,
            "evaluations": r.evaluations, "explore_ms": r.explore_ms, "refine_ms": r.refine_ms}


def decode_code(code: int, n_modes: int = 12):
    base = n_modes + 1
    L = code % base
    code //= base
    out = []
    for _ in range(L):
        out.append(code % base - 1)
        code //= base
    return tuple(out)


def comet_mode_code(seq, n_modes: int = 12) -> int:
    if not isinstance(seq, ModeSeq):
        s = ModeSeq()
        s.instance = 0
        s.len = len(seq)
        for i, m in enumerate(seq):
            s.modes[i] = int(m)
        seq = s
    return int(lib().comet_mode_code(ctypes.byref(seq), n_modes))


def comet_last_error() -> str:
    return lib().comet_last_error().decode()


# ------------------------------------------------------------- marshalling

def pack_mode_seqs(seqs, inst_idx=None, lens=None) -> np.ndarray:
    """Pack orders into the 40-byte comet_mode_seq records.  seqs: integer
    [n, L] (all of length L, or padded with `lens`) or a list of tuples."""
    if isinstance(seqs, np.ndarray) and seqs.ndim == 2:
        n, L = seqs.shape
        out = np.zeros(n, dtype=MODE_SEQ_DTYPE)
        out["modes"][:, :L] = seqs
        out["len"] = L if lens is None else np.asarray(lens, dtype=np.uint8)
    else:
        n = len(seqs)
        out = np.zeros(n, dtype=MODE_SEQ_DTYPE)
        for i, s in enumerate(seqs):
            out["modes"][i, : len(s)] = s
            out["len"][i] = len(s)
    out["instance"] = 0 if inst_idx is None else np.asarray(inst_idx, dtype=np.int32)
    return out


class Problem:
    """Convenience owner of a comet_problem handle (torch tensors in/out)."""

    def __init__(self, instances, opts=None, stream=None):
        import torch

        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = comet_problem_create(instances, opts, self.stream.cuda_stream)
        self.stride = comet_traj_stride(self.handle)
        self.instances = list(instances)

    def close(self):
        if self.handle:
            comet_problem_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def eval(self, seqs_dev, warm=None, want_traj=False, max_iters=0):
        """seqs_dev: uint8 CUDA tensor [n, 40] of packed orders.  Returns a dict
        of CUDA tensors: cost, status, viol, merit, iters, stat (and traj)."""
        torch = self.torch
        n = seqs_dev.shape[0]
        dev = seqs_dev.device
        cost = torch.empty(n, dtype=torch.float32, device=dev)
        status = torch.empty(n, dtype=torch.int32, device=dev)
        traj = torch.empty((n, self.stride), dtype=torch.float32, device=dev) if want_traj else None
        comet_eval_modes_budget(self.handle, seqs_dev, n, warm, max_iters, cost, traj, status)
        out = {"cost": cost, "status": status}
        if traj is not None:
            out["traj"] = traj
        viol = torch.empty(n, dtype=torch.float32, device=dev)
        merit = torch.empty_like(viol)
        iters = torch.empty(n, dtype=torch.int32, device=dev)
        stat = torch.empty_like(viol)
        comet_eval_stats(self.handle, viol, merit, iters, stat)
        out.update(viol=viol, merit=merit, iters=iters, stat=stat)
        return out


# ------------------------------------------------------ learned proposal

def comet_default_proposal_desc() -> ProposalDesc:
    d = ProposalDesc()
    lib().comet_default_proposal_desc(ctypes.byref(d))
    return d


def comet_default_adamw_opts() -> AdamWOpts:
    o = AdamWOpts()
    lib().comet_default_adamw_opts(ctypes.byref(o))
    return o


def _fill(struct, defaults, over):
    for k, v in (over or {}).items():
        if not hasattr(defaults, k):
            raise KeyError(k)
        setattr(defaults, k, v)
    return defaults


def comet_proposal_create(problem, desc=None) -> int:
    d = desc if isinstance(desc, ProposalDesc) else _fill(ProposalDesc, comet_default_proposal_desc(), desc)
    h = ctypes.c_void_p()
    _check(lib().comet_proposal_create(problem, ctypes.byref(d), ctypes.byref(h)))
    return h.value


def comet_proposal_destroy(q):
    _check(lib().comet_proposal_destroy(q))


def comet_proposal_dims(q):
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    n = ctypes.c_int64()
    _check(lib().comet_proposal_dims(q, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(n)))
    return a.value, b.value, c.value, n.value


def comet_proposal_set_params(q, flat):
    _check(lib().comet_proposal_set_params(q, _ptr(flat)))


def comet_proposal_get_params(q, flat, grad=None):
    _check(lib().comet_proposal_get_params(q, _ptr(flat), _ptr(grad)))


def comet_proposal_save(q, path):
    """Parameters, AdamW moments and step count to a checkpoint file."""
    _check(lib().comet_proposal_save(q, os.fsencode(path)))


def comet_proposal_load(q, path):
    """Resume from a checkpoint file of the same network layout."""
    _check(lib().comet_proposal_load(q, os.fsencode(path)))


def comet_proposal_features(q, seqs, n, out_x):
    _check(lib().comet_proposal_features(q, _ptr(seqs), n, _ptr(out_x)))


def comet_proposal_forward(q, x, n, out_y):
    _check(lib().comet_proposal_forward(q, _ptr(x), n, _ptr(out_y)))


def comet_proposal_time_forward(q, x, n, reps=20) -> float:
    ms = ctypes.c_float()
    _check(lib().comet_proposal_time_forward(q, _ptr(x), n, reps, ctypes.byref(ms)))
    return ms.value


def comet_proposal_train_batch(q, x, target, weight, n, opts=None) -> float:
    o = opts if isinstance(opts, AdamWOpts) else _fill(AdamWOpts, comet_default_adamw_opts(), opts)
    loss = ctypes.c_float()
    _check(lib().comet_proposal_train_batch(q, _ptr(x), _ptr(target), _ptr(weight), n, ctypes.byref(o),
                                            ctypes.byref(loss)))
    return loss.value


def comet_proposal_add_samples(q, seqs, n, cost, viol, status, traj):
    _check(lib().comet_proposal_add_samples(q, _ptr(seqs), n, _ptr(cost), _ptr(viol), _ptr(status), _ptr(traj)))


def comet_proposal_dataset_size(q) -> int:
    n = ctypes.c_int64()
    _check(lib().comet_proposal_dataset_size(q, ctypes.byref(n)))
    return n.value


def comet_proposal_dataset_rows(q, first, n, out_x=None, out_t=None, out_w=None):
    _check(lib().comet_proposal_dataset_rows(q, first, n, _ptr(out_x), _ptr(out_t), _ptr(out_w)))


def proposal_dataset_rows(q, n, first=0):
    """(targets, weights, feature bits) of n training rows as numpy arrays."""
    din, _, dout, _ = comet_proposal_dims(q)
    x = np.zeros((n, din), np.uint16)
    t = np.zeros((n, dout), np.float32)
    w = np.zeros((n, dout), np.float32)
    comet_proposal_dataset_rows(q, first, n, x, t, w)
    return t, w, x


def comet_proposal_train(q, steps, batch, opts=None, seed=0) -> np.ndarray:
    o = opts if isinstance(opts, AdamWOpts) else _fill(AdamWOpts, comet_default_adamw_opts(), opts)
    losses = np.zeros(max(steps, 1), dtype=np.float32)
    _check(lib().comet_proposal_train(q, steps, batch, ctypes.byref(o), seed, losses.ctypes.data))
    return losses[:steps]


def comet_proposal_predict(q, seqs, n, out_merit=None, out_warm=None):
    _check(lib().comet_proposal_predict(q, _ptr(seqs), n, _ptr(out_merit), _ptr(out_warm)))


def comet_proposal_prune(q, frontier, keep, out_warm=None):
    _check(lib().comet_proposal_prune(q, frontier, keep, _ptr(out_warm)))


def comet_gemm_bf16(a, lda, b, ldb, m, n, k, kind=GEMM_STORE, k_splits=1, bias=None, out_f32=None, ld_f32=0,
                    out_bf16=None, ld_bf16=0, out_bf16_t=None, ld_bf16_t=0, z_in=None, ld_z=0, stream=None):
    ep = GemmEpilogue(kind, k_splits, _ptr(bias), _ptr(out_f32), ld_f32, _ptr(out_bf16), ld_bf16,
                      _ptr(out_bf16_t), ld_bf16_t, _ptr(z_in), ld_z)
    _check(lib().comet_gemm_bf16(_ptr(a), lda, _ptr(b), ldb, m, n, k, ctypes.byref(ep), stream))


# ------------------------------------------------------- launch shape

def comet_get_launch_config(problem) -> dict:
    c = LaunchConfig()
    _check(lib().comet_get_launch_config(problem, ctypes.byref(c)))
    return {"warps_per_block": c.warps_per_block, "blocks_per_sm": c.blocks_per_sm,
            "max_blocks_per_sm": c.max_blocks_per_sm, "unroll": c.unroll}


def comet_set_launch_config(problem, warps_per_block: int, blocks_per_sm: int, unroll: int = 1):
    c = LaunchConfig(warps_per_block, blocks_per_sm, 0, unroll)
    _check(lib().comet_set_launch_config(problem, ctypes.byref(c)))


def comet_autotune(problem, sample, n: int, max_iters: int = 0):
    """Returns (picked config dict, list of candidate times in ms)."""
    c = LaunchConfig()
    ms = np.zeros(16, np.float32)
    nc = ctypes.c_int32()
    _check(lib().comet_autotune(problem, _ptr(sample), n, max_iters, ctypes.byref(c), ms.ctypes.data,
                                ctypes.byref(nc)))
    return ({"warps_per_block": c.warps_per_block, "blocks_per_sm": c.blocks_per_sm,
             "max_blocks_per_sm": c.max_blocks_per_sm, "unroll": c.unroll}, [float(x) for x in ms[: nc.value]])
