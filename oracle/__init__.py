"""FP64 CPU oracle of the CoMET hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs may import this package.  The
product library (``paper_2609_21803_gb300``) never imports, links or calls
it, and the two share no code: the only common module is ``workloads``,
which draws seeded inputs and holds none of the method's arithmetic.

Contents
  * ``comet_oracle.c``  -- the mode-conditioned TO (Eq. mode_nlp) in FP64,
    solved by the augmented-Lagrangian Gauss-Newton / backward-sweep method
    of Sec. III-C, scored by Eq. inexact_mode_value and Eq. search_merit.
  * ``search.py``       -- full enumeration (Eq. mode_selection), the
    neighbourhood N_1(m) and the batch-synchronous greedy expansion of
    Algorithm 1 (Sec. III-B), in plain Python.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "comet_oracle.c")
_SRC_BIM = os.path.join(_HERE, "bimanual.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libcomet_oracle.so")
_LIB_FLOPS_PATH = os.path.join(_HERE, "_build", "libcomet_oracle_flops.so")
_lock = threading.Lock()
_lib = None

CONVERGED, MAX_ITER, INFEASIBLE, FACTOR_FAIL, NONFINITE = range(5)
# pushing mode 12: free motion (faces 0..3 x {stick, slide+, slide-} are 0..11)
MODE_FREE = 12


def build(force: bool = False, count_flops: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE double, no fast-math).
    count_flops: the separate build with the method's flop counter compiled
    in (libcomet_oracle_flops.so), used to measure flops per stage and
    iteration; the default build carries no counter."""
    path = _LIB_FLOPS_PATH if count_flops else _LIB_PATH
    os.makedirs(os.path.dirname(path), exist_ok=True)
    srcs = [_SRC, _SRC_BIM, os.path.join(_HERE, "comet_oracle.h"), os.path.join(_HERE, "bimanual.h"),
            os.path.join(_HERE, "flops.h")]
    if force or not os.path.exists(path) or os.path.getmtime(path) < max(os.path.getmtime(f) for f in srcs):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-Wall"]
            + (["-DORC_COUNT_FLOPS"] if count_flops else [])
            + ["-o", tmp, _SRC, _SRC_BIM, "-lm", "-lpthread"]
        )
        os.replace(tmp, path)
    return path


class Instance(ctypes.Structure):
    _fields_ = [
        ("side_x", ctypes.c_double), ("side_y", ctypes.c_double), ("c_ls", ctypes.c_double),
        ("mu", ctypes.c_double), ("dt", ctypes.c_double), ("kappa", ctypes.c_double),
        ("knots_per_segment", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("start", ctypes.c_double * 3), ("goal", ctypes.c_double * 3),
        ("w_terminal", ctypes.c_double), ("w_control", ctypes.c_double),
    ]


class Opts(ctypes.Structure):
    _fields_ = [
        ("max_iters", ctypes.c_int32), ("max_factor_retries", ctypes.c_int32),
        ("n_alpha", ctypes.c_int32), ("max_inner", ctypes.c_int32),
        ("beta0", ctypes.c_double), ("beta_max", ctypes.c_double), ("beta_growth", ctypes.c_double),
        ("rho0", ctypes.c_double), ("rho_min", ctypes.c_double), ("rho_max", ctypes.c_double),
        ("armijo_c1", ctypes.c_double), ("ls_slack", ctypes.c_double),
        ("eps_primal", ctypes.c_double), ("eps_dual", ctypes.c_double), ("eps_comp", ctypes.c_double),
        ("omega_ratio", ctypes.c_double), ("eta_ratio", ctypes.c_double),
        ("eps_feas", ctypes.c_double), ("merit_mu", ctypes.c_double), ("beta_ref", ctypes.c_double),
        ("curv_skip", ctypes.c_int32), ("pad1", ctypes.c_int32),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("cost", ctypes.c_double), ("viol", ctypes.c_double), ("merit", ctypes.c_double),
        ("stat", ctypes.c_double), ("comp", ctypes.c_double),
        ("beta", ctypes.c_double), ("rho", ctypes.c_double),
        ("status", ctypes.c_int32), ("iters", ctypes.c_int32),
        ("n_outer", ctypes.c_int32), ("n_rejected", ctypes.c_int32),
        ("n_curv_fail", ctypes.c_int32), ("pad1", ctypes.c_int32),
    ]


class BimInstance(ctypes.Structure):
    _fields_ = [
        ("ax", ctypes.c_double), ("az", ctypes.c_double), ("mass", ctypes.c_double),
        ("mu_g", ctypes.c_double), ("mu_h", ctypes.c_double), ("dt", ctypes.c_double),
        ("grav", ctypes.c_double), ("knots_per_segment", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("start", ctypes.c_double * 3), ("goal", ctypes.c_double * 3),
        ("w_terminal", ctypes.c_double), ("w_v", ctypes.c_double), ("w_f", ctypes.c_double),
        ("w_s", ctypes.c_double), ("w_c", ctypes.c_double),
    ]


RESULT_DTYPE = np.dtype([
    ("cost", "f8"), ("viol", "f8"), ("merit", "f8"), ("stat", "f8"), ("comp", "f8"),
    ("beta", "f8"), ("rho", "f8"), ("status", "i4"), ("iters", "i4"),
    ("n_outer", "i4"), ("n_rejected", "i4"), ("n_curv_fail", "i4"), ("pad1", "i4"),
])
assert RESULT_DTYPE.itemsize == ctypes.sizeof(Result)

_P = ctypes.POINTER
_dp = _P(ctypes.c_double)
_u8p = _P(ctypes.c_uint8)
_u16p = _P(ctypes.c_uint16)
_i32p = _P(ctypes.c_int32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_default_opts.argtypes = [_P(Opts)]
            L.orc_dynamics.argtypes = [_P(Instance), ctypes.c_int32, _dp, _dp, _dp, _dp, _dp]
            L.orc_segment_of.argtypes = [ctypes.c_int32] * 3
            L.orc_segment_of.restype = ctypes.c_int32
            L.orc_cold_start.argtypes = [_P(Instance), ctypes.c_int32, _dp]
            L.orc_rows.argtypes = [_P(Instance), ctypes.c_int32, _u8p, ctypes.c_int32, _dp, _dp, _u8p, _dp, _dp]
            L.orc_dense_jacobian.argtypes = [_P(Instance), ctypes.c_int32, _u8p, ctypes.c_int32, _dp, _dp]
            L.orc_gn_step.argtypes = [_P(Instance), ctypes.c_int32, _u8p, ctypes.c_int32, _dp, _dp,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int32, _dp, _dp]
            L.orc_gn_step.restype = ctypes.c_int32
            L.orc_al_merit.argtypes = [_P(Instance), ctypes.c_int32, _u8p, ctypes.c_int32, _dp, _dp,
                                       ctypes.c_double, _dp]
            L.orc_al_merit.restype = ctypes.c_double
            L.orc_solve.argtypes = [_P(Instance), ctypes.c_int32, _u8p, ctypes.c_int32, _dp, _P(Opts),
                                    _dp, _dp, _P(Result)]
            L.orc_solve.restype = ctypes.c_int32
            L.orc_solve_batch.argtypes = [_P(Instance), _i32p, _i32p, _u8p, ctypes.c_int32, _i32p,
                                          ctypes.c_int64, _P(Opts), ctypes.c_int32, _dp, ctypes.c_int64,
                                          ctypes.c_void_p]
            L.orc_solve_batch.restype = ctypes.c_int32
            L.orc_solve_batch_ex.argtypes = [_P(Instance), _i32p, _i32p, _u8p, ctypes.c_int32, _i32p,
                                             ctypes.c_int64, _P(Opts), ctypes.c_int32, _dp, ctypes.c_int64,
                                             _dp, _dp, ctypes.c_int64, _dp, ctypes.c_int64, ctypes.c_void_p]
            L.orc_solve_batch_ex.restype = ctypes.c_int32
            B = _P(BimInstance)
            L.bim_interval_rows.argtypes = [B, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _dp, _dp, _dp, _dp,
                                            _u8p, _u8p, _dp, _dp]
            L.bim_rows.argtypes = [B, ctypes.c_int32, _u16p, ctypes.c_int32, _dp, _dp, _u8p, _dp, _dp]
            L.bim_dense_jacobian.argtypes = [B, ctypes.c_int32, _u16p, ctypes.c_int32, _dp, _dp]
            L.bim_cold_start.argtypes = [B, ctypes.c_int32, _dp]
            L.bim_cost.argtypes = [B, ctypes.c_int32, _dp]
            L.bim_cost.restype = ctypes.c_double
            L.bim_gn_step.argtypes = [B, ctypes.c_int32, _u16p, ctypes.c_int32, _dp, _dp, ctypes.c_double,
                                      ctypes.c_double, _dp, _dp]
            L.bim_gn_step.restype = ctypes.c_int32
            L.bim_al_merit.argtypes = [B, ctypes.c_int32, _u16p, ctypes.c_int32, _dp, _dp, ctypes.c_double]
            L.bim_al_merit.restype = ctypes.c_double
            L.bim_solve.argtypes = [B, ctypes.c_int32, _u16p, ctypes.c_int32, _dp, _P(Opts), _dp, _dp, _P(Result)]
            L.bim_solve.restype = ctypes.c_int32
            L.bim_solve_batch.argtypes = [B, _i32p, _i32p, _u16p, ctypes.c_int32, _i32p, ctypes.c_int64, _P(Opts),
                                          ctypes.c_int32, _dp, ctypes.c_int64, ctypes.c_void_p]
            L.bim_solve_batch.restype = ctypes.c_int32
            L.bim_solve_batch_ex.argtypes = [B, _i32p, _i32p, _u16p, ctypes.c_int32, _i32p, ctypes.c_int64,
                                             _P(Opts), ctypes.c_int32, _dp, ctypes.c_int64, _dp, _dp,
                                             ctypes.c_int64, _dp, ctypes.c_int64, ctypes.c_void_p]
            L.bim_solve_batch_ex.restype = ctypes.c_int32
            _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def make_instance(d: dict) -> Instance:
    """Build the oracle's instance struct from a workload descriptor dict."""
    s = Instance()
    s.side_x, s.side_y = d["side_x"], d["side_y"]
    s.c_ls, s.mu, s.dt = d["c_ls"], d["mu"], d["dt"]
    s.kappa = d.get("kappa", 1.0)
    s.knots_per_segment = int(d["knots_per_segment"])
    for i in range(3):
        s.start[i] = d["start"][i]
        s.goal[i] = d["goal"][i]
    s.w_terminal, s.w_control = d["w_terminal"], d["w_control"]
    return s


def default_opts(**over) -> Opts:
    o = Opts()
    lib().orc_default_opts(ctypes.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def traj_len(N: int) -> int:
    return 7 * N + 4


def dynamics(inst: dict, face: int, x, u):
    """f(x,u), Fx (4x4), Fu (4x3) of the pusher-slider on `face`."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    f = np.zeros(4)
    Fx = np.zeros((4, 4))
    Fu = np.zeros((4, 3))
    s = make_instance(inst)
    lib().orc_dynamics(ctypes.byref(s), face, _ptr(x, _dp), _ptr(u, _dp), _ptr(f, _dp), _ptr(Fx, _dp), _ptr(Fu, _dp))
    return f, Fx, Fu


def segment_of(k: int, length: int, N: int) -> int:
    return lib().orc_segment_of(k, length, N)


def cold_start(inst: dict, N: int) -> np.ndarray:
    tr = np.zeros(traj_len(N))
    s = make_instance(inst)
    lib().orc_cold_start(ctypes.byref(s), N, _ptr(tr, _dp))
    return tr


def rows(inst: dict, modes, N: int, traj):
    """(c[N,11], mask[N,11], scale[N,11], c_init[3]) at traj."""
    m = np.ascontiguousarray(modes, dtype=np.uint8)
    traj = np.ascontiguousarray(traj, dtype=np.float64)
    c = np.zeros((N, 11))
    mask = np.zeros((N, 11), dtype=np.uint8)
    scale = np.zeros((N, 11))
    ci = np.zeros(3)
    s = make_instance(inst)
    lib().orc_rows(ctypes.byref(s), len(m), _ptr(m, _u8p), N, _ptr(traj, _dp),
                   _ptr(c, _dp), _ptr(mask, _u8p), _ptr(scale, _dp), _ptr(ci, _dp))
    return c, mask, scale, ci


def dense_jacobian(inst: dict, modes, N: int, traj) -> np.ndarray:
    m = np.ascontiguousarray(modes, dtype=np.uint8)
    traj = np.ascontiguousarray(traj, dtype=np.float64)
    jac = np.zeros((3 + 11 * N, 7 * N + 4))
    s = make_instance(inst)
    lib().orc_dense_jacobian(ctypes.byref(s), len(m), _ptr(m, _u8p), N, _ptr(traj, _dp), _ptr(jac, _dp))
    return jac


def gn_step(inst: dict, modes, N: int, traj, lam, beta: float, rho: float, curvature: bool = False):
    """(dz, grad) of one backward-sweep step (interleaved z order); with
    ``curvature`` the Lagrangian curvature of the dynamics rows is included."""
    m = np.ascontiguousarray(modes, dtype=np.uint8)
    traj = np.ascontiguousarray(traj, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    dz = np.zeros(7 * N + 4)
    g = np.zeros(7 * N + 4)
    s = make_instance(inst)
    rc = lib().orc_gn_step(ctypes.byref(s), len(m), _ptr(m, _u8p), N, _ptr(traj, _dp), _ptr(lam, _dp),
                           beta, rho, int(curvature), _ptr(dz, _dp), _ptr(g, _dp))
    if rc != 0:
        raise RuntimeError("local Cholesky failed")
    return dz, g


def al_merit(inst: dict, modes, N: int, traj, lam, beta: float):
    m = np.ascontiguousarray(modes, dtype=np.uint8)
    traj = np.ascontiguousarray(traj, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    J = ctypes.c_double()
    s = make_instance(inst)
    L = lib().orc_al_merit(ctypes.byref(s), len(m), _ptr(m, _u8p), N, _ptr(traj, _dp), _ptr(lam, _dp),
                           beta, ctypes.byref(J))
    return L, J.value


def solve(inst: dict, modes, N: int | None = None, warm=None, opts: Opts | None = None):
    """Solve one mode-conditioned TO; returns (traj, lam, result dict)."""
    m = np.ascontiguousarray(modes, dtype=np.uint8)
    if N is None:
        N = int(inst["knots_per_segment"]) * len(m)
    tr = np.zeros(traj_len(N))
    lam = np.zeros(3 + 11 * N)
    w = None if warm is None else np.ascontiguousarray(warm, dtype=np.float64)
    r = Result()
    o = opts if opts is not None else default_opts()
    s = make_instance(inst)
    lib().orc_solve(ctypes.byref(s), len(m), _ptr(m, _u8p), N, _ptr(w, _dp), ctypes.byref(o),
                    _ptr(tr, _dp), _ptr(lam, _dp), ctypes.byref(r))
    res = {f: getattr(r, f) for f, _ in Result._fields_}
    return tr, lam, res


def solve_batch(insts: list, inst_idx, seqs, lens, Ns=None, opts: Opts | None = None,
                nthreads: int | None = None, want_traj: bool = False):
    """Solve many TOs on host threads.  seqs: uint8 [n, lmax]; returns
    (structured result array, traj array [n, 7*Nmax+4] or None)."""
    seqs = np.ascontiguousarray(seqs, dtype=np.uint8)
    n, lmax = seqs.shape
    lens = np.ascontiguousarray(lens, dtype=np.int32)
    inst_idx = np.ascontiguousarray(inst_idx, dtype=np.int32)
    if Ns is None:
        K = np.array([int(insts[i]["knots_per_segment"]) for i in range(len(insts))], dtype=np.int32)
        Ns = K[inst_idx] * lens
    Ns = np.ascontiguousarray(Ns, dtype=np.int32)
    arr = (Instance * len(insts))(*[make_instance(d) for d in insts])
    res = np.zeros(n, dtype=RESULT_DTYPE)
    stride = traj_len(int(Ns.max())) if n else 0
    tr = np.zeros((n, stride)) if want_traj else None
    o = opts if opts is not None else default_opts()
    nth = nthreads or os.cpu_count() or 1
    lib().orc_solve_batch(arr, _ptr(inst_idx, _i32p), _ptr(lens, _i32p), _ptr(seqs, _u8p), lmax,
                          _ptr(Ns, _i32p), n, ctypes.byref(o), nth, _ptr(tr, _dp), stride,
                          res.ctypes.data_as(ctypes.c_void_p))
    return res, tr


def solve_batch_ex(insts: list, inst_idx, seqs, lens, warm=None, opts: Opts | None = None,
                   nthreads: int | None = None, warm_lam=None):
    """solve_batch with optional warm starts and the multipliers.  warm:
    float64 [n, 7*Nmax+4], row i holding TO i's component-major trajectory
    for its own N at the start of the row (as returned by solve_batch).
    warm_lam: float64 [n, 3+11*Nmax] starting multipliers (row i for TO i's
    own N), or None for zero.
    Returns (results, trajectories [n, 7*Nmax+4], multipliers [n, 3+11*Nmax])."""
    seqs = np.ascontiguousarray(seqs, dtype=np.uint8)
    n, lmax = seqs.shape
    lens = np.ascontiguousarray(lens, dtype=np.int32)
    inst_idx = np.ascontiguousarray(inst_idx, dtype=np.int32)
    K = np.array([int(insts[i]["knots_per_segment"]) for i in range(len(insts))], dtype=np.int32)
    Ns = np.ascontiguousarray(K[inst_idx] * lens, dtype=np.int32)
    arr = (Instance * len(insts))(*[make_instance(d) for d in insts])
    res = np.zeros(n, dtype=RESULT_DTYPE)
    Nmax = int(Ns.max()) if n else 0
    stride, lstride = traj_len(Nmax), 3 + 11 * Nmax
    tr = np.zeros((n, stride))
    lam = np.zeros((n, lstride))
    w = None
    if warm is not None:
        w = np.ascontiguousarray(warm, dtype=np.float64)
        assert w.shape[0] == n and w.shape[1] >= stride
    wl = None
    if warm_lam is not None:
        wl = np.ascontiguousarray(warm_lam, dtype=np.float64)
        assert wl.shape == (n, lstride)
    o = opts if opts is not None else default_opts()
    lib().orc_solve_batch_ex(arr, _ptr(inst_idx, _i32p), _ptr(lens, _i32p), _ptr(seqs, _u8p), lmax,
                             _ptr(Ns, _i32p), n, ctypes.byref(o), nthreads or os.cpu_count() or 1,
                             _ptr(w, _dp), w.shape[1] if w is not None else 0, _ptr(wl, _dp), _ptr(tr, _dp),
                             stride, _ptr(lam, _dp), lstride, res.ctypes.data_as(ctypes.c_void_p))
    return res, tr, lam


# ------------------------------------------------------------- bimanual

BIM_NX, BIM_NU, BIM_NROW, BIM_NMODES = 5, 12, 32, 507
GRAVITY = 9.81


def bim_make_instance(d: dict) -> BimInstance:
    """The oracle's bimanual instance from a workload descriptor (the same
    dict the library takes: side_x, side_y = box width and height, mu = hand
    friction, ground_mu, mass, w_control = the weight of twist, sliding rates
    and p_c; forces are weighted by w_control / (m g)^2)."""
    s = BimInstance()
    s.ax, s.az = 0.5 * d["side_x"], 0.5 * d["side_y"]
    s.mass, s.mu_g, s.mu_h = d["mass"], d["ground_mu"], d["mu"]
    s.dt, s.grav = d["dt"], GRAVITY
    s.knots_per_segment = int(d["knots_per_segment"])
    for i in range(3):
        s.start[i] = d["start"][i]
        s.goal[i] = d["goal"][i]
    mg = d["mass"] * GRAVITY
    s.w_terminal = d["w_terminal"]
    s.w_v = s.w_s = s.w_c = d["w_control"]
    s.w_f = d["w_control"] / (mg * mg)
    return s


def bim_traj_len(N: int) -> int:
    return (BIM_NX + BIM_NU) * N + BIM_NX


def bim_interval_rows(inst: dict, mode: int, mask_sL: bool, mask_sR: bool, xk, uk, xk1):
    """(c[32], mask, ineq, scale, J[32][22]) of one interval."""
    c = np.zeros(BIM_NROW)
    mask = np.zeros(BIM_NROW, np.uint8)
    ineq = np.zeros(BIM_NROW, np.uint8)
    scale = np.zeros(BIM_NROW)
    J = np.zeros((BIM_NROW, 2 * BIM_NX + BIM_NU))
    xk, uk, xk1 = (np.ascontiguousarray(a, dtype=np.float64) for a in (xk, uk, xk1))
    lib().bim_interval_rows(ctypes.byref(bim_make_instance(inst)), int(mode), int(mask_sL), int(mask_sR),
                            _ptr(xk, _dp), _ptr(uk, _dp), _ptr(xk1, _dp), _ptr(c, _dp), _ptr(mask, _u8p),
                            _ptr(ineq, _u8p), _ptr(scale, _dp), _ptr(J, _dp))
    return c, mask.astype(bool), ineq.astype(bool), scale, J


def bim_cold_start(inst: dict, N: int) -> np.ndarray:
    tr = np.zeros(5 * (N + 1) + 12 * N)
    lib().bim_cold_start(ctypes.byref(bim_make_instance(inst)), N, _ptr(tr, _dp))
    return tr


def bim_rows(inst: dict, modes, N: int, traj):
    modes = np.ascontiguousarray(modes, dtype=np.uint16)
    traj = np.ascontiguousarray(traj, dtype=np.float64)
    c = np.zeros((N, BIM_NROW))
    mask = np.zeros((N, BIM_NROW), np.uint8)
    scale = np.zeros((N, BIM_NROW))
    ci = np.zeros(3)
    lib().bim_rows(ctypes.byref(bim_make_instance(inst)), len(modes), _ptr(modes, _u16p), N, _ptr(traj, _dp),
                   _ptr(c, _dp), _ptr(mask, _u8p), _ptr(scale, _dp), _ptr(ci, _dp))
    return c, mask.astype(bool), scale, ci


def bim_dense_jacobian(inst: dict, modes, N: int, traj) -> np.ndarray:
    modes = np.ascontiguousarray(modes, dtype=np.uint16)
    traj = np.ascontiguousarray(traj, dtype=np.float64)
    nz, nr = bim_traj_len(N), 3 + BIM_NROW * N
    jac = np.zeros((nr, nz))
    lib().bim_dense_jacobian(ctypes.byref(bim_make_instance(inst)), len(modes), _ptr(modes, _u16p), N,
                             _ptr(traj, _dp), _ptr(jac, _dp))
    return jac


def bim_cost(inst: dict, N: int, traj) -> float:
    traj = np.ascontiguousarray(traj, dtype=np.float64)
    return lib().bim_cost(ctypes.byref(bim_make_instance(inst)), N, _ptr(traj, _dp))


def bim_gn_step(inst: dict, modes, N: int, traj, lam, beta: float, rho: float):
    modes = np.ascontiguousarray(modes, dtype=np.uint16)
    traj = np.ascontiguousarray(traj, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    dz = np.zeros(bim_traj_len(N))
    grad = np.zeros(bim_traj_len(N))
    ok = lib().bim_gn_step(ctypes.byref(bim_make_instance(inst)), len(modes), _ptr(modes, _u16p), N,
                           _ptr(traj, _dp), _ptr(lam, _dp), beta, rho, _ptr(dz, _dp), _ptr(grad, _dp))
    return ok, dz, grad


def bim_al_merit(inst: dict, modes, N: int, traj, lam, beta: float) -> float:
    modes = np.ascontiguousarray(modes, dtype=np.uint16)
    traj = np.ascontiguousarray(traj, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    return lib().bim_al_merit(ctypes.byref(bim_make_instance(inst)), len(modes), _ptr(modes, _u16p), N,
                              _ptr(traj, _dp), _ptr(lam, _dp), beta)


def bim_solve(inst: dict, modes, N: int | None = None, warm=None, opts: Opts | None = None):
    """(result dict, trajectory, multipliers) of one bimanual mode order."""
    modes = np.ascontiguousarray(modes, dtype=np.uint16)
    N = N if N is not None else inst["knots_per_segment"] * len(modes)
    tr = np.zeros(bim_traj_len(N))
    lam = np.zeros(3 + BIM_NROW * N)
    r = Result()
    o = opts if opts is not None else default_opts()
    w = None if warm is None else np.ascontiguousarray(warm, dtype=np.float64)
    lib().bim_solve(ctypes.byref(bim_make_instance(inst)), len(modes), _ptr(modes, _u16p), N, _ptr(w, _dp),
                    ctypes.byref(o), _ptr(tr, _dp), _ptr(lam, _dp), ctypes.byref(r))
    res = {f: getattr(r, f) for f, _ in Result._fields_ if f != "pad1"}
    return res, tr, lam


def bim_solve_batch(insts: list, inst_idx, seqs, lens, opts: Opts | None = None, nthreads: int | None = None,
                    want_traj: bool = False):
    """Solve many bimanual orders on host threads; returns (results, trajs)."""
    n = len(inst_idx)
    lmax = max(1, max((len(s) for s in seqs), default=1))
    modes = np.zeros((n, lmax), np.uint16)
    for i, s in enumerate(seqs):
        modes[i, : len(s)] = s
    lens = np.ascontiguousarray(lens, dtype=np.int32)
    inst_idx = np.ascontiguousarray(inst_idx, dtype=np.int32)
    Ns = np.array([insts[j]["knots_per_segment"] * int(L) for j, L in zip(inst_idx, lens)], np.int32)
    arr = (BimInstance * len(insts))(*[bim_make_instance(d) for d in insts])
    res = np.zeros(n, dtype=RESULT_DTYPE)
    stride = bim_traj_len(int(Ns.max())) if n else 0
    tr = np.zeros((n, stride)) if want_traj else None
    o = opts if opts is not None else default_opts()
    lib().bim_solve_batch(arr, _ptr(inst_idx, _i32p), _ptr(lens, _i32p), _ptr(modes, _u16p), lmax,
                          _ptr(Ns, _i32p), n, ctypes.byref(o), nthreads or (os.cpu_count() or 1),
                          _ptr(tr, _dp), stride, res.ctypes.data)
    return res, tr


def bim_solve_batch_ex(insts: list, inst_idx, seqs, lens, warm=None, opts: Opts | None = None,
                       nthreads: int | None = None, warm_lam=None):
    """bim_solve_batch with optional warm starts (float64 [n, stride], TO i's
    trajectory for its own N at the start of row i) and the multipliers.
    Returns (results, trajectories [n, 17*Nmax+5], multipliers [n, 3+32*Nmax])."""
    n = len(inst_idx)
    lmax = max(1, max((len(s) for s in seqs), default=1))
    modes = np.zeros((n, lmax), np.uint16)
    for i, s in enumerate(seqs):
        modes[i, : len(s)] = s
    lens = np.ascontiguousarray(lens, dtype=np.int32)
    inst_idx = np.ascontiguousarray(inst_idx, dtype=np.int32)
    Ns = np.array([insts[j]["knots_per_segment"] * int(L) for j, L in zip(inst_idx, lens)], np.int32)
    arr = (BimInstance * len(insts))(*[bim_make_instance(d) for d in insts])
    res = np.zeros(n, dtype=RESULT_DTYPE)
    Nmax = int(Ns.max()) if n else 0
    stride, lstride = bim_traj_len(Nmax), 3 + BIM_NROW * Nmax
    tr = np.zeros((n, stride))
    lam = np.zeros((n, lstride))
    w = None
    if warm is not None:
        w = np.ascontiguousarray(warm, dtype=np.float64)
        assert w.shape[0] == n and w.shape[1] >= stride
    wl = None
    if warm_lam is not None:
        wl = np.ascontiguousarray(warm_lam, dtype=np.float64)
        assert wl.shape == (n, lstride)
    o = opts if opts is not None else default_opts()
    lib().bim_solve_batch_ex(arr, _ptr(inst_idx, _i32p), _ptr(lens, _i32p), _ptr(modes, _u16p), lmax,
                             _ptr(Ns, _i32p), n, ctypes.byref(o), nthreads or (os.cpu_count() or 1),
                             _ptr(w, _dp), w.shape[1] if w is not None else 0, _ptr(wl, _dp), _ptr(tr, _dp),
                             stride, _ptr(lam, _dp), lstride, res.ctypes.data_as(ctypes.c_void_p))
    return res, tr, lam


def flops_per_stage_iteration(insts, inst_idx, seqs, lens, opts: Opts | None = None):
    """The method's floating-point operations per stage and solver iteration,
    measured by the counting build of the oracle over the given orders
    (solved one by one on the calling thread): total counted flops divided by
    sum over the TOs of (iterations x intervals).  Returns (flops per
    stage-iteration, total flops, sum of iterations x intervals)."""
    L = ctypes.CDLL(build(count_flops=True))
    L.orc_solve.argtypes = [_P(Instance), ctypes.c_int32, _u8p, ctypes.c_int32, _dp, _P(Opts), _dp, _dp, _P(Result)]
    L.orc_flop_count.restype = ctypes.c_uint64
    o = opts if opts is not None else default_opts()
    seqs = np.ascontiguousarray(seqs, dtype=np.uint8)
    L.orc_flop_reset()
    work = 0
    for t in range(len(inst_idx)):
        inst = insts[int(inst_idx[t])]
        m = np.ascontiguousarray(seqs[t][: int(lens[t])])
        N = int(inst["knots_per_segment"]) * int(lens[t])
        tr = np.zeros(traj_len(N))
        r = Result()
        L.orc_solve(ctypes.byref(make_instance(inst)), len(m), _ptr(m, _u8p), N, None, ctypes.byref(o),
                    _ptr(tr, _dp), None, ctypes.byref(r))
        work += r.iters * N
    total = int(L.orc_flop_count())
    return total / max(work, 1), total, work


def bim_flops_per_stage_iteration(insts, inst_idx, seqs, lens, opts: Opts | None = None):
    """flops_per_stage_iteration for the bimanual task (counting build of the
    bimanual oracle, orders solved one by one on the calling thread)."""
    L = ctypes.CDLL(build(count_flops=True))
    L.bim_solve.argtypes = [_P(BimInstance), ctypes.c_int32, _u16p, ctypes.c_int32, _dp, _P(Opts), _dp, _dp,
                            _P(Result)]
    L.orc_flop_count.restype = ctypes.c_uint64
    o = opts if opts is not None else default_opts()
    L.orc_flop_reset()
    work = 0
    for t in range(len(inst_idx)):
        inst = insts[int(inst_idx[t])]
        m = np.ascontiguousarray(seqs[t][: int(lens[t])], dtype=np.uint16)
        N = int(inst["knots_per_segment"]) * int(lens[t])
        tr = np.zeros(bim_traj_len(N))
        r = Result()
        L.bim_solve(ctypes.byref(bim_make_instance(inst)), len(m), _ptr(m, _u16p), N, None, ctypes.byref(o),
                    _ptr(tr, _dp), None, ctypes.byref(r))
        work += r.iters * N
    total = int(L.orc_flop_count())
    return total / max(work, 1), total, work
