"""Timing optimisation of the pushing TO -- TEST INFRASTRUCTURE ONLY (numpy,
FP64; imported by tests/, never by the product path).

Sec. III-C of the paper: when timing is optimised, the interval durations
are part of the controls; the experiments of Sec. IV-A optimise the time
step under the benchmark's duration bound.  The paper gives no rows or
variables for it; the readings taken here:
  * interval k has its own duration h_k, a fourth control, with bounds
    h_min <= h_k <= h_max (two inequality rows of unit scale);
  * the duration bound sum_k h_k <= T is carried by an elapsed-time state
    tau (a fifth state): tau_{k+1} = tau_k + h_k (an equality row divided by
    its Jacobian-row norm sqrt(3)), tau_0 = 0 (an initial row) and
    tau_N <= T (a terminal inequality row of unit scale).  The coupling of
    all intervals through the sum thus stays stage-wise, which keeps the
    backward sweep of Sec. III-C applicable;
  * the dynamics rows become (x_{k+1} - x_k - h_k f(x_k, u_k)) / sigma_i
    with the row scales sigma_i of the fixed-step problem (at the instance's
    dt); free motion (mode 12) moves s at the pusher's rate for h_k;
  * the cost is that of the fixed-step problem (no term in h);
  * cold start: the fixed-step cold start, h_k = dt clipped into the bounds,
    tau_k the running sum;
  * the other reading, one optimised time step shared by every interval
    (timing["shared"]): h is a fifth state held constant along the chain
    (h_{k+1} = h_k, an equality row divided by sqrt(2)), free at k = 0, with
    the terminal rows N h_N <= T, h_min <= h_N and h_N <= h_max; the
    dynamics rows use h_k.
Everything else -- the rows of each mode, the PHR augmented Lagrangian, the
damped Newton / Gauss-Newton step with the Lagrangian curvature of the
dynamics rows, the trial-step line search, the multiplier and penalty
updates and the stop test -- is the method of Sec. III-C as the C oracle
(comet_oracle.c) states it, restated here over a general state and control
size.  The step solves the assembled system (H + rho I) dz = -g with a dense
Cholesky factorisation instead of the backward sweep: the two are the same
linear algebra, and H + rho I is positive definite exactly when every
pivot block of the sweep is, so a failed factorisation means the same in
both.  With timing=None the problem is the fixed-step one and the iterates
are those of the C oracle (pinned in tests/test_oracle_timing.py).
"""
from __future__ import annotations

import math

import numpy as np

MODE_FREE = 12
NROW = 11     # rows of the fixed-step problem per interval, fixed positions
NEQ = 5       # rows 0..4 are equalities, 5..10 inequalities
CONVERGED, MAX_ITER, INFEASIBLE, FACTOR_FAIL, NONFINITE = 0, 1, 2, 3, 4

DEFAULTS = dict(max_iters=300, max_factor_retries=8, n_alpha=7, max_inner=40, beta0=100.0, beta_max=1e4,
                beta_growth=10.0, rho0=1e-4, rho_min=1e-4, rho_max=1e6, armijo_c1=1e-4, ls_slack=1e-6,
                eps_primal=1e-6, eps_dual=1e-4, eps_comp=1e-6, omega_ratio=1.0, eta_ratio=0.25, eps_feas=1e-5,
                merit_mu=100.0, beta_ref=1e3, curv_skip=3)


# ---------------------------------------------------------- flop counting
# The method's arithmetic per stage and iteration, counted the way the C
# oracle's counting build counts it (flops.h): one per add, multiply,
# divide, square root, sine or cosine; products with structurally zero
# Jacobian entries are not counted; the symmetric model on its lower
# triangle; rows that the step re-evaluates at the point the measures have
# just taken are not counted, nor are Jacobians for merit values.  The
# step is counted as the backward sweep over w_k = (u_k, x_{k+1}) that the
# method prescribes (Sec. III-C), not as this module's dense factorisation,
# and a failed factorisation as a whole sweep.  Off unless count_flops()
# is active.
_FLOPS = None


def _flops(n):
    global _FLOPS
    if _FLOPS is not None:
        _FLOPS += int(n)


def count_flops(on: bool):
    """Start (on=True, counter at 0) or stop counting; returns the count."""
    global _FLOPS
    got = _FLOPS or 0
    _FLOPS = 0 if on else None
    return got


def _rows_flops(L, free, jac):
    """Values (and with `jac` the nonzero Jacobian entries) of one interval's
    rows: dynamics f (21: body wrench, twist, sine, cosine, f) and its
    Jacobians (24), the four defects (12) and their Jacobian entries (24),
    the mode rows (18); free motion only the defects (12) and d(s)/d(sdot)
    (1).  With timing: the duration column of the defects (one per nonzero
    f_i) and the tau row and the two duration bounds (5), or for the shared
    step the h row (2)."""
    v = 12 if free else 21 + 12 + 18
    j = 1 if free else 24 + 24
    if L.timing:
        v += 2 if L.shared else 5
        j += 1 if free else 4
    return v + (j if jac else 0)


def _curv_flops(L, free):
    """The dynamics rows' Lagrangian curvature on one interval: the second
    derivatives of f (39), yd (12) and the four entries times h (8); with
    timing also the cross terms sum_i yd_i df_i/dv (6 + 14 nonzero products)
    and their 7 entries; free motion only yd and its one cross term."""
    c = 0 if free else 39 + 12 + 8
    if L.timing:
        c += 12 + 3 if free else 6 + 14 + 7
    return c


def _chol_flops(n):
    return sum((2 * j + 1) * (n - j) for j in range(n))


def _sweep_stage_flops(nx, nu):
    """One stage of the backward sweep over w = (u_k, x_{k+1}), n = nu + nx:
    S = H_ww + rho I + V_{k+1} (n + nx(nx+1)/2 + nx), its Cholesky factor,
    the gains for the nx columns of H_wx and the rhs (2 n^2 each), and
    V_k, v_k (lower triangle and vector, 2 n each entry)."""
    n = nu + nx
    return (n + nx * (nx + 1) // 2 + nx + _chol_flops(n) + (nx + 1) * 2 * n * n
            + nx * (nx + 1) // 2 * n * 2 + nx * n * 2)


# ------------------------------------------------------------------ model

def face_frame(inst, face):
    n = [(1.0, 0.0), (0.0, 1.0), (-1.0, 0.0), (0.0, -1.0)][face]
    t = (-n[1], n[0])
    if face % 2 == 0:
        return n, t, 0.5 * inst["side_x"], 0.5 * inst["side_y"]
    return n, t, 0.5 * inst["side_y"], 0.5 * inst["side_x"]


def dynamics(inst, face, x, u):
    """Quasi-static pusher-slider on an ellipsoidal limit surface: f(x, u)
    and its Jacobians Fx (4x4), Fu (4x3); x = (x, y, theta, s), u = (f_n,
    f_t, s_dot)."""
    n, t, a, _ = face_frame(inst, face)
    k, c2 = inst.get("kappa", 1.0), inst["c_ls"] ** 2
    th, s = x[2], x[3]
    fn, ft, sd = u[0], u[1], u[2]
    Fbx, Fby = fn * n[0] + ft * t[0], fn * n[1] + ft * t[1]
    mz = -a * ft - s * fn
    vx, vy, w = k * Fbx, k * Fby, k * mz / c2
    ct, st = math.cos(th), math.sin(th)
    f = np.array([ct * vx - st * vy, st * vx + ct * vy, w, sd])
    Fx = np.zeros((4, 4))
    Fx[0, 2] = -st * vx - ct * vy
    Fx[1, 2] = ct * vx - st * vy
    Fx[2, 3] = -k * fn / c2
    Fu = np.zeros((4, 3))
    Fu[0, 0], Fu[1, 0], Fu[2, 0] = k * (ct * n[0] - st * n[1]), k * (st * n[0] + ct * n[1]), -k * s / c2
    Fu[0, 1], Fu[1, 1], Fu[2, 1] = k * (ct * t[0] - st * t[1]), k * (st * t[0] + ct * t[1]), -k * a / c2
    Fu[3, 2] = 1.0
    return f, Fx, Fu


def dynamics_hessian(inst, face, x, u, yd):
    """sum_i yd_i d^2 f_i over (x, y, theta, s, f_n, f_t, s_dot), 7x7: f is
    bilinear in the forces and (cos theta, sin theta), so only the (theta,
    theta), (theta, f_n), (theta, f_t) and (s, f_n) entries are non-zero."""
    n, t, a, _ = face_frame(inst, face)
    k, c2 = inst.get("kappa", 1.0), inst["c_ls"] ** 2
    th, fn, ft = x[2], u[0], u[1]
    ct, st = math.cos(th), math.sin(th)
    vx, vy = k * (fn * n[0] + ft * t[0]), k * (fn * n[1] + ft * t[1])
    H = np.zeros((7, 7))
    H[2, 2] = -yd[0] * (ct * vx - st * vy) - yd[1] * (st * vx + ct * vy)
    H[2, 4] = H[4, 2] = yd[0] * k * (-st * n[0] - ct * n[1]) + yd[1] * k * (ct * n[0] - st * n[1])
    H[2, 5] = H[5, 2] = yd[0] * k * (-st * t[0] - ct * t[1]) + yd[1] * k * (ct * t[0] - st * t[1])
    H[3, 4] = H[4, 3] = -yd[2] * k / c2
    return H


def dyn_row_scale(inst, i):
    """sigma_i: median over the four faces of the norm of dynamics row i's
    Jacobian at the cold-start reference point (x = 0, u = 0), at the
    instance's dt (Sec. IV-A row scaling)."""
    dt = inst["dt"]
    nrm = []
    for face in range(4):
        _, Fx, Fu = dynamics(inst, face, np.zeros(4), np.zeros(3))
        v = [-(1.0 if i == j else 0.0) - dt * Fx[i, j] for j in range(4)] + [dt * Fu[i, j] for j in range(3)]
        nrm.append(math.sqrt(1.0 + sum(e * e for e in v)))
    nrm.sort()
    return 0.5 * (nrm[1] + nrm[2])


class Layout:
    """Sizes and offsets of one TO: z = (x_0, u_0, x_1, u_1, ..., x_N)."""

    def __init__(self, N, timing):
        self.N, self.timing = N, timing is not None
        self.shared = bool(timing and timing.get("shared"))
        if self.shared:     # h a state: x = (x, y, theta, s, h), u = (f_n, f_t, s_dot)
            self.nx, self.nu, self.nr, self.ni, self.nt = 5, 3, NROW + 1, 3, 3
        elif self.timing:   # h_k a control, tau a state
            self.nx, self.nu, self.nr, self.ni, self.nt = 5, 4, NROW + 3, 4, 1
        else:
            self.nx, self.nu, self.nr, self.ni, self.nt = 4, 3, NROW, 3, 0
        self.stage = self.nx + self.nu
        self.nz = N * self.stage + self.nx
        self.nl = self.ni + N * self.nr + self.nt

    def x(self, k):
        return k * self.stage

    def u(self, k):
        return k * self.stage + self.nx

    def h_local(self):
        """Index of the duration in the local (x_k, u_k, x_{k+1}) vector."""
        return 4 if self.shared else self.nx + 3

    def local(self, k):
        """z indices of interval k's local variables (x_k, u_k, x_{k+1})."""
        a = k * self.stage
        return np.arange(a, a + self.stage + self.nx)

    def row(self, k, r):
        return self.ni + k * self.nr + r


def segment_of(k, length, N):
    return (k * length) // N


def s_row_masked(modes, N, k):
    m0 = modes[segment_of(k, len(modes), N)]
    if m0 == MODE_FREE:
        return True
    if k + 1 >= N:
        return False
    m1 = modes[segment_of(k + 1, len(modes), N)]
    return m1 == MODE_FREE or (m0 // 3) != (m1 // 3)


def interval_rows(inst, mode, smask, xk, uk, xk1, L: Layout, timing, sig):
    """Rows of one interval at fixed positions: scaled values c, presence
    mask, physical factor (physical value = c / scale), inequality flags and
    the local Jacobian over (x_k, u_k, x_{k+1})."""
    nx, nu, nr = L.nx, L.nu, L.nr
    nloc = 2 * nx + nu
    c, mask = np.zeros(nr), np.ones(nr, bool)
    scale, ineq = np.ones(nr), np.zeros(nr, bool)
    ineq[NEQ:NROW] = True
    J = np.zeros((nr, nloc))
    X, U, Y = 0, nx, nx + nu                      # local offsets of x_k, u_k, x_{k+1}
    h = (xk[4] if L.shared else uk[3]) if L.timing else inst["dt"]
    free = mode == MODE_FREE
    face, kind = (0, 3) if free else (mode // 3, mode % 3)
    if free:
        f = np.array([0.0, 0.0, 0.0, uk[2]])
        Fx, Fu = np.zeros((4, 4)), np.zeros((4, 3))
        Fu[3, 2] = 1.0
    else:
        f, Fx, Fu = dynamics(inst, face, xk[:4], uk[:3])
    for i in range(4):
        c[i] = (xk1[i] - xk[i] - h * f[i]) / sig[i]
        J[i, X:X + 4] = (-np.eye(4)[i] - h * Fx[i]) / sig[i]
        J[i, U:U + 3] = -h * Fu[i] / sig[i]
        J[i, Y + i] = 1.0 / sig[i]
        if L.timing:
            J[i, L.h_local()] = -f[i] / sig[i]
        scale[i] = 1.0 / sig[i]
    if smask:
        mask[3] = False
    fn, ft, sd = uk[0], uk[1], uk[2]
    mu = inst["mu"]
    sc = 1.0 / math.sqrt(1.0 + mu * mu)
    if free:
        c[4] = fn
        J[4, U + 0] = 1.0
        mask[5:NROW] = False
    else:
        _, _, _, ell = face_frame(inst, face)
        sgn = -1.0 if kind == 1 else 1.0
        if kind == 0:
            c[4], J[4, U + 2] = sd, 1.0
        else:
            c[4] = sc * (ft + sgn * mu * fn)
            J[4, U + 0], J[4, U + 1], scale[4] = sc * sgn * mu, sc, sc
        c[5], J[5, U + 0], J[5, U + 1], scale[5] = sc * (ft - mu * fn), -sc * mu, sc, sc
        c[6], J[6, U + 0], J[6, U + 1], scale[6] = sc * (-ft - mu * fn), -sc * mu, -sc, sc
        if kind != 0:
            mask[5] = mask[6] = False
        if kind == 0:
            mask[7] = False
        else:
            c[7], J[7, U + 2] = sgn * sd, sgn
        c[8], J[8, U + 0] = -fn, -1.0
        c[9], J[9, X + 3] = xk[3] - ell, 1.0
        c[10], J[10, X + 3] = -xk[3] - ell, -1.0
    if L.shared:
        r2 = math.sqrt(2.0)
        c[11] = (xk1[4] - xk[4]) / r2
        J[11, X + 4], J[11, Y + 4], scale[11] = -1.0 / r2, 1.0 / r2, 1.0 / r2
    elif L.timing:
        r3 = math.sqrt(3.0)
        c[11] = (xk1[4] - xk[4] - uk[3]) / r3
        J[11, X + 4], J[11, U + 3], J[11, Y + 4], scale[11] = -1.0 / r3, -1.0 / r3, 1.0 / r3, 1.0 / r3
        c[12], J[12, U + 3], ineq[12] = timing["h_min"] - uk[3], -1.0, True
        c[13], J[13, U + 3], ineq[13] = uk[3] - timing["h_max"], 1.0, True
    c[~mask] = 0.0
    J[~mask] = 0.0
    return c, mask, scale, ineq, J


def stage_curvature(inst, mode, xk, uk, yd, L: Layout):
    """sum_i yd_i d^2 (-h f_i) over the local (x_k, u_k) block: the
    Lagrangian curvature of the dynamics rows with yd_i = y_i / sigma_i; with
    timing, h is a variable and the cross terms -yd_i df_i/dv appear."""
    nx, nu = L.nx, L.nu
    H = np.zeros((nx + nu, nx + nu))
    h = (xk[4] if L.shared else uk[3]) if L.timing else inst["dt"]
    xs, us = [0, 1, 2, 3], [nx + 0, nx + 1, nx + 2]
    idx = xs + us
    if mode != MODE_FREE:
        Hf = dynamics_hessian(inst, mode // 3, xk[:4], uk[:3], yd)
        H[np.ix_(idx, idx)] -= h * Hf
    if L.timing:
        if mode == MODE_FREE:
            Fx, Fu = np.zeros((4, 4)), np.zeros((4, 3))
            Fu[3, 2] = 1.0
        else:
            _, Fx, Fu = dynamics(inst, mode // 3, xk[:4], uk[:3])
        grad = np.concatenate([yd @ Fx, yd @ Fu])   # sum_i yd_i df_i / dv
        hi = L.h_local()
        H[hi, idx] -= grad
        H[idx, hi] -= grad
    return H


# ----------------------------------------------------------- the problem

class Problem:
    def __init__(self, inst, modes, N, timing=None):
        self.inst, self.modes, self.N, self.timing = inst, tuple(int(m) for m in modes), N, timing
        self.L = Layout(N, timing)
        self.sig = [dyn_row_scale(inst, i) for i in range(4)]
        self.mode_k = [self.modes[segment_of(k, len(self.modes), N)] for k in range(N)]
        self.smask_k = [s_row_masked(self.modes, N, k) for k in range(N)]

    def cold_start(self):
        L, inst = self.L, self.inst
        z = np.zeros(L.nz)
        h = inst["dt"]
        if L.timing:
            h = min(max(h, self.timing["h_min"]), self.timing["h_max"])
        for k in range(self.N + 1):
            a = k / self.N
            for i in range(3):
                z[L.x(k) + i] = (1.0 - a) * inst["start"][i] + a * inst["goal"][i]
            if L.timing:
                z[L.x(k) + 4] = h if L.shared else k * h
        if L.timing and not L.shared:
            for k in range(self.N):
                z[L.u(k) + 3] = h
        return z

    def stage(self, z, k):
        L = self.L
        loc = z[L.local(k)]
        xk, uk, xk1 = loc[:L.nx], loc[L.nx:L.nx + L.nu], loc[L.nx + L.nu:]
        return xk, uk, xk1, interval_rows(self.inst, self.mode_k[k], self.smask_k[k], xk, uk, xk1, L,
                                          self.timing, self.sig)

    def initial_rows(self, z):
        L, inst = self.L, self.inst
        c = [z[L.x(0) + i] - inst["start"][i] for i in range(3)]
        idx = [L.x(0) + i for i in range(3)]
        if L.timing and not L.shared:
            c.append(z[L.x(0) + 4])
            idx.append(L.x(0) + 4)
        return np.array(c), idx

    def terminal_rows(self, z):
        """Terminal inequality rows: values, the z index each depends on and
        its (constant) derivative."""
        if not self.L.timing:
            return np.zeros(0), [], []
        i = self.L.x(self.N) + 4
        if self.L.shared:
            t = self.timing
            return (np.array([self.N * z[i] - t["T"], t["h_min"] - z[i], z[i] - t["h_max"]]), [i, i, i],
                    [float(self.N), -1.0, 1.0])
        return np.array([z[i] - self.timing["T"]]), [i], [1.0]

    def cost(self, z):
        L, inst = self.L, self.inst
        J = sum(inst["w_terminal"] * (z[L.x(self.N) + i] - inst["goal"][i]) ** 2 for i in range(3))
        for k in range(self.N):
            J += inst["w_control"] * float(np.sum(z[L.u(k):L.u(k) + 3] ** 2))
        return J

    def cost_grad(self, z):
        L, inst = self.L, self.inst
        g = np.zeros(L.nz)
        for i in range(3):
            g[L.x(self.N) + i] += 2.0 * inst["w_terminal"] * (z[L.x(self.N) + i] - inst["goal"][i])
        for k in range(self.N):
            g[L.u(k):L.u(k) + 3] += 2.0 * inst["w_control"] * z[L.u(k):L.u(k) + 3]
        return g

    def cost_hess_diag(self):
        L, inst = self.L, self.inst
        d = np.zeros(L.nz)
        for i in range(3):
            d[L.x(self.N) + i] = 2.0 * inst["w_terminal"]
        for k in range(self.N):
            d[L.u(k):L.u(k) + 3] = 2.0 * inst["w_control"]
        return d


def row_y(ineq, lam, beta, c):
    y = lam + beta * c
    return max(y, 0.0) if ineq else y


def row_al(ineq, lam, beta, c):
    if not ineq:
        return lam * c + 0.5 * beta * c * c
    p = max(lam + beta * c, 0.0)
    return (p * p - lam * lam) / (2.0 * beta)


def al_merit(P: Problem, z, lam, beta):
    L = P.L
    phi = P.cost(z)
    _flops(3 * 4 + 3 * P.N * 3)
    ci, _ = P.initial_rows(z)
    for i, c in enumerate(ci):
        phi += row_al(False, lam[i], beta, c)
    for k in range(P.N):
        *_, (c, mask, _, ineq, _) = P.stage(z, k)
        _flops(_rows_flops(L, P.mode_k[k] == MODE_FREE, False) + 6 * int(np.count_nonzero(mask)))
        for r in range(L.nr):
            if mask[r]:
                phi += row_al(ineq[r], lam[L.row(k, r)], beta, c[r])
    ct, _, _ = P.terminal_rows(z)
    for j, c in enumerate(ct):
        phi += row_al(True, lam[L.ni + P.N * L.nr + j], beta, c)
    return phi


def measures(P: Problem, z, lam, beta):
    """y (PHR multiplier estimates), grad of the AL, and the scaled
    violation, physical violation, complementarity and stationarity."""
    L = P.L
    y = np.zeros(L.nl)
    grad = P.cost_grad(z)
    viol = comp = vphys = 0.0
    finite = True
    ci, idx = P.initial_rows(z)
    for i, c in enumerate(ci):
        y[i] = row_y(False, lam[i], beta, c)
        grad[idx[i]] += y[i]
        viol, vphys = max(viol, abs(c)), max(vphys, abs(c))
        finite &= math.isfinite(c)
    for k in range(P.N):
        *_, (c, mask, scale, ineq, J) = P.stage(z, k)
        loc = L.local(k)
        _flops(_rows_flops(L, P.mode_k[k] == MODE_FREE, True))
        for r in range(L.nr):
            q = L.row(k, r)
            if not mask[r]:
                continue
            _flops(6 + (2 * np.count_nonzero(J[r]) if row_y(ineq[r], lam[q], beta, c[r]) != 0.0 else 0))
            finite &= math.isfinite(c[r])
            y[q] = row_y(ineq[r], lam[q], beta, c[r])
            v = max(c[r], 0.0) if ineq[r] else abs(c[r])
            viol, vphys = max(viol, v), max(vphys, v / scale[r])
            if ineq[r]:
                comp = max(comp, abs(y[q] * c[r]))
            if y[q] != 0.0:
                grad[loc] += y[q] * J[r]
    ct, tidx, tder = P.terminal_rows(z)
    for j, c in enumerate(ct):
        q = L.ni + P.N * L.nr + j
        y[q] = row_y(True, lam[q], beta, c)
        viol, vphys = max(viol, max(c, 0.0)), max(vphys, max(c, 0.0))
        comp = max(comp, abs(y[q] * c))
        grad[tidx[j]] += y[q] * tder[j]
    finite &= bool(np.all(np.isfinite(grad)))
    return y, grad, dict(viol=viol, vphys=vphys, comp=comp, stat=float(np.max(np.abs(grad))), finite=finite)


def step(P: Problem, z, lam, beta, rho, curvature):
    """Damped Newton (curvature) or Gauss-Newton step of the AL model:
    (H + rho I) dz = -g with H = cost Hessian + beta A^T A over the active
    rows (+ the dynamics rows' Lagrangian curvature); None when H + rho I is
    not positive definite.  Returns (dz, g)."""
    L = P.L
    H = np.diag(P.cost_hess_diag())
    g = P.cost_grad(z)
    ci, idx = P.initial_rows(z)
    for i, c in enumerate(ci):
        yv = row_y(False, lam[i], beta, c)
        H[idx[i], idx[i]] += beta
        g[idx[i]] += yv
    mflops = [9] * P.N  # the local model's arithmetic per stage
    for k in range(P.N):
        xk, uk, _, (c, mask, _, ineq, J) = P.stage(z, k)
        loc = L.local(k)
        for r in range(L.nr):
            if not mask[r]:
                continue
            q = L.row(k, r)
            if ineq[r] and not (lam[q] + beta * c[r] > 0.0):
                continue
            nnz = np.count_nonzero(J[r])
            mflops[k] += 2 + 3 * nnz + nnz * (nnz + 1)
            yv = row_y(ineq[r], lam[q], beta, c[r])
            g[loc] += yv * J[r]
            H[np.ix_(loc, loc)] += beta * np.outer(J[r], J[r])
        if curvature:
            mflops[k] += _curv_flops(L, P.mode_k[k] == MODE_FREE)
            yd = np.array([row_y(False, lam[L.row(k, r)], beta, c[r]) / P.sig[r] if mask[r] else 0.0
                           for r in range(4)])
            xu = loc[:L.nx + L.nu]
            H[np.ix_(xu, xu)] += stage_curvature(P.inst, P.mode_k[k], xk, uk, yd, L)
    ct, tidx, tder = P.terminal_rows(z)
    for j, c in enumerate(ct):
        q = L.ni + P.N * L.nr + j
        if lam[q] + beta * c > 0.0:
            H[tidx[j], tidx[j]] += beta * tder[j] * tder[j]
            g[tidx[j]] += row_y(True, lam[q], beta, c) * tder[j]
    H += rho * np.eye(L.nz)
    try:
        C = np.linalg.cholesky(H)
    except np.linalg.LinAlgError:
        if _FLOPS is not None:
            _flops(_failed_sweep_flops(P, H, mflops))
        return None, g
    _flops(sum(mflops) + P.N * (_sweep_stage_flops(L.nx, L.nu) + (L.nu + L.nx) * 2 * L.nx)
           + _chol_flops(L.nx) + 2 * L.nx * L.nx)
    dz = -np.linalg.solve(C.T, np.linalg.solve(C, g))
    return dz, g


def _failed_sweep_flops(P: Problem, H, mflops):
    """What the backward sweep counts before it meets the non-positive pivot:
    the sweep is the Cholesky factorisation of H + rho I with the variables
    in the order w_{N-1}, ..., w_0, x_0 (w_k = (u_k, x_{k+1})), so LAPACK's
    dpotrf on that ordering finds the same pivot; the stages before it are
    counted whole, the failing one up to and including that column."""
    from scipy.linalg import lapack

    L = P.L
    n = L.nu + L.nx
    order = []
    for k in range(P.N - 1, -1, -1):
        order += list(range(L.u(k), L.u(k) + L.nu)) + list(range(L.x(k + 1), L.x(k + 1) + L.nx))
    order += list(range(L.x(0), L.x(0) + L.nx))
    _, info = lapack.dpotrf(H[np.ix_(order, order)], lower=1)
    p = int(info) - 1
    b, j = divmod(p, n)
    part = lambda m, jj: sum((2 * q + 1) * (m - q) for q in range(jj + 1))  # noqa: E731
    full = _sweep_stage_flops(L.nx, L.nu)
    if b < P.N:  # stage k = N - 1 - b: model, S, its factor up to column j
        done = sum(mflops[P.N - 1 - i] for i in range(b + 1))
        return done + b * full + n + L.nx * (L.nx + 1) // 2 + L.nx + part(n, j)
    return sum(mflops) + P.N * full + part(L.nx, p - P.N * n)


def trial_step(phi0, D, merit_at, n_alpha, c1, ls_slack):
    """The largest alpha = 2^-i (i < n_alpha) meeting the Armijo condition
    phi(alpha) <= phi(0) + c1 alpha D (D the directional derivative), 0 if
    none does.  When |D| <= ls_slack |phi(0)| the merit cannot rank the
    trials and the full step is taken if it raises phi by at most that."""
    slack = ls_slack * abs(phi0)
    flat = abs(D) <= slack
    for i in range(n_alpha):
        a = math.ldexp(1.0, -i)
        phi = merit_at(a)
        if phi <= phi0 + c1 * a * D or (flat and i == 0 and phi <= phi0 + slack):
            return a
    return 0.0


def solve(inst, modes, N=None, timing=None, warm=None, **over):
    """The method of Sec. III-C on one order; timing = None (fixed step),
    {"h_min", "h_max", "T"} (a duration per interval) or the same with
    "shared": True (one step for every interval).  Options override
    DEFAULTS (the C oracle's).  Returns (z, lam, result dict); z in the
    interleaved layout of Layout."""
    o = dict(DEFAULTS, **over)
    if N is None:
        N = int(inst["knots_per_segment"]) * len(modes)
    P = Problem(inst, modes, N, timing)
    L = P.L
    z = P.cold_start() if warm is None else np.array(warm, dtype=np.float64)
    lam = np.zeros(L.nl)
    beta, rho, eta = o["beta0"], o["rho0"], math.inf
    inner = n_outer = n_rej = curv_hold = n_curv_fail = 0
    status = MAX_ITER
    it = 0
    m = None
    for it in range(o["max_iters"]):
        y, grad, m = measures(P, z, lam, beta)
        if not m["finite"]:
            status = NONFINITE
            break
        # stop test of Sec. III-C as in the C oracle: stationarity relative to
        # max(1, |J|), scaled rows within eps_primal, physical rows within
        # half eps_feas
        _flops(3 * 4 + 3 * N * 3)
        eps_d = o["eps_dual"] * max(1.0, beta / o["beta_ref"]) * max(1.0, abs(P.cost(z)))
        if (m["viol"] <= o["eps_primal"] and m["vphys"] <= 0.5 * o["eps_feas"] and m["stat"] <= eps_d
                and m["comp"] <= o["eps_comp"]):
            lam = y.copy()
            status = CONVERGED
            break
        omega = max(eps_d, o["omega_ratio"] * m["viol"])
        solved = m["stat"] <= omega
        if solved or inner >= o["max_inner"]:
            lam = y.copy()
            if solved and m["viol"] > o["eps_primal"] and m["viol"] > o["eta_ratio"] * eta:
                beta = min(o["beta_max"], beta * o["beta_growth"])
            eta = m["viol"]
            inner = 0
            n_outer += 1
        dz = None
        if curv_hold == 0:
            dz, g = step(P, z, lam, beta, rho, True)
            if dz is None:
                n_curv_fail += 1
                curv_hold = o["curv_skip"]
        else:
            curv_hold -= 1
        r = 0
        while dz is None and r <= o["max_factor_retries"]:
            if r > 0:
                rho = min(o["rho_max"], rho * 10.0)
            dz, g = step(P, z, lam, beta, rho, False)
            r += 1
        inner += 1
        if dz is None:
            n_rej += 1
            continue
        D = float(np.dot(g, dz))
        _flops(2 * L.nz)
        phi0 = al_merit(P, z, lam, beta)

        def merit_at(a):
            _flops(2 * L.nz)  # the trial point z + a dz
            return al_merit(P, z + a * dz, lam, beta)

        alpha = trial_step(phi0, D, merit_at, o["n_alpha"], o["armijo_c1"], o["ls_slack"])
        if alpha > 0.0:
            _flops(2 * L.nz)
            z = z + alpha * dz
            rho = max(o["rho_min"], rho / 10.0)
        else:
            rho = min(o["rho_max"], rho * 10.0)
            n_rej += 1
    else:
        it = o["max_iters"]
    if status != CONVERGED:
        y, grad, m = measures(P, z, lam, beta)
    _flops(3 * 4 + 3 * N * 3)
    cost = P.cost(z)
    if not math.isfinite(cost) or not m["finite"]:
        status = NONFINITE
    if status == CONVERGED and not (m["vphys"] <= o["eps_feas"]):
        status = INFEASIBLE
    res = dict(cost=cost, viol=m["vphys"], stat=m["stat"], comp=m["comp"], status=status, iters=it,
               n_outer=n_outer, n_rejected=n_rej, n_curv_fail=n_curv_fail, beta=beta, rho=rho,
               merit=cost + o["merit_mu"] * max(m["vphys"] - o["eps_feas"], 0.0))
    return z, (lam if status == CONVERGED else y), res


def all_rows(P: Problem, z):
    """Every row at z in multiplier order (initial, per interval, terminal):
    values c, dense Jacobian A over z, inequality flags and presence mask."""
    L = P.L
    c = np.zeros(L.nl)
    A = np.zeros((L.nl, L.nz))
    ineq = np.zeros(L.nl, bool)
    mask = np.ones(L.nl, bool)
    ci, idx = P.initial_rows(z)
    for i, v in enumerate(ci):
        c[i], A[i, idx[i]] = v, 1.0
    for k in range(P.N):
        *_, (ck, mk, _, ik, Jk) = P.stage(z, k)
        loc = L.local(k)
        for r in range(L.nr):
            q = L.row(k, r)
            c[q], mask[q], ineq[q] = ck[r], mk[r], ik[r]
            A[q, loc] = Jk[r]
    ct, tidx, tder = P.terminal_rows(z)
    for j, v in enumerate(ct):
        q = L.ni + P.N * L.nr + j
        c[q], A[q, tidx[j]], ineq[q] = v, tder[j], True
    return c, A, ineq, mask


def durations(inst, modes, z, N=None, timing=None):
    """The interval durations h_k of an interleaved solution (the instance's
    dt when timing is fixed)."""
    if N is None:
        N = int(inst["knots_per_segment"]) * len(modes)
    L = Layout(N, timing)
    if not L.timing:
        return np.full(N, inst["dt"])
    if L.shared:
        return np.array([z[L.x(k) + 4] for k in range(N)])
    return np.array([z[L.u(k) + 3] for k in range(N)])


def interleave_c_traj(tr, N):
    """The C oracle's component-major trajectory as the interleaved z of the
    fixed-step layout."""
    z = np.zeros(7 * N + 4)
    for k in range(N + 1):
        for i in range(4):
            z[7 * k + i] = tr[i * (N + 1) + k]
    for k in range(N):
        for j in range(3):
            z[7 * k + 4 + j] = tr[4 * (N + 1) + j * N + k]
    return z


def flops_per_stage_iteration(insts, orders, timing, **over):
    """(flops per stage-iteration, total flops, stage-iterations) of the
    method over the given (instance index, modes) orders solved with these
    options: the count above divided by the sum over the orders of
    iterations x intervals."""
    total = work = 0
    for i, modes in orders:
        count_flops(True)
        try:
            _, _, r = solve(insts[i], modes, timing=timing, **over)
        finally:
            f = count_flops(False)
        total += f
        work += r["iters"] * int(insts[i]["knots_per_segment"]) * len(modes)
    return total / max(work, 1), total, work
