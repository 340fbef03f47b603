"""Test helpers: layout conversions and a dense assembly of the AL
Gauss-Newton / Newton system used to pin the oracle's backward sweep."""
import numpy as np

import oracle


def to_interleaved(tr, N):
    X = tr[: 4 * (N + 1)].reshape(4, N + 1)
    U = tr[4 * (N + 1):].reshape(3, N)
    z = np.zeros(7 * N + 4)
    for k in range(N + 1):
        z[7 * k: 7 * k + 4] = X[:, k]
    for k in range(N):
        z[7 * k + 4: 7 * k + 7] = U[:, k]
    return z


def to_component(z, N):
    X = np.zeros((4, N + 1))
    U = np.zeros((3, N))
    for k in range(N + 1):
        X[:, k] = z[7 * k: 7 * k + 4]
    for k in range(N):
        U[:, k] = z[7 * k + 4: 7 * k + 7]
    return np.concatenate([X.ravel(), U.ravel()])


def cost_grad_hess(inst, N, z):
    g = np.zeros(7 * N + 4)
    h = np.zeros(7 * N + 4)
    for k in range(N):
        g[7 * k + 4: 7 * k + 7] = 2 * inst["w_control"] * z[7 * k + 4: 7 * k + 7]
        h[7 * k + 4: 7 * k + 7] = 2 * inst["w_control"]
    g[7 * N: 7 * N + 3] = 2 * inst["w_terminal"] * (z[7 * N: 7 * N + 3] - np.array(inst["goal"]))
    h[7 * N: 7 * N + 3] = 2 * inst["w_terminal"]
    return g, np.diag(h)


def multipliers(inst, modes, N, tr, lam, beta):
    """(y, active, c, is_dyn) over the 3 + 11N rows (PHR estimates)."""
    c, mask, _, ci = oracle.rows(inst, modes, N, tr)
    cc = np.concatenate([ci, c.ravel()])
    mk = np.concatenate([np.ones(3, bool), mask.ravel().astype(bool)])
    ineq = np.zeros(3 + 11 * N, bool)
    ineq[3:] = np.tile(np.arange(11) >= 5, N)
    dyn = np.zeros(3 + 11 * N, bool)
    dyn[3:] = np.tile(np.arange(11) < 4, N)
    y = lam + beta * cc
    act = mk.copy()
    act[ineq] &= y[ineq] > 0
    y = np.where(act, y, 0.0)
    return y, act, cc, dyn & mk


def dense_step(inst, modes, N, tr, lam, beta, rho, curvature):
    """Dense solve of (H + rho I) dz = -g assembled row by row."""
    z = to_interleaved(tr, N)
    J = oracle.dense_jacobian(inst, modes, N, tr)
    y, act, _, dyn = multipliers(inst, modes, N, tr, lam, beta)
    gJ, HJ = cost_grad_hess(inst, N, z)
    g = gJ + J.T @ y
    H = HJ + beta * J[act].T @ J[act] + rho * np.eye(len(z))
    if curvature:
        # sum_i y_i d^2 c_i over dynamics rows, by central differences of J^T y
        yd = np.where(dyn, y, 0.0)
        h = 1e-6
        C = np.zeros_like(H)
        for j in range(len(z)):
            e = np.zeros(len(z)); e[j] = h
            Jp = oracle.dense_jacobian(inst, modes, N, to_component(z + e, N))
            Jm = oracle.dense_jacobian(inst, modes, N, to_component(z - e, N))
            C[:, j] = (Jp.T @ yd - Jm.T @ yd) / (2 * h)
        H = H + 0.5 * (C + C.T)
    return -np.linalg.solve(H, g), g
