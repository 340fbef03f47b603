"""FP64 CPU oracle of the learned proposal -- TEST INFRASTRUCTURE ONLY.

The learned proposal is not part of the paper: it is a cost and warm-start
predictor placed in front of the expansion of Algorithm 1 (Sec. III-B).  A
4-layer MLP of width 256 with GELU maps the features of an (instance, mode
order) pair to the log of the order's merit (Eq. search_merit) and to the
controls of its solved trajectory; it orders and prunes the neighbours of
the beam, and its controls warm-start the TOs of Eq. mode_nlp.

Everything here is the plain definition written out in float64 numpy, on
BF16-rounded (round-to-nearest-even) weights and inputs, so that it can be
compared with the GPU's BF16 tensor-core path:

  * ``bf16``           round-to-nearest-even of float32 values to bfloat16;
  * ``features``       the input vector of one order (layout below);
  * ``forward``        Z_l = H_{l-1} W_l^T + b_l, H_l = GELU(Z_l) for the
                       hidden layers, Y = H_3 W_4^T + b_4 (no activation);
  * ``loss``           L = (1/B) sum_{b,j} Omega_bj (Y_bj - T_bj)^2;
  * ``backward``       the exact gradient of L by the chain rule;
  * ``adamw``          one AdamW step (decoupled weight decay, bias-corrected
                       moments).

GELU is the tanh form of Hendrycks and Gimpel, 0.5 x (1 + tanh(a (x + b x^3)))
with a = sqrt(2 / pi), b = 0.044715; its derivative follows by the chain
rule.  With ``round_hidden`` the hidden activations (and, in
the backward pass, the layer gradients) are rounded to BF16 between layers,
as the GPU stores them; the arithmetic stays float64.

Feature layout of an order m of length L on an instance (in_dim = 12 +
13 L_max, padded with zeros to a multiple of 64): start pose (x, y, theta),
goal pose, 10 side_x, 10 side_y, the goal in the start frame (3 x', 3 y',
theta_g - theta_s), one zero, then one 13-way one-hot per segment slot
i < L_max (entries 0..11 = the mode m_i, entry 12 = blank for i >= L).

Output layout (out_dim = 1 + 3 N_max, padded to a multiple of 16): entry 0
is log M_hat; entry 1 + c N_max + k is control component c (f_n, f_t, s_dot)
of interval k.

Bimanual task (``bim_dims``, ``bim_features``, ``bim_targets``, ``bim_warm``):
the 507 modes m = 169 g + 13 h_L + h_R (ground g, hands h_L, h_R) enter as a
factored one-hot of 30 entries per slot (g at 0..2, h_L at 3..15, h_R at
16..28, blank at 29); the instance part is the start pose (x, z, theta), the
goal pose, 10 side_x, 10 side_y, 3 (x_g - x_s), 3 (z_g - z_s), theta_g -
theta_s and the mass.  Outputs: log M_hat, then the 12 controls (xd, zd,
thd, fn_L, ft_L, sd_L, fn_R, ft_R, sd_R, lam_n, lam_t, p_c) of every
interval, the forces in units of the box's weight m g (g = 9.81).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (round to nearest, ties to even) and return float64.

    The value is first taken as float32 (the GPU's storage type before
    conversion); NaN stays NaN."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isnan(a), np.nan, out).reshape(a.shape)


def bf16_bits(x) -> np.ndarray:
    """The uint16 bit patterns of bf16(x)."""
    return (bf16(x).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def from_bf16_bits(b) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


GELU_A = np.sqrt(2.0 / np.pi)
GELU_B = 0.044715


def gelu(x):
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * x * (1.0 + np.tanh(GELU_A * (x + GELU_B * x ** 3)))


def gelu_grad(x):
    x = np.asarray(x, dtype=np.float64)
    t = np.tanh(GELU_A * (x + GELU_B * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * GELU_A * (1.0 + 3.0 * GELU_B * x * x)


def gelu_erf(x):
    """The exact form 0.5 x (1 + erf(x / sqrt 2)) (for comparison only)."""
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def pad_to(n: int, m: int) -> int:
    return (n + m - 1) // m * m


def dims(l_max: int, n_max: int, width: int = 256, n_modes: int = 12):
    """(in_dim, width, out_dim) of the proposal for an instance family."""
    return pad_to(12 + (n_modes + 1) * l_max, 64), width, pad_to(1 + 3 * n_max, 16)


def features(inst: dict, modes, l_max: int, in_dim: int, n_modes: int = 12) -> np.ndarray:
    s, g = np.asarray(inst["start"], float), np.asarray(inst["goal"], float)
    x = np.zeros(in_dim)
    x[0:3] = s
    x[3:6] = g
    x[6] = 10.0 * inst["side_x"]
    x[7] = 10.0 * inst["side_y"]
    # the goal in the start frame (the quasi-static model is invariant under
    # planar rigid motions of the world frame): 3 R(-theta_s)(g - s), dtheta
    d = g[:2] - s[:2]
    c, sn = np.cos(s[2]), np.sin(s[2])
    x[8] = 3.0 * (c * d[0] + sn * d[1])
    x[9] = 3.0 * (-sn * d[0] + c * d[1])
    x[10] = g[2] - s[2]
    for i in range(l_max):
        e = modes[i] if i < len(modes) else n_modes
        x[12 + (n_modes + 1) * i + e] = 1.0
    return x


def param_shapes(in_dim: int, width: int, out_dim: int, n_layers: int = 4):
    d = [in_dim] + [width] * (n_layers - 1) + [out_dim]
    return [((d[l + 1], d[l]), (d[l + 1],)) for l in range(n_layers)]


def unflatten(flat, in_dim, width, out_dim, n_layers=4):
    """Flat float32 parameter vector [W_1, b_1, ..., W_4, b_4] (W row-major
    [out][in]) -> list of (W, b) in float64."""
    out, o = [], 0
    flat = np.asarray(flat, dtype=np.float64)
    for (ws, bs) in param_shapes(in_dim, width, out_dim, n_layers):
        nw, nb = ws[0] * ws[1], bs[0]
        out.append((flat[o:o + nw].reshape(ws), flat[o + nw:o + nw + nb].copy()))
        o += nw + nb
    return out


def flatten(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def forward(params, X, round_hidden=False, bf16_weights=True):
    """Returns (Y, cache).  X and the weights are BF16-rounded (the GPU's
    operands); biases stay full precision."""
    H = bf16(X) if bf16_weights else np.asarray(X, np.float64)
    cache = {"H": [H], "Z": []}
    n = len(params)
    for l, (W, b) in enumerate(params):
        Wq = bf16(W) if bf16_weights else W
        Z = H @ Wq.T + b
        cache["Z"].append(Z)
        if l < n - 1:
            H = gelu(Z)
            if round_hidden:
                H = bf16(H)
            cache["H"].append(H)
        else:
            H = Z
    return H, cache


def loss(Y, T, Omega) -> float:
    return float(np.sum(Omega * (Y - T) ** 2) / Y.shape[0])


def backward(params, cache, Y, T, Omega, round_hidden=False, bf16_weights=True):
    """Gradient of ``loss`` w.r.t. every W_l and b_l (list of (dW, db))."""
    B = Y.shape[0]
    G = 2.0 * Omega * (Y - T) / B          # dL/dZ of the output layer
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        Wq = bf16(W) if bf16_weights else W
        if round_hidden:
            G = bf16(G)
        grads[l] = (G.T @ cache["H"][l], G.sum(axis=0))
        if l > 0:
            dH = G @ Wq
            G = dH * gelu_grad(cache["Z"][l - 1])
    return grads


def adamw(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step at step count t >= 1; returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    p = p - lr * (mh / (np.sqrt(vh) + eps) + wd * p)
    return p, m, v


def targets(cost, viol, status, traj_controls, N, n_max, out_dim, lambda_w=1.0, merit_mu=100.0, eps_feas=1e-5):
    """Training target T and weight Omega of one evaluated order.

    T_0 = log max(M_hat, 1e-12), M_hat = J_hat + merit_mu max(v_hat - eps_feas,
    0) (Eq. search_merit), weight 1 unless the TO ended NONFINITE (status 4);
    T_{1 + c n_max + k} = control c of interval k (traj_controls[c][k]) for
    k < N, weight lambda_w / (3 N) when the TO CONVERGED (status 0), else 0."""
    T = np.zeros(out_dim)
    Om = np.zeros(out_dim)
    m = cost + merit_mu * max(viol - eps_feas, 0.0)
    if status != 4 and np.isfinite(m):
        T[0] = np.log(max(m, 1e-12))
        Om[0] = 1.0
    if status == 0:
        for c in range(3):
            for k in range(N):
                T[1 + c * n_max + k] = traj_controls[c][k]
                Om[1 + c * n_max + k] = lambda_w / (3.0 * N)
    return T, Om


# ------------------------------------------------------------ bimanual task

GRAV = 9.81
BIM_SLOT = 30
BIM_FORCES = (3, 4, 6, 7, 9, 10)   # fn_L, ft_L, fn_R, ft_R, lam_n, lam_t


def bim_dims(l_max: int, n_max: int, width: int = 256):
    """(in_dim, width, out_dim) of the proposal for a bimanual family."""
    return pad_to(12 + BIM_SLOT * l_max, 64), width, pad_to(1 + 12 * n_max, 16)


def bim_features(inst: dict, modes, l_max: int, in_dim: int) -> np.ndarray:
    s, g = np.asarray(inst["start"], float), np.asarray(inst["goal"], float)
    x = np.zeros(in_dim)
    x[0:3] = s
    x[3:6] = g
    x[6] = 10.0 * inst["side_x"]
    x[7] = 10.0 * inst["side_y"]
    x[8] = 3.0 * (g[0] - s[0])
    x[9] = 3.0 * (g[1] - s[1])
    x[10] = g[2] - s[2]
    x[11] = inst["mass"]
    for i in range(l_max):
        base = 12 + BIM_SLOT * i
        if i < len(modes):
            m = int(modes[i])
            x[base + m // 169] = 1.0
            x[base + 3 + (m // 13) % 13] = 1.0
            x[base + 16 + m % 13] = 1.0
        else:
            x[base + BIM_SLOT - 1] = 1.0
    return x


def bim_targets(cost, viol, status, traj_controls, N, n_max, out_dim, mass, lambda_w=1.0, merit_mu=100.0,
                eps_feas=1e-5):
    """As ``targets`` for the 12 bimanual controls (traj_controls[c][k]),
    forces divided by m g, control weights lambda_w / (12 N)."""
    T = np.zeros(out_dim)
    Om = np.zeros(out_dim)
    m = cost + merit_mu * max(viol - eps_feas, 0.0)
    if status != 4 and np.isfinite(m):
        T[0] = np.log(max(m, 1e-12))
        Om[0] = 1.0
    if status == 0:
        for c in range(12):
            scale = 1.0 / (mass * GRAV) if c in BIM_FORCES else 1.0
            for k in range(N):
                T[1 + c * n_max + k] = traj_controls[c][k] * scale
                Om[1 + c * n_max + k] = lambda_w / (12.0 * N)
    return T, Om


def bim_warm(inst: dict, N: int, n_max: int, y) -> np.ndarray:
    """Warm start of a bimanual order from the outputs y: the cold start's
    poses (linear from start to goal, hand offsets 0) and the predicted
    controls, forces times m g; trajectory layout x[5][n_max+1], u[12][n_max]."""
    w = np.zeros(5 * (n_max + 1) + 12 * n_max)
    s, g = np.asarray(inst["start"], float), np.asarray(inst["goal"], float)
    for k in range(N + 1):
        a = k / N
        for c in range(3):
            w[c * (n_max + 1) + k] = (1.0 - a) * s[c] + a * g[c]
    mg = inst["mass"] * GRAV
    for c in range(12):
        for k in range(N):
            w[5 * (n_max + 1) + c * n_max + k] = y[1 + c * n_max + k] * (mg if c in BIM_FORCES else 1.0)
    return w
