"""Seeded synthetic inputs for the CoMET hot path.

This module is shared by the CUDA path's tests/bench and by the oracle.  It
draws instances and lists mode sequences; it holds none of the method's
arithmetic (no dynamics, rows, costs or solver steps).

Workloads (all synthetic; the paper's benchmark poses and slider geometry
are not used):
  * ``push_l2``  -- square slider 0.09 m, c = 0.04 m, mu = 0.3, 12 modes per
    segment (face 0..3 x stick/slide+/slide-), sequence length 2 (144
    sequences), 8 intervals per segment, dt = 0.1 s, start at the origin,
    goal x, y ~ U[-0.2, 0.2] m, theta ~ U[-pi/2, pi/2] (seeds 0..31).
  * ``push_l4``  -- same slider, sequence length 4 (20,736 sequences), 20
    intervals per segment, start and goal x, y ~ U[-0.3, 0.3] m,
    theta ~ U[-pi, pi] (seeds 0..63), cold start.
  * ``push_mixed`` -- rectangles of side 0.05-0.15 m and aspect 1-3,
    mu ~ U[0.2, 0.6], sequence caps 1..6, 10..30 intervals per segment.
Every draw uses numpy's PCG64 (``np.random.default_rng(seed)``) in the order
stated in each generator.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

N_MODES_PUSH = 12          # face 0..3 x {stick, slide+, slide-}
MAX_SEGMENTS = 16          # longest mode sequence carried by the ABI


def _instance(side_x, side_y, c_ls, mu, dt, K, start, goal, L):
    return {
        "task": 0,
        "side_x": float(side_x), "side_y": float(side_y), "c_ls": float(c_ls),
        "mu": float(mu), "dt": float(dt), "kappa": 1.0,
        "knots_per_segment": int(K), "max_segments": int(L), "n_modes": N_MODES_PUSH,
        "start": [float(v) for v in start], "goal": [float(v) for v in goal],
        "w_terminal": 10.0, "w_control": 0.1,
    }


def push_l2_instance(seed: int) -> dict:
    """Square slider, L = 2, K = 8; goal drawn x, y, theta in that order."""
    rng = np.random.default_rng(seed)
    gx = rng.uniform(-0.2, 0.2)
    gy = rng.uniform(-0.2, 0.2)
    gth = rng.uniform(-math.pi / 2, math.pi / 2)
    return _instance(0.09, 0.09, 0.04, 0.3, 0.1, 8, (0.0, 0.0, 0.0), (gx, gy, gth), 2)


def push_l2_straight(d: float = 0.1) -> dict:
    """The straight-push special case: start at the origin, goal (d, 0, 0)."""
    return _instance(0.09, 0.09, 0.04, 0.3, 0.1, 8, (0.0, 0.0, 0.0), (d, 0.0, 0.0), 2)


def push_l4_instance(seed: int) -> dict:
    """Square slider, L = 4, K = 20; start x, y, theta then goal x, y, theta."""
    rng = np.random.default_rng(seed)
    v = [rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(-math.pi, math.pi),
         rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(-math.pi, math.pi)]
    return _instance(0.09, 0.09, 0.04, 0.3, 0.1, 20, v[:3], v[3:], 4)


def mean_radius_rect(a: float, b: float, n: int = 400) -> float:
    """(1/A) * integral of |r| over an a x b rectangle centred at the origin
    (midpoint quadrature); the limit-surface radius of a uniformly pressed
    rectangle used for the mixed workload's instances."""
    xs = (np.arange(n) + 0.5) / n * a - a / 2
    ys = (np.arange(n) + 0.5) / n * b - b / 2
    X, Y = np.meshgrid(xs, ys)
    return float(np.mean(np.hypot(X, Y)))


def push_mixed_instance(seed: int) -> dict:
    """Rectangular slider of the mixed workload.  Draw order: side, aspect,
    orientation of the long side (x or y), mu, cap L in 1..6, K in 10..30,
    start x, y, theta, goal x, y, theta."""
    rng = np.random.default_rng(10_000 + seed)
    side = rng.uniform(0.05, 0.15)
    aspect = rng.uniform(1.0, 3.0)
    long_x = rng.uniform() < 0.5
    mu = rng.uniform(0.2, 0.6)
    L = int(rng.integers(1, 7))
    K = int(rng.integers(10, 31))
    v = [rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(-math.pi, math.pi),
         rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(-math.pi, math.pi)]
    a, b = (side, side / aspect) if long_x else (side / aspect, side)
    return _instance(a, b, mean_radius_rect(a, b), mu, 0.1, K, v[:3], v[3:], L)


def all_sequences(n_modes: int, length: int) -> np.ndarray:
    """Every sequence of `length` modes, lexicographic with the first
    segment most significant: uint8 [n_modes**length, length]."""
    return np.array(list(itertools.product(range(n_modes), repeat=length)), dtype=np.uint8).reshape(
        -1, length)


def sequences_up_to(n_modes: int, max_len: int) -> list[tuple[int, ...]]:
    """All sequences of length 1..max_len, shorter first, each length
    lexicographic."""
    out: list[tuple[int, ...]] = []
    for L in range(1, max_len + 1):
        out.extend(itertools.product(range(n_modes), repeat=L))
    return out


def random_sequences(seed: int, n: int, n_modes: int, length: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, n_modes, size=(n, length), dtype=np.uint8)


def pad_sequences(seqs, lmax: int = MAX_SEGMENTS) -> tuple[np.ndarray, np.ndarray]:
    """(modes uint8 [n, lmax] zero padded, lens int32 [n])."""
    n = len(seqs)
    modes = np.zeros((n, lmax), dtype=np.uint8)
    lens = np.zeros(n, dtype=np.int32)
    for i, s in enumerate(seqs):
        s = list(s)
        modes[i, : len(s)] = s
        lens[i] = len(s)
    return modes, lens


def mlp_params(in_dim: int, width: int, out_dim: int, seed: int, n_layers: int = 4, bias_scale: float = 0.0):
    """Seeded weights of an MLP in_dim -> width x (n_layers-1) -> out_dim:
    W_l ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) row-major [out][in], biases
    ~ U(-bias_scale, bias_scale).  Returns a list of (W, b) float64 arrays."""
    rng = np.random.default_rng(seed)
    d = [in_dim] + [width] * (n_layers - 1) + [out_dim]
    out = []
    for l in range(n_layers):
        a = 1.0 / np.sqrt(d[l])
        out.append((rng.uniform(-a, a, (d[l + 1], d[l])), rng.uniform(-bias_scale, bias_scale, d[l + 1])))
    return out


def bimanual_instance(seed: int) -> dict:
    """Bimanual box flip in the vertical plane.  Draw order: width, height
    (full sides U[0.1, 0.3] m), mass U[0.5, 2] kg, rotation sign sigma (+-1),
    offset U[0, 0.3].  Ground friction 0.5, hand friction 0.5, dt 0.05 s, 15
    knots per segment, up to 6 segments, 507 modes per segment.  Start: the
    box resting on its bottom face at the origin (x, z, theta) = (0, h/2, 0);
    goal: theta_g = pi/2 + sigma offset, the box turned about its lower-left
    corner (x_g, z_g follow from that rotation)."""
    rng = np.random.default_rng(20_000 + seed)
    w = rng.uniform(0.1, 0.3)
    h = rng.uniform(0.1, 0.3)
    mass = rng.uniform(0.5, 2.0)
    sigma = 1.0 if rng.uniform() < 0.5 else -1.0
    off = rng.uniform(0.0, 0.3)
    ax, az = 0.5 * w, 0.5 * h
    th = math.pi / 2 + sigma * off
    # corner (-ax, -az) of the start pose sits at (-ax, 0); rotating the box
    # about it by th puts the centre at corner + R(th) (ax, az)
    xg = -ax + ax * math.cos(th) - az * math.sin(th)
    zg = ax * math.sin(th) + az * math.cos(th)
    return {
        "task": 1, "side_x": w, "side_y": h, "c_ls": 0.0, "mu": 0.5, "dt": 0.05, "kappa": 1.0,
        "knots_per_segment": 15, "max_segments": 6, "n_modes": 507,
        "start": [0.0, az, 0.0], "goal": [xg, zg, th], "w_terminal": 10.0, "w_control": 0.1,
        "mass": mass, "ground_mu": 0.5,
    }


def bimanual_mode(ground: int, hand_l: int, hand_r: int) -> int:
    """Mode index of (ground 0 stick / 1 slide / 2 pivot, hand codes 0 none or
    1 + 3 face + kind)."""
    return ground * 169 + hand_l * 13 + hand_r


def push_grammar_instance(seed: int) -> dict:
    """Square box of the grammar experiments: the push_l4 slider and poses
    (same draws), the 13-mode pushing alphabet (mode 12 = free motion),
    orders of at most 8 segments of K = 10 intervals."""
    d = push_l4_instance(seed)
    d["n_modes"] = 13
    d["max_segments"] = 8
    d["knots_per_segment"] = 10
    return d


def admissible_push_orders(cap: int) -> list[tuple[int, ...]]:
    """Seed orders for the pushing grammar of the four-faced box: every order
    of 1..cap segments over {stick on face f = mode 3 f, free motion = 12}
    that starts in free motion, never repeats a mode in consecutive
    segments, and switches directly between contacts only on adjacent faces;
    by length, then lexicographically (601 orders at cap 6, 6,297 at 8)."""
    alpha = (0, 3, 6, 9, 12)
    out, level = [], [(12,)]
    for _ in range(cap):
        out += level
        nxt = []
        for s in level:
            for m in alpha:
                a = s[-1]
                if m == a:
                    continue
                if a != 12 and m != 12 and (a // 3 - m // 3) % 4 not in (1, 3):
                    continue
                nxt.append(s + (m,))
        level = nxt
    return out
