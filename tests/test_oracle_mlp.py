"""Pins of the learned proposal's FP64 oracle (oracle/mlp.py) to facts that
do not come from the oracle itself: the tanh-form GELU by hand with the
library tanh and its distance to the exact (erf) GELU, the bfloat16 rounding
rule, central differences of the loss, closed forms of the first AdamW step,
and a width-1 network evaluated by hand."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import mlp


def test_bf16_round_to_nearest_even():
    one = 1.0
    cases = {
        one: one,
        one + 2 ** -8: one,                        # tie -> even (1.0)
        one + 3 * 2 ** -8: one + 2 ** -6,          # tie -> even (1 + 2 ulp)
        one + 2 ** -8 + 2 ** -20: one + 2 ** -7,   # above the tie -> up
        -(one + 2 ** -9): -one,                    # below the tie -> down
        3.140625: 3.140625,                        # exactly representable
        65504.0: 65536.0,                          # 0x477FE000: above half-way -> up
    }
    for x, want in cases.items():
        assert mlp.bf16(np.float32(x)) == want, x
    assert mlp.bf16_bits(np.float32(1.0)) == 0x3F80
    assert mlp.bf16_bits(np.float32(-2.0)) == 0xC000
    assert np.isnan(mlp.bf16(np.float32(np.nan)))
    b = mlp.bf16_bits(np.linspace(-3, 3, 101).astype(np.float32))
    np.testing.assert_array_equal(mlp.from_bf16_bits(b), mlp.bf16(np.linspace(-3, 3, 101)))


def test_gelu_tanh_form():
    # the tanh form, by hand with the library tanh at a few points
    a, b = math.sqrt(2 / math.pi), 0.044715
    for x in (-3.0, -1.0, -0.25, 0.5, 1.0, 2.5):
        want = 0.5 * x * (1 + math.tanh(a * (x + b * x ** 3)))
        assert float(mlp.gelu(x)) == pytest.approx(want, rel=1e-15, abs=1e-300)
    assert mlp.gelu(0.0) == 0.0
    assert float(mlp.gelu(12.0)) == pytest.approx(12.0, abs=1e-12)
    assert abs(float(mlp.gelu(-12.0))) < 1e-12
    # a close approximation of the exact GELU 0.5 x (1 + erf(x / sqrt 2)):
    # Phi(1) = 0.8413447460685429 (normal CDF) and |tanh form - exact| < 1e-3
    assert float(mlp.gelu(1.0)) == pytest.approx(0.8413447460685429, abs=1e-3)
    x = np.linspace(-6, 6, 241)
    assert np.max(np.abs(mlp.gelu(x) - mlp.gelu_erf(x))) < 1e-3
    # derivative: 1/2 at 0, central differences elsewhere
    assert float(mlp.gelu_grad(0.0)) == 0.5
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)


def test_width_one_network_through_library_tanh():
    # 1 -> 1 -> 1 -> 1 -> 1 with weights w and biases b, by hand with
    # math.tanh
    ws = [0.5, -1.25, 2.0, 0.75]
    bs = [0.125, 0.25, -0.5, 1.0]
    params = [(np.array([[w]]), np.array([b])) for w, b in zip(ws, bs)]
    a, c3 = math.sqrt(2 / math.pi), 0.044715
    x = 0.875
    h = x
    for l in range(3):
        z = ws[l] * h + bs[l]
        h = 0.5 * z * (1 + math.tanh(a * (z + c3 * z ** 3)))
    want = ws[3] * h + bs[3]
    y, _ = mlp.forward(params, np.array([[x]]))
    assert y[0, 0] == pytest.approx(want, rel=1e-14)


def _small_problem(seed, B=5, din=6, width=7, dout=4):
    params = W.mlp_params(din, width, dout, seed, bias_scale=0.3)
    rng = np.random.default_rng(seed + 100)
    X = rng.normal(size=(B, din))
    T = rng.normal(size=(B, dout))
    Om = rng.uniform(0, 1, size=(B, dout)) * (rng.uniform(size=(B, dout)) > 0.3)
    return params, X, T, Om


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backward_matches_central_differences(seed):
    params, X, T, Om = _small_problem(seed)

    def L(ps):
        Y, _ = mlp.forward(ps, X, bf16_weights=False)
        return mlp.loss(Y, T, Om)

    Y, cache = mlp.forward(params, X, bf16_weights=False)
    grads = mlp.backward(params, cache, Y, T, Om, bf16_weights=False)
    h = 1e-6
    for l, (Wl, bl) in enumerate(params):
        for arr, g in ((Wl, grads[l][0]), (bl, grads[l][1])):
            num = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + h
                lp = L(params)
                arr[idx] = old - h
                lm = L(params)
                arr[idx] = old
                num[idx] = (lp - lm) / (2 * h)
            np.testing.assert_allclose(g, num, rtol=1e-6, atol=1e-9)


def test_loss_definition_special_cases():
    Y = np.array([[1.0, 2.0], [3.0, 4.0]])
    T = np.array([[0.0, 2.0], [1.0, 1.0]])
    assert mlp.loss(Y, T, np.ones_like(Y)) == pytest.approx((1 + 0 + 4 + 9) / 2)
    assert mlp.loss(Y, T, np.zeros_like(Y)) == 0.0
    assert mlp.loss(Y, T, np.array([[1.0, 0], [0, 0.5]])) == pytest.approx((1 + 0.5 * 9) / 2)


def test_adamw_first_step_closed_forms():
    p = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.3, -4.0, 1e-3, 0.0])
    z = np.zeros(4)
    lr = 1e-2
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> p - lr g / (|g| + eps)
    p1, m1, v1 = mlp.adamw(p, g, z, z, 1, lr, eps=1e-8, wd=0.0)
    np.testing.assert_allclose(p1[:3], p[:3] - lr * np.sign(g[:3]), rtol=0, atol=1e-7)
    assert p1[3] == p[3]
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)
    # decoupled weight decay with a zero gradient: p (1 - lr wd)
    p2, _, _ = mlp.adamw(p, np.zeros(4), z, z, 1, lr, wd=0.1)
    np.testing.assert_allclose(p2, p * (1 - lr * 0.1))
    # constant gradient: m_hat = g and v_hat = g^2 at every step
    pt, m, v = p[:3].copy(), z[:3].copy(), z[:3].copy()
    for t in range(1, 6):
        pt, m, v = mlp.adamw(pt, g[:3], m, v, t, lr, eps=0.0)
    np.testing.assert_allclose(pt, p[:3] - 5 * lr * np.sign(g[:3]), rtol=1e-12)


def test_features_layout():
    inst = {"start": [0.1, -0.2, 0.3], "goal": [0.4, 0.5, -0.6], "side_x": 0.09, "side_y": 0.12}
    din, width, dout = mlp.dims(4, 80)
    assert (din, width, dout) == (64, 256, 256)
    x = mlp.features(inst, (3, 11), 4, din)
    np.testing.assert_allclose(x[:8], [0.1, -0.2, 0.3, 0.4, 0.5, -0.6, 0.9, 1.2])
    onehot = x[12:64].reshape(4, 13)
    assert onehot.sum() == 4 and onehot[0, 3] == 1 and onehot[1, 11] == 1
    assert onehot[2, 12] == 1 and onehot[3, 12] == 1 and x[11] == 0
    assert mlp.dims(6, 180) == (128, 256, 544)
    # goal in the start frame: start rotated by +90 degrees, goal one unit
    # ahead along the world y axis -> (x', y') = (3, 0), dtheta = 0.25
    x = mlp.features({"start": [1.0, 2.0, np.pi / 2], "goal": [1.0, 3.0, np.pi / 2 + 0.25], "side_x": 0.1,
                      "side_y": 0.1}, (0,), 4, din)
    np.testing.assert_allclose(x[8:11], [3.0, 0.0, 0.25], atol=1e-12)
    # invariance: a planar rigid motion of the world frame leaves 8..10 fixed
    a, t = 0.7, np.array([0.3, -0.1])
    R = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    s0, g0 = np.array([0.1, -0.2, 0.3]), np.array([0.4, 0.5, -0.6])
    moved = {"start": np.r_[R @ s0[:2] + t, s0[2] + a], "goal": np.r_[R @ g0[:2] + t, g0[2] + a],
             "side_x": 0.09, "side_y": 0.12}
    np.testing.assert_allclose(mlp.features(moved, (3, 11), 4, din)[8:11], mlp.features(inst, (3, 11), 4, din)[8:11],
                               atol=1e-12)


def test_bimanual_features_layout():
    # mode m = 169 g + 13 h_L + h_R: three hand-decoded cases, a blank slot,
    # the instance part, and a bijection of the 507 modes onto 3 x 13 x 13
    inst = {"start": [0.0, 0.05, 0.0], "goal": [0.1, 0.05, 1.7], "side_x": 0.2, "side_y": 0.1, "mass": 1.5}
    din, width, dout = mlp.bim_dims(6, 90)
    assert (din, width, dout) == (192, 256, 1088)
    x = mlp.bim_features(inst, (0, 506, 200), 6, din)
    np.testing.assert_allclose(x[:12], [0.0, 0.05, 0.0, 0.1, 0.05, 1.7, 2.0, 1.0, 0.3, 0.0, 1.7, 1.5], atol=1e-12)
    slots = x[12:12 + 30 * 6].reshape(6, 30)
    assert list(np.nonzero(slots[0])[0]) == [0, 3, 16]            # g 0, h_L 0, h_R 0
    assert list(np.nonzero(slots[1])[0]) == [2, 15, 28]           # 506 = 2*169 + 12*13 + 12
    assert list(np.nonzero(slots[2])[0]) == [1, 5, 21]            # 200 = 169 + 2*13 + 5
    for i in range(3, 6):
        assert list(np.nonzero(slots[i])[0]) == [29]
    assert np.all(x[12 + 30 * 6:] == 0)
    seen = set()
    for m in range(507):
        nz = tuple(np.nonzero(mlp.bim_features(inst, (m,), 1, din)[12:42])[0])
        assert len(nz) == 3 and nz[0] < 3 and 3 <= nz[1] < 16 and 16 <= nz[2] < 29
        seen.add(nz)
    assert len(seen) == 507


def test_bimanual_targets_and_warm_start_scale_the_forces():
    n_max, N, mass = 30, 15, 2.0
    _, _, dout = mlp.bim_dims(2, n_max)
    rng = np.random.default_rng(3)
    ctrl = rng.normal(size=(12, n_max))
    T, Om = mlp.bim_targets(0.5, 0.0, 0, ctrl, N, n_max, dout, mass)
    assert T[0] == pytest.approx(np.log(0.5)) and Om[0] == 1.0
    for c in range(12):
        want = ctrl[c, :N] / (mass * 9.81) if c in (3, 4, 6, 7, 9, 10) else ctrl[c, :N]
        np.testing.assert_allclose(T[1 + c * n_max:1 + c * n_max + N], want, rtol=1e-15)
        assert np.all(T[1 + c * n_max + N:1 + (c + 1) * n_max] == 0)
        np.testing.assert_allclose(Om[1 + c * n_max:1 + c * n_max + N], 1.0 / (12 * N))
    # not converged: only the merit entry carries weight
    T2, Om2 = mlp.bim_targets(0.5, 1e-3, 1, ctrl, N, n_max, dout, mass)
    assert Om2[0] == 1.0 and np.all(Om2[1:] == 0)
    assert T2[0] == pytest.approx(np.log(0.5 + 100.0 * (1e-3 - 1e-5)))
    # the warm start undoes the force scaling: targets in, controls out
    inst = {"start": [0.0, 0.1, 0.0], "goal": [0.2, 0.1, 1.6], "mass": mass}
    w = mlp.bim_warm(inst, N, n_max, T)
    u = w[5 * (n_max + 1):].reshape(12, n_max)
    np.testing.assert_allclose(u[:, :N], ctrl[:, :N], rtol=1e-12)
    xs = w[:5 * (n_max + 1)].reshape(5, n_max + 1)
    np.testing.assert_allclose(xs[2, :N + 1], np.linspace(0.0, 1.6, N + 1), atol=1e-12)
    assert np.all(xs[3:] == 0) and np.all(xs[:, N + 1:] == 0)
