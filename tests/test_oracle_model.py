"""Pins of the oracle's model layer against closed forms and finite
differences (no GPU).  Paper: Sec. III-A (problem), Sec. III-C (shared
masked representation)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

INST = W.push_l2_instance(3)


def test_straight_push_twist_closed_form():
    # ellipsoidal limit surface: twist = kappa * (F, m_z / c^2); a push along the
    # face normal through the centre (s = 0, f_t = 0) translates along n_f only
    for face, n in enumerate([(1, 0), (0, 1), (-1, 0), (0, -1)]):
        th = 0.3
        f, _, _ = oracle.dynamics(INST, face, [0.1, -0.2, th, 0.0], [0.05, 0.0, 0.0])
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        np.testing.assert_allclose(f[:2], R @ (0.05 * np.array(n, float)), rtol=0, atol=1e-15)
        assert abs(f[2]) < 1e-15 and f[3] == 0.0


def test_offset_push_rotation_rate():
    # offset push (s != 0, f_t = 0): m_z = -s f_n, theta_dot = -s f_n / c^2
    c2 = INST["c_ls"] ** 2
    for face in range(4):
        for s in (-0.03, 0.01, 0.04):
            f, _, _ = oracle.dynamics(INST, face, [0.0, 0.0, 1.1, s], [0.07, 0.0, 0.0])
            assert f[2] == pytest.approx(-s * 0.07 / c2, rel=1e-14)


def test_tangential_force_moment_arm():
    # f_t acts at lever arm a_f (half-depth): m_z = -a f_t  (s = 0)
    a0 = INST["side_x"] / 2
    f, _, _ = oracle.dynamics(INST, 0, [0, 0, 0, 0.0], [0.0, 0.02, 0.0])
    assert f[2] == pytest.approx(-a0 * 0.02 / INST["c_ls"] ** 2, rel=1e-14)
    # body-frame force on face 0 with f_t: along t_0 = (0, 1)
    assert f[0] == pytest.approx(0.0, abs=1e-16) and f[1] == pytest.approx(0.02, rel=1e-14)


@pytest.mark.parametrize("face", range(4))
def test_jacobians_match_central_differences(face):
    rng = np.random.default_rng(face)
    for _ in range(5):
        x = rng.uniform(-1, 1, 4) * [0.3, 0.3, 3.0, 0.04]
        u = rng.uniform(-1, 1, 3) * [0.1, 0.05, 0.02]
        _, Fx, Fu = oracle.dynamics(INST, face, x, u)
        h = 1e-6
        for j in range(4):
            e = np.zeros(4); e[j] = h
            fd = (oracle.dynamics(INST, face, x + e, u)[0] - oracle.dynamics(INST, face, x - e, u)[0]) / (2 * h)
            np.testing.assert_allclose(Fx[:, j], fd, rtol=1e-6, atol=1e-9)
        for j in range(3):
            e = np.zeros(3); e[j] = h
            fd = (oracle.dynamics(INST, face, x, u + e)[0] - oracle.dynamics(INST, face, x, u - e)[0]) / (2 * h)
            np.testing.assert_allclose(Fu[:, j], fd, rtol=1e-6, atol=1e-9)


def test_segment_allocation_uniform():
    # N intervals split among `len` segments deterministically (Sec. III-C)
    assert [oracle.segment_of(k, 2, 16) for k in range(16)] == [0] * 8 + [1] * 8
    assert [oracle.segment_of(k, 3, 10) for k in range(10)] == [0, 0, 0, 0, 1, 1, 1, 2, 2, 2]


def _mode(face, kind):
    return 3 * face + kind


def test_row_masks_and_values_per_mode():
    N = 16
    mu = INST["mu"]
    sc = 1 / math.sqrt(1 + mu * mu)
    rng = np.random.default_rng(0)
    tr = rng.normal(size=7 * N + 4) * 0.05
    fn, ft, sd = tr[4 * 17 + 0], tr[4 * 17 + N], tr[4 * 17 + 2 * N]
    s0 = tr[3 * 17 + 0]
    for face in range(4):
        ell = (INST["side_y"] if face % 2 == 0 else INST["side_x"]) / 2
        for kind in range(3):
            m = _mode(face, kind)
            c, mask, scale, ci = oracle.rows(INST, [m, m], N, tr)
            # interval 0 rows
            row, mk = c[0], mask[0]
            assert list(mk[:4]) == [1, 1, 1, 1]
            if kind == 0:
                assert row[4] == pytest.approx(sd)
                assert mk[5] and mk[6] and not mk[7]
                assert row[5] == pytest.approx(sc * (ft - mu * fn))
                assert row[6] == pytest.approx(sc * (-ft - mu * fn))
            else:
                sg = -1 if kind == 1 else 1
                assert row[4] == pytest.approx(sc * (ft + sg * mu * fn))
                assert not mk[5] and not mk[6] and mk[7]
                assert row[7] == pytest.approx(sg * sd)
                assert row[5] == 0 and row[6] == 0
            assert row[8] == pytest.approx(-fn)
            assert row[9] == pytest.approx(s0 - ell) and row[10] == pytest.approx(-s0 - ell)


def test_s_row_masked_only_at_face_changes():
    N = 16
    tr = oracle.cold_start(INST, N)
    _, mask, _, _ = oracle.rows(INST, [0, 1], N, tr)     # same face: continuous offset
    assert mask[:, 3].all()
    _, mask, _, _ = oracle.rows(INST, [0, 3], N, tr)     # face change at interval 8
    assert not mask[7, 3] and mask[np.arange(16) != 7, 3].all()


def test_cold_start_layout():
    inst = W.push_l4_instance(2)
    N = 80
    tr = oracle.cold_start(inst, N)
    X = tr[: 4 * (N + 1)].reshape(4, N + 1)
    np.testing.assert_allclose(X[:3, 0], inst["start"])
    np.testing.assert_allclose(X[:3, -1], inst["goal"])
    assert np.all(X[3] == 0) and np.all(tr[4 * (N + 1):] == 0)
    np.testing.assert_allclose(np.diff(X[0]), (inst["goal"][0] - inst["start"][0]) / N)
