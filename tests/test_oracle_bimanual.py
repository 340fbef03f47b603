"""Pins of the bimanual oracle (oracle/bimanual.c) to facts outside it:
central differences of every row, a dense solve of the assembled Gauss-Newton
system, closed forms of two special cases (a box at rest, a box pushed
sideways while sliding), the torque balance about the pivot corner, the KKT
conditions on the dense Jacobian, and the left/right symmetry of the hands.
"""
import numpy as np
import pytest

import oracle
import workloads as W

N1 = 15
G = oracle.GRAVITY


def _rand_local(rng, inst):
    ax, az = 0.5 * inst["side_x"], 0.5 * inst["side_y"]
    xk = np.array([rng.normal(0, 0.1), az + rng.normal(0, 0.05), rng.uniform(-0.3, 1.8),
                   rng.uniform(-az, az), rng.uniform(-ax, ax)])
    uk = rng.normal(0, 1.0, 12)
    uk[3:5] *= 5.0
    uk[6:8] *= 5.0
    uk[9:11] *= 5.0
    uk[11] = rng.normal(0, 0.05)
    xk1 = xk + rng.normal(0, 0.02, 5)
    return xk, uk, xk1


@pytest.mark.parametrize("seed", range(3))
def test_row_jacobians_match_central_differences(seed):
    rng = np.random.default_rng(seed)
    inst = W.bimanual_instance(seed)
    modes = rng.choice(507, 60, replace=False)
    h = 1e-6
    for m in modes:
        xk, uk, xk1 = _rand_local(rng, inst)
        mL, mR = bool(rng.integers(0, 2)), bool(rng.integers(0, 2))
        c, mask, ineq, scale, J = oracle.bim_interval_rows(inst, m, mL, mR, xk, uk, xk1)
        v = np.concatenate([xk, uk, xk1])
        num = np.zeros_like(J)
        for j in range(22):
            vp, vm = v.copy(), v.copy()
            vp[j] += h
            vm[j] -= h
            cp = oracle.bim_interval_rows(inst, m, mL, mR, vp[:5], vp[5:17], vp[17:])[0]
            cm = oracle.bim_interval_rows(inst, m, mL, mR, vm[:5], vm[5:17], vm[17:])[0]
            num[:, j] = (cp - cm) / (2 * h)
        np.testing.assert_allclose(J, num, rtol=1e-6, atol=1e-7, err_msg=f"mode {m}")
        assert np.all(c[~mask] == 0) and np.all(J[~mask] == 0)


def test_mode_layout():
    # ground stick and both hands none: three velocity rows, no hand forces
    inst = W.bimanual_instance(0)
    c, mask, ineq, scale, J = oracle.bim_interval_rows(inst, W.bimanual_mode(0, 0, 0), False, False,
                                                       np.zeros(5), np.zeros(12), np.zeros(5))
    assert mask[:16].all() and mask[16:19].all() and not mask[19:24].any() and not mask[27:].any()
    assert list(np.flatnonzero(ineq)) == list(range(11, 16)) + list(range(19, 24)) + list(range(27, 32))
    # pivot: no CoP bounds; slide: one friction row; a sliding hand has no cone
    _, mask_p, *_ = oracle.bim_interval_rows(inst, W.bimanual_mode(2, 1, 0), False, False,
                                             np.zeros(5), np.ones(12), np.zeros(5))
    assert not mask_p[14] and not mask_p[15] and mask_p[11] and mask_p[12]
    _, mask_s, *_ = oracle.bim_interval_rows(inst, W.bimanual_mode(1, 2, 0), True, False,
                                             np.zeros(5), np.ones(12), np.zeros(5))
    assert mask_s[11] and not mask_s[12] and not mask_s[3]
    assert mask_s[16] and not mask_s[17] and mask_s[19] and not mask_s[20]


def _dense_step(inst, modes, N, tr, lam, beta, rho):
    """(H + rho I) dz = -g assembled from the dense Jacobian, the cost
    Hessian and the active rows (the definition of the step)."""
    jac = oracle.bim_dense_jacobian(inst, modes, N, tr)
    c, mask, scale, ci = oracle.bim_rows(inst, modes, N, tr)
    call = np.concatenate([ci, c.ravel()])
    ineq_row = np.zeros(32, bool)
    ineq_row[11:16] = ineq_row[19:24] = ineq_row[27:] = True
    ineq = np.concatenate([np.zeros(3, bool), np.tile(ineq_row, N)])
    present = np.concatenate([np.ones(3, bool), mask.ravel()])
    t = lam + beta * call
    active = present & (~ineq | (t > 0))
    y = np.where(active, t, 0.0)
    nz = 17 * N + 5
    mg = inst["mass"] * G
    R = np.array([0.1, 0.1, 0.1, 0.1 / mg**2, 0.1 / mg**2, 0.1, 0.1 / mg**2, 0.1 / mg**2, 0.1, 0.1 / mg**2,
                  0.1 / mg**2, 0.1])
    Hc = np.zeros(nz)
    gc = np.zeros(nz)
    for k in range(N):
        for j in range(12):
            u = tr[5 * (N + 1) + j * N + k]
            Hc[17 * k + 5 + j] = 2 * R[j]
            gc[17 * k + 5 + j] = 2 * R[j] * u
    for i in range(3):
        Hc[17 * N + i] = 2 * 10.0
        gc[17 * N + i] = 2 * 10.0 * (tr[i * (N + 1) + N] - inst["goal"][i])
    A = jac[active]
    H = np.diag(Hc) + beta * A.T @ A + rho * np.eye(nz)
    g = gc + jac.T @ y
    return np.linalg.solve(H, -g), g


def _cost_gradient(inst, N, tr):
    mg = inst["mass"] * G
    w = inst["w_control"]
    R = np.array([w, w, w, w / mg**2, w / mg**2, w, w / mg**2, w / mg**2, w, w / mg**2, w / mg**2, w])
    g = np.zeros(17 * N + 5)
    for k in range(N):
        for j in range(12):
            g[17 * k + 5 + j] = 2 * R[j] * tr[5 * (N + 1) + j * N + k]
    for i in range(3):
        g[17 * N + i] = 2 * inst["w_terminal"] * (tr[i * (N + 1) + N] - inst["goal"][i])
    return g


@pytest.mark.parametrize("modes", [[358], [W.bimanual_mode(0, 1, 7), W.bimanual_mode(2, 4, 7),
                                           W.bimanual_mode(1, 0, 10)]])
def test_backward_sweep_equals_dense_solve(modes):
    inst = W.bimanual_instance(1)
    N = 15 * len(modes)
    rng = np.random.default_rng(3)
    tr = oracle.bim_cold_start(inst, N) + rng.normal(0, 0.01, 5 * (N + 1) + 12 * N)
    lam = rng.normal(0, 0.1, 3 + 32 * N)
    for beta, rho in [(100.0, 1e-4), (1e4, 1e-2)]:
        ok, dz, grad = oracle.bim_gn_step(inst, modes, N, tr, lam, beta, rho)
        assert ok == 0
        want, g = _dense_step(inst, modes, N, tr, lam, beta, rho)
        np.testing.assert_allclose(grad, g, rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(dz, want, rtol=1e-6, atol=1e-9 * np.max(np.abs(want)))


def test_box_at_rest_closed_form():
    # both hands none, ground stick, goal = start: the box cannot move; the
    # ground carries the weight at the centre (lam_n = mg, lam_t = 0, p_c =
    # 0) and J* = N w_control (forces are weighted by w_control / (mg)^2)
    inst = W.bimanual_instance(2)
    inst["goal"] = list(inst["start"])
    r, tr, lam = oracle.bim_solve(inst, [W.bimanual_mode(0, 0, 0)], N1)
    assert r["status"] == oracle.CONVERGED
    mg = inst["mass"] * G
    U = tr[5 * (N1 + 1):].reshape(12, N1)
    np.testing.assert_allclose(U[9], mg, rtol=1e-6)
    np.testing.assert_allclose(U[[0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 11]], 0.0, atol=1e-6)
    X = tr[: 5 * (N1 + 1)].reshape(5, N1 + 1)
    np.testing.assert_allclose(X[:3], np.repeat(np.array(inst["start"])[:, None], N1 + 1, axis=1), atol=1e-7)
    # (up to the first-order effect of the stop test's allowed infeasibility)
    assert r["cost"] == pytest.approx(N1 * inst["w_control"], rel=1e-5)


def test_sliding_push_closed_form():
    # hand L sticks on face 0 (pushes +x), hand R none, the ground slides:
    # force balance gives f_n = mu_g (mg - f_t), lam_n = mg - f_t, lam_t =
    # -mu_g lam_n.  Minimising the force cost along that line drives f_t up
    # to the hand's friction cone (f_t = mu_h f_n): with mu_g = mu_h = 1/2,
    # f_n = 0.4 mg, f_t = 0.2 mg, lam_n = 0.8 mg, lam_t = -0.4 mg.
    inst = W.bimanual_instance(3)
    ax, az = 0.5 * inst["side_x"], 0.5 * inst["side_y"]
    inst["side_y"] = min(inst["side_y"], 2.5 * ax)      # the CoP stays on the face
    az = 0.5 * inst["side_y"]
    inst["start"] = [0.0, az, 0.0]
    inst["goal"] = [0.05, az, 0.0]
    r, tr, lam = oracle.bim_solve(inst, [W.bimanual_mode(1, 1, 0)], N1)
    assert r["status"] == oracle.CONVERGED
    mg = inst["mass"] * G
    U = tr[5 * (N1 + 1):].reshape(12, N1)
    assert np.all(U[0] > 1e-3)                            # the box moves along +x
    np.testing.assert_allclose(U[3] / mg, 0.4, atol=1e-4)  # f_n
    np.testing.assert_allclose(U[4] / mg, 0.2, atol=1e-4)  # f_t
    np.testing.assert_allclose(U[9] / mg, 0.8, atol=1e-4)  # lam_n
    np.testing.assert_allclose(U[10] / mg, -0.4, atol=1e-4)  # lam_t
    # the identity of the two force balances holds exactly
    np.testing.assert_allclose(U[3] + 0.5 * U[4], 0.5 * mg, rtol=1e-6)


@pytest.mark.parametrize("mode", [358, W.bimanual_mode(2, 2, 7), W.bimanual_mode(2, 1, 10)])
def test_pivot_torque_balance_about_the_corner(mode):
    # with the ground force at the pivot corner, gravity and the hands have no
    # net moment about the corner, up to the moment of the ground's tangential
    # force from the corner's height above the ground, -(z + r_cz) lam_t (zero
    # while the corner touches; explicit Euler lets it drift by O(dt^2))
    inst = W.bimanual_instance(0)
    r, tr, lam = oracle.bim_solve(inst, [mode], N1)
    assert r["status"] == oracle.CONVERGED
    ax, az = 0.5 * inst["side_x"], 0.5 * inst["side_y"]
    mg = inst["mass"] * G
    X = tr[: 5 * (N1 + 1)].reshape(5, N1 + 1)
    U = tr[5 * (N1 + 1):].reshape(12, N1)
    nrm = {0: (1, 0), 1: (0, 1), 2: (-1, 0), 3: (0, -1)}
    hL, hR = (mode // 13) % 13, mode % 13
    for k in range(N1):
        th, z = X[2, k], X[1, k]
        c, s = np.cos(th), np.sin(th)
        Rm = np.array([[c, -s], [s, c]])
        rc = Rm @ np.array([-ax, -az])
        tau = -(rc[0] * (-mg))                              # gravity at the centre, about the corner
        for h, (ifn, ift, isl) in ((hL, (3, 4, 3)), (hR, (6, 7, 4))):
            if h == 0:
                continue
            f = (h - 1) // 3
            n = np.array(nrm[f], float)
            t = np.array([-n[1], n[0]])
            a = ax if f % 2 == 0 else az
            p = Rm @ (-a * n + X[isl, k] * t)
            F = Rm @ (U[ifn, k] * n + U[ift, k] * t)
            d = p - rc
            tau += d[0] * F[1] - d[1] * F[0]
        # each of the three balance rows may be off by eps_primal of its scale
        assert abs(tau + (z + rc[1]) * U[10, k]) <= 1e-5 * mg * max(ax, az)


def test_kkt_at_converged_points():
    inst = W.bimanual_instance(4)
    for modes in ([358], [W.bimanual_mode(0, 1, 7), W.bimanual_mode(2, 1, 7)]):
        N = 15 * len(modes)
        r, tr, lam = oracle.bim_solve(inst, modes, N)
        assert r["status"] == oracle.CONVERGED
        jac = oracle.bim_dense_jacobian(inst, modes, N, tr)
        c, mask, scale, ci = oracle.bim_rows(inst, modes, N, tr)
        g = _cost_gradient(inst, N, tr)
        stat = g + jac.T @ lam
        # the stop test's stationarity tolerance, relative to max(1, |J|)
        assert np.max(np.abs(stat)) <= 1e-4 * max(1.0, r["beta"] / 1e3) * max(1.0, r["cost"])
        ineq = np.zeros(32, bool)
        ineq[11:16] = ineq[19:24] = ineq[27:] = True
        lam_rows = lam[3:].reshape(N, 32)
        assert np.all(lam_rows[:, ineq] >= -1e-12)
        cr = c[:, ineq] * mask[:, ineq]
        assert np.max(cr) <= 1e-6
        assert np.max(np.abs(lam_rows[:, ineq] * cr)) <= 1e-6
        # the stop test holds every row within half eps_feas in physical units
        phys = np.where(np.broadcast_to(ineq, c.shape), np.maximum(c, 0), np.abs(c)) / scale * mask
        assert np.max(phys) <= 0.5e-5
        assert r["viol"] <= 0.5e-5


def test_hands_are_interchangeable():
    # swapping the two hands' modes leaves the problem the same
    inst = W.bimanual_instance(5)
    for hL, hR in ((1, 4), (2, 8), (0, 7)):
        a, *_ = oracle.bim_solve(inst, [W.bimanual_mode(2, hL, hR)], N1)
        b, *_ = oracle.bim_solve(inst, [W.bimanual_mode(2, hR, hL)], N1)
        assert a["status"] == b["status"]
        assert a["cost"] == pytest.approx(b["cost"], rel=1e-6)


def test_vhat_in_physical_units():
    """v_hat (Eq. inexact_mode_value) is scored in physical units, separately
    from the internal scaling (Sec. III-C "Stopping and scoring").  A box
    resting on the ground with its normal force off by delta newtons has
    v_hat = delta [N], not delta / (m g); each scaled row maps back to its
    physical quantity through c / scale."""
    inst = W.bimanual_instance(6)
    inst["mass"] = 2.0
    mg = 2.0 * G
    N = 15
    delta = 0.3
    tr = np.zeros(oracle.bim_traj_len(N))
    X = tr[: 5 * (N + 1)].reshape(5, N + 1)
    U = tr[5 * (N + 1):].reshape(12, N)
    X[:3] = np.array(inst["start"])[:, None]
    U[9] = mg + delta  # lam_n; everything else at rest
    opts = oracle.default_opts(max_iters=0)
    r, _, _ = oracle.bim_solve(inst, [W.bimanual_mode(0, 0, 0)], N, warm=tr, opts=opts)
    assert r["viol"] == pytest.approx(delta, rel=1e-12)
    # row by row, with random values: physical = c / scale
    rng = np.random.default_rng(7)
    ax, az = 0.5 * inst["side_x"], 0.5 * inst["side_y"]
    mu = inst["ground_mu"]
    for _ in range(20):
        xk = rng.normal(size=5) * 0.1
        uk = rng.normal(size=12) * mg
        xk1 = xk + rng.normal(size=5) * 0.01
        for g in range(3):
            m = W.bimanual_mode(g, 1, 4)  # left stick on face 0, right stick on face 1
            c, mask, ineq, scale, J = oracle.bim_interval_rows(inst, m, False, False, xk, uk, xk1)
            phys = c / scale
            ln, lt, pc, xd = uk[9], uk[10], uk[11], uk[0]
            assert phys[13] == pytest.approx(-ln, rel=1e-12)                    # N
            assert phys[6] == pytest.approx(uk[9] + (np.sin(xk[2]) * uk[3] + np.cos(xk[2]) * uk[4])
                                            + (np.sin(xk[2]) * -uk[7] + np.cos(xk[2]) * uk[6]) - mg,
                                            rel=1e-10, abs=1e-9)                  # F_z - m g [N]
            assert phys[21] == pytest.approx(-uk[3], rel=1e-12)                  # -f_n of the left hand [N]
            if g == 1:
                assert phys[10] == pytest.approx(abs(lt) - mu * abs(ln), rel=1e-10, abs=1e-9)  # cone edge [N]
                assert phys[11] == pytest.approx(lt * xd, rel=1e-12)             # friction power [W]
            else:
                assert phys[11] == pytest.approx(lt - mu * ln, rel=1e-10, abs=1e-9)  # cone [N]
            tau = pc * ln + xk[1] * lt - ax * uk[4] - xk[3] * uk[3] - az * uk[7] - xk[4] * uk[6]
            assert phys[7] == pytest.approx(tau, rel=1e-10, abs=1e-9)            # torque [N m]
