"""Pins of the free-motion pushing mode in the oracle (Sec. III-A: a mode is
which face the pusher contacts, or free motion, and a contact changes faces
only through a free-motion segment).  Reading: during free motion the
pusher is off the slider (the mode equality f_n = 0 is the only force row;
f_t acts on nothing and the effort cost sets it to zero), the slider rests,
the contact offset is unconstrained (its dynamics row and the face bounds
are off) and may jump at either end.
Checked: the rows and masks of a free interval, their Jacobian against
central differences of the row values, two closed forms (a free order
cannot move the slider; free motion followed by a straight sticking push
equals the straight push over the contact intervals alone), the backward
sweep against the dense solve, and KKT at converged points."""
import numpy as np
import pytest

import oracle
import workloads as W
from _helpers import cost_grad_hess, dense_step, to_component, to_interleaved

FREE = oracle.MODE_FREE
TIGHT = dict(eps_dual=1e-9, eps_primal=1e-11, eps_comp=1e-11, max_iters=1000, beta_max=1e6)
INST = W.push_l2_straight(0.1)


def test_free_rows_and_masks():
    N = 16
    rng = np.random.default_rng(1)
    tr = oracle.cold_start(INST, N) + rng.normal(size=7 * N + 4) * 0.05
    X = tr[: 4 * (N + 1)].reshape(4, N + 1)
    U = tr[4 * (N + 1):].reshape(3, N)
    c, mask, scale, _ = oracle.rows(INST, [FREE, 0], N, tr)
    for k in range(8):                      # free intervals
        assert list(mask[k]) == [1, 1, 1, 0, 1, 0, 0, 0, 0, 0, 0]
        # the slider rests: physical defect of the pose rows is x_{k+1} - x_k
        np.testing.assert_allclose(c[k, :3] / scale[k, :3], X[:3, k + 1] - X[:3, k], rtol=1e-12)
        assert c[k, 4] == pytest.approx(U[0, k])
        assert c[k, 3] == 0 and np.all(c[k, 5:] == 0)
    # contact intervals keep the sticking rows; the offset is continuous on
    # the face after the free segment
    assert mask[8:, 3].all() and mask[8:, 9].all() and mask[8:, 5].all()
    # contact -> free and free -> other face: offset rows open at the boundary
    _, m2, _, _ = oracle.rows(INST, [0, FREE, 3], 24, oracle.cold_start(INST, 24))
    assert not m2[7, 3] and not m2[8:16, 3].any() and m2[16:, 3].all()


def test_free_jacobian_central_differences():
    N = 12
    rng = np.random.default_rng(2)
    modes = [FREE, 3, FREE]
    tr = oracle.cold_start(INST, N) + rng.normal(size=7 * N + 4) * 0.03
    z = to_interleaved(tr, N)
    J = oracle.dense_jacobian(INST, modes, N, tr)

    def vals(zz):
        c, mask, _, ci = oracle.rows(INST, modes, N, to_component(zz, N))
        return np.concatenate([ci, (c * mask).ravel()])

    h = 1e-6
    for j in range(len(z)):
        e = np.zeros(len(z)); e[j] = h
        fd = (vals(z + e) - vals(z - e)) / (2 * h)
        np.testing.assert_allclose(J[:, j], fd, rtol=1e-6, atol=1e-8)


def test_free_order_cannot_move_the_slider():
    inst = W.push_l2_instance(3)
    tr, lam, res = oracle.solve(inst, [FREE, FREE], opts=oracle.default_opts(**TIGHT))
    assert res["status"] == oracle.CONVERGED
    N = 16
    X = tr[: 4 * (N + 1)].reshape(4, N + 1)
    np.testing.assert_allclose(X[:3], np.array(inst["start"])[:, None] * np.ones((1, N + 1)), atol=1e-9)
    np.testing.assert_allclose(tr[4 * (N + 1):], 0.0, atol=1e-9)
    d2 = np.sum((np.array(inst["goal"]) - np.array(inst["start"])) ** 2)
    assert res["cost"] == pytest.approx(inst["w_terminal"] * d2, rel=1e-9)


@pytest.mark.parametrize("d", [0.05, 0.1])
def test_free_then_straight_push_closed_form(d):
    # goal (d, 0, 0): free motion on the first K intervals, face 0 sticking on
    # the last K.  Only the contact intervals move the slider, so the straight
    # push closed form holds with N replaced by K: J* = W R d^2 / (R + W K dt^2)
    inst = W.push_l2_straight(d)
    K, Wt, R, dt = inst["knots_per_segment"], inst["w_terminal"], inst["w_control"], inst["dt"]
    tr, lam, res = oracle.solve(inst, [FREE, 0], opts=oracle.default_opts(**TIGHT))
    assert res["status"] == oracle.CONVERGED
    assert res["cost"] == pytest.approx(Wt * R * d * d / (R + Wt * K * dt * dt), rel=1e-7)
    N = 2 * K
    U = tr[4 * (N + 1):].reshape(3, N)
    np.testing.assert_allclose(U[:, :K], 0.0, atol=1e-9)
    np.testing.assert_allclose(U[0, K:], Wt * dt * d / (Wt * K * dt * dt + R), rtol=1e-6)


@pytest.mark.parametrize("modes", [[FREE, 0], [0, FREE], [FREE, 9]])
@pytest.mark.parametrize("curvature", [False, True])
def test_sweep_equals_dense_solve_with_free_segments(modes, curvature):
    inst = W.push_l2_instance(5)
    N = 6 if curvature else 16
    rng = np.random.default_rng(sum(modes))
    tr = oracle.cold_start(inst, N) + rng.normal(size=7 * N + 4) * 0.02
    lam = rng.normal(size=3 + 11 * N) * 0.1
    for beta, rho in ([(100.0, 1.0)] if curvature else [(100.0, 1e-4), (1e4, 1e-2)]):
        while True:
            # with the curvature the model at a random point may be
            # indefinite: raise the damping until every local S_k factors
            try:
                dz, g = oracle.gn_step(inst, modes, N, tr, lam, beta, rho, curvature)
                break
            except RuntimeError:
                assert curvature and rho < 1e6
                rho *= 10.0
        dz_ref, g_ref = dense_step(inst, modes, N, tr, lam, beta, rho, curvature)
        np.testing.assert_allclose(g, g_ref, rtol=1e-12, atol=1e-12)
        tol = 1e-6 if curvature else 1e-9
        assert np.max(np.abs(dz - dz_ref)) <= tol * max(1.0, np.max(np.abs(dz_ref)))


@pytest.mark.parametrize("seed", [0, 2])
def test_kkt_with_free_segments(seed):
    inst = W.push_l2_instance(seed)
    N = 16
    seen = 0
    for modes in ([FREE, 0], [FREE, 3], [0, FREE], [FREE, 6]):
        tr, lam, res = oracle.solve(inst, modes, opts=oracle.default_opts(**TIGHT))
        if res["status"] != oracle.CONVERGED:
            continue
        seen += 1
        c, mask, scale, ci = oracle.rows(inst, modes, N, tr)
        cc = np.concatenate([ci, c.ravel()])
        mk = np.concatenate([np.ones(3, bool), mask.ravel().astype(bool)])
        ineq = np.zeros_like(mk); ineq[3:] = np.tile(np.arange(11) >= 5, N)
        assert np.max(np.abs(cc[mk & ~ineq])) <= 1e-9
        assert np.max(np.maximum(cc[mk & ineq], 0)) <= 1e-9
        assert np.all(lam[ineq] >= 0) and np.all(lam[~mk] == 0)
        gJ, _ = cost_grad_hess(inst, N, to_interleaved(tr, N))
        r = gJ + oracle.dense_jacobian(inst, modes, N, tr).T @ lam
        assert np.max(np.abs(r)) <= 1e-7
        # no contact force during free motion
        seg = np.array([oracle.segment_of(k, 2, N) for k in range(N)])
        free_k = np.array([modes[s] == FREE for s in seg])
        U = tr[4 * (N + 1):].reshape(3, N)
        assert np.max(np.abs(U[:2, free_k])) <= 1e-8
    assert seen >= 2


def test_scipy_slsqp_finds_no_better_point_with_free_motion():
    # tiny orders with free motion (two segments of K = 3): SciPy's SLSQP on
    # the same NLP (Eq. mode_nlp with the free-motion rows), started next to
    # the oracle's solution, finds no lower cost
    so = pytest.importorskip("scipy.optimize")
    inst = W.push_l2_instance(9)
    inst["knots_per_segment"] = 3
    N = 6
    for modes in ([FREE, 0], [FREE, 3], [6, FREE]):
        tr, lam, res = oracle.solve(inst, modes, opts=oracle.default_opts(**TIGHT))
        assert res["status"] == oracle.CONVERGED

        def fun(z):
            return inst["w_terminal"] * np.sum((z[7 * N: 7 * N + 3] - inst["goal"]) ** 2) + inst["w_control"] * sum(
                np.sum(z[7 * k + 4: 7 * k + 7] ** 2) for k in range(N))

        def rows(z):
            c, mask, _, ci = oracle.rows(inst, modes, N, to_component(z, N))
            return np.concatenate([ci, c.ravel()]), mask.ravel().astype(bool)

        def eq(z):
            cc, mk = rows(z)
            return cc[np.concatenate([np.ones(3, bool), np.tile(np.arange(11) < 5, N) & mk])]

        def ineq(z):
            cc, mk = rows(z)
            return -cc[np.concatenate([np.zeros(3, bool), np.tile(np.arange(11) >= 5, N) & mk])]

        cons = [{"type": "eq", "fun": eq}, {"type": "ineq", "fun": ineq}]
        rng = np.random.default_rng(sum(modes))
        zo = to_interleaved(tr, N)
        solved = 0
        for _ in range(3):
            r = so.minimize(fun, zo + rng.normal(size=zo.shape) * 1e-4, method="SLSQP", constraints=cons,
                            options={"maxiter": 1000, "ftol": 1e-14})
            if r.success:
                solved += 1
                assert r.fun >= res["cost"] - 1e-7 * max(1.0, res["cost"])
        assert solved >= 1
