"""Pins of the timing-optimisation oracle (Sec. III-C: interval durations
among the controls; Sec. IV-A: an optimised time step under a duration
bound).  The dense restatement of the method reproduces the C oracle's
iterates when timing is fixed; with durations free the rows' Jacobians and
the curvature match finite differences, the straight push reaches its closed
form, pinned durations give back the fixed-step solution, a binding duration
bound ends at a KKT point, and SciPy finds no lower cost next to a solution."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import timing as TM

TIGHT = dict(eps_dual=1e-9, eps_primal=1e-11, eps_comp=1e-11, max_iters=1000, beta_max=1e6)


@pytest.mark.parametrize("modes", [(0, 3), (1, 7), (11, 2), (12, 0)])
def test_fixed_step_iterates_match_c_oracle(modes):
    inst = dict(W.push_l2_instance(3), n_modes=13)
    for it in (1, 5, 300):
        z, _, r = TM.solve(inst, modes, max_iters=it)
        tr, _, rc = oracle.solve(inst, np.array(modes, np.uint8), opts=oracle.default_opts(max_iters=it))
        zc = TM.interleave_c_traj(tr, 16)
        assert np.max(np.abs(z - zc)) <= 1e-9 * max(1.0, np.max(np.abs(zc))), (modes, it)
        assert (r["status"], r["iters"]) == (rc["status"], rc["iters"])
        assert r["cost"] == pytest.approx(rc["cost"], rel=1e-9)


@pytest.mark.parametrize("mode", range(13))
def test_timing_rows_jacobian_central_differences(mode):
    inst = W.push_l2_instance(1)
    timing = dict(h_min=0.05, h_max=0.2, T=2.0)
    rng = np.random.default_rng(mode)
    for smask in (False, True):
        L = TM.Layout(4, timing)
        sig = [TM.dyn_row_scale(inst, i) for i in range(4)]
        v = rng.normal(size=2 * L.nx + L.nu) * 0.1
        v[L.nx + 3] = 0.12
        split = lambda w: (w[:L.nx], w[L.nx:L.nx + L.nu], w[L.nx + L.nu:])
        c, mask, _, _, J = TM.interval_rows(inst, mode, smask, *split(v), L, timing, sig)
        eps = 1e-6
        Jfd = np.zeros_like(J)
        for j in range(len(v)):
            vp, vm = v.copy(), v.copy()
            vp[j] += eps
            vm[j] -= eps
            cp = TM.interval_rows(inst, mode, smask, *split(vp), L, timing, sig)[0]
            cm = TM.interval_rows(inst, mode, smask, *split(vm), L, timing, sig)[0]
            Jfd[:, j] = (cp - cm) / (2 * eps)
        np.testing.assert_allclose(J, Jfd, atol=1e-7, rtol=1e-6)


@pytest.mark.parametrize("mode", [0, 4, 8, 11, 12])
def test_timing_curvature_is_the_hessian_of_the_dynamics_rows(mode):
    # sum_i y_i d^2 c_i over (x_k, u_k) against differences of sum_i y_i grad c_i
    inst = W.push_l2_instance(5)
    timing = dict(h_min=0.05, h_max=0.2, T=2.0)
    L = TM.Layout(4, timing)
    sig = [TM.dyn_row_scale(inst, i) for i in range(4)]
    rng = np.random.default_rng(10 + mode)
    v = rng.normal(size=2 * L.nx + L.nu) * 0.2
    v[L.nx + 3] = 0.13
    y = rng.normal(size=4)
    split = lambda w: (w[:L.nx], w[L.nx:L.nx + L.nu], w[L.nx + L.nu:])

    def g(w):
        J = TM.interval_rows(inst, mode, False, *split(w), L, timing, sig)[4]
        return y @ J[:4]

    nxu = L.nx + L.nu
    Hfd = np.zeros((nxu, nxu))
    eps = 1e-6
    for j in range(nxu):
        vp, vm = v.copy(), v.copy()
        vp[j] += eps
        vm[j] -= eps
        Hfd[:, j] = (g(vp) - g(vm))[:nxu] / (2 * eps)
    xk, uk, _ = split(v)
    H = TM.stage_curvature(inst, mode, xk, uk, y / np.array(sig), L)
    np.testing.assert_allclose(H, Hfd, atol=1e-6, rtol=1e-6)


def test_straight_push_with_free_durations_closed_form():
    # goal (d, 0, 0), sticking on face 0: for durations h_k the optimal push
    # gives J = W R d^2 / (R + W kappa^2 sum h_k^2), decreasing in every h_k,
    # so with room in the duration bound every h_k sits at h_max
    d, N = 0.1, 16
    inst = W.push_l2_straight(d)
    Wt, R = inst["w_terminal"], inst["w_control"]
    timing = dict(h_min=0.05, h_max=0.15, T=3.0)
    z, lam, r = TM.solve(inst, (0, 0), timing=timing, **TIGHT)
    assert r["status"] == TM.CONVERGED
    h = TM.durations(inst, (0, 0), z, timing=timing)
    np.testing.assert_allclose(h, 0.15, atol=1e-9)
    assert r["cost"] == pytest.approx(Wt * R * d * d / (R + Wt * N * 0.15 ** 2), rel=1e-7)
    L = TM.Layout(N, timing)
    assert z[L.x(N) + 4] == pytest.approx(N * 0.15, rel=1e-9)            # elapsed time
    assert lam[-1] == 0.0                                               # the bound is slack
    fn = np.array([z[L.u(k)] for k in range(N)])
    np.testing.assert_allclose(fn, Wt * 0.15 * d / (Wt * N * 0.15 ** 2 + R), rtol=1e-6)


def test_pinned_durations_give_the_fixed_step_solution():
    inst = W.push_l2_instance(4)
    for modes in ((0, 3), (2, 2)):
        z, _, r = TM.solve(inst, modes, timing=dict(h_min=inst["dt"], h_max=inst["dt"], T=5.0), **TIGHT)
        zf, _, rf = TM.solve(inst, modes, **TIGHT)
        assert r["status"] == rf["status"] == TM.CONVERGED
        assert r["cost"] == pytest.approx(rf["cost"], rel=1e-7)
        Lt, Lf = TM.Layout(16, {}), TM.Layout(16, None)
        for k in range(17):
            np.testing.assert_allclose(z[Lt.x(k):Lt.x(k) + 4], zf[Lf.x(k):Lf.x(k) + 4], atol=1e-7)


def test_binding_duration_bound_ends_at_a_kkt_point():
    inst = W.push_l2_instance(2)
    timing = dict(h_min=0.02, h_max=0.3, T=1.2)
    modes = (7, 10)
    z, lam, r = TM.solve(inst, modes, timing=timing, max_iters=1500)
    assert r["status"] == TM.CONVERGED
    h = TM.durations(inst, modes, z, timing=timing)
    assert abs(h.sum() - 1.2) <= 1e-5 and np.all(h >= 0.02 - 1e-6) and np.all(h <= 0.3 + 1e-6)
    assert lam[-1] > 0.0                                                 # the bound binds
    P = TM.Problem(inst, modes, 16, timing)
    c, A, ineq, mask = TM.all_rows(P, z)
    # feasibility, sign and complementarity of the multipliers, stationarity
    assert np.max(np.abs(c[mask & ~ineq])) <= 1e-6 and np.max(c[mask & ineq]) <= 1e-6
    assert np.all(lam[mask & ineq] >= 0.0) and np.max(np.abs(lam * c)[mask & ineq]) <= 1e-6
    gl = P.cost_grad(z) + A[mask].T @ lam[mask]
    assert np.max(np.abs(gl)) <= 1e-4 * max(1.0, r["beta"] / 1e3)


def test_scipy_slsqp_finds_no_better_point_nearby():
    so = pytest.importorskip("scipy.optimize")
    inst = dict(W.push_l2_instance(9), knots_per_segment=4)
    timing = dict(h_min=0.05, h_max=0.2, T=0.6)
    N = 4
    for mode in (0, 4):
        z, lam, r = TM.solve(inst, (mode,), timing=timing, **TIGHT)
        assert r["status"] == TM.CONVERGED
        P = TM.Problem(inst, (mode,), N, timing)

        def eq(w):
            c, _, ineq, mask = TM.all_rows(P, w)
            return c[mask & ~ineq]

        def ineq_(w):
            c, _, ineq, mask = TM.all_rows(P, w)
            return -c[mask & ineq]

        cons = [{"type": "eq", "fun": eq}, {"type": "ineq", "fun": ineq_}]
        rng = np.random.default_rng(mode)
        ok = 0
        for _ in range(2):
            s = so.minimize(P.cost, z + rng.normal(size=z.shape) * 1e-4, method="SLSQP", constraints=cons,
                            options={"maxiter": 1000, "ftol": 1e-14})
            if s.success:
                ok += 1
                assert s.fun >= r["cost"] - 1e-7 * max(1.0, r["cost"])
        assert ok >= 1


def test_trial_step_is_the_armijo_rule():
    # sufficient decrease (Nocedal and Wright, Sec. 3.1) on phi(a) = (1 - a)^2
    # from phi(0) = 1 with phi'(0) = D = -2: alpha = 1 gives 0 <= 1 - 2 c1,
    # accepted for c1 < 1/2; with c1 = 0.6 it needs (1 - a)^2 <= 1 - 1.2 a,
    # i.e. a <= 0.8, so 1/2 is the largest accepted trial
    phi = lambda a: (1.0 - a) ** 2
    assert TM.trial_step(1.0, -2.0, phi, 7, 1e-4, 1e-6) == 1.0
    assert TM.trial_step(1.0, -2.0, phi, 7, 0.6, 1e-6) == 0.5
    # an ascent direction is never accepted, however small the increase
    assert TM.trial_step(1.0, -2.0, lambda a: 1.0 + 1e-9 * a, 7, 1e-4, 1e-12) == 0.0
    # a decrease below the merit's resolution: the full step is taken when it
    # raises phi by at most ls_slack |phi(0)|, else the Armijo test applies
    assert TM.trial_step(1.0, -1e-9, lambda a: 1.0 + 5e-7 * a, 7, 1e-4, 1e-6) == 1.0
    assert TM.trial_step(1.0, -1e-9, lambda a: 1.0 + 2e-6 * a, 7, 1e-4, 1e-6) == 0.0


# the other reading: one optimised time step shared by every interval

@pytest.mark.parametrize("mode", [0, 5, 9, 12])
def test_shared_step_rows_and_curvature_against_differences(mode):
    inst = W.push_l2_instance(6)
    timing = dict(shared=True, h_min=0.05, h_max=0.2, T=2.0)
    L = TM.Layout(4, timing)
    sig = [TM.dyn_row_scale(inst, i) for i in range(4)]
    rng = np.random.default_rng(40 + mode)
    v = rng.normal(size=2 * L.nx + L.nu) * 0.1
    v[4] = v[L.nx + L.nu + 4] = 0.11
    split = lambda w: (w[:L.nx], w[L.nx:L.nx + L.nu], w[L.nx + L.nu:])
    J = TM.interval_rows(inst, mode, False, *split(v), L, timing, sig)[4]
    y = rng.normal(size=4)
    eps = 1e-6
    Jfd = np.zeros_like(J)
    nxu = L.nx + L.nu
    Hfd = np.zeros((nxu, nxu))
    for j in range(len(v)):
        vp, vm = v.copy(), v.copy()
        vp[j] += eps
        vm[j] -= eps
        Jp = TM.interval_rows(inst, mode, False, *split(vp), L, timing, sig)
        Jm = TM.interval_rows(inst, mode, False, *split(vm), L, timing, sig)
        Jfd[:, j] = (Jp[0] - Jm[0]) / (2 * eps)
        if j < nxu:
            Hfd[:, j] = (y @ Jp[4][:4] - y @ Jm[4][:4])[:nxu] / (2 * eps)
    np.testing.assert_allclose(J, Jfd, atol=1e-7, rtol=1e-6)
    H = TM.stage_curvature(inst, mode, *split(v)[:2], y / np.array(sig), L)
    np.testing.assert_allclose(H, Hfd, atol=1e-6, rtol=1e-6)


@pytest.mark.parametrize("T,h_expect", [(2.0, 2.0 / 16), (3.0, 0.15)])
def test_straight_push_with_one_shared_step_closed_form(T, h_expect):
    # J(h) = W R d^2 / (R + W kappa^2 N h^2) decreases in h, so the optimal
    # shared step is min(h_max, T / N): the duration bound decides when it
    # binds, h_max otherwise
    d, N = 0.1, 16
    inst = W.push_l2_straight(d)
    Wt, R = inst["w_terminal"], inst["w_control"]
    timing = dict(shared=True, h_min=0.05, h_max=0.15, T=T)
    z, lam, r = TM.solve(inst, (0, 0), timing=timing, **TIGHT)
    assert r["status"] == TM.CONVERGED
    h = TM.durations(inst, (0, 0), z, timing=timing)
    np.testing.assert_allclose(h, h_expect, atol=1e-9)
    assert r["cost"] == pytest.approx(Wt * R * d * d / (R + Wt * N * h_expect ** 2), rel=1e-7)
    # the duration bound's multiplier is positive exactly when it binds
    assert (lam[-3] > 0.0) == (T / N < 0.15)


def test_shared_step_pinned_at_dt_gives_the_fixed_step_solution():
    inst = W.push_l2_instance(4)
    z, _, r = TM.solve(inst, (0, 3), timing=dict(shared=True, h_min=inst["dt"], h_max=inst["dt"], T=5.0),
                       **TIGHT)
    _, _, rf = TM.solve(inst, (0, 3), **TIGHT)
    assert r["status"] == rf["status"] == TM.CONVERGED
    assert r["cost"] == pytest.approx(rf["cost"], rel=1e-7)
