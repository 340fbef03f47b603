"""Pins of the oracle's solver (no GPU): the backward sweep equals a dense
solve of the assembled system; closed-form straight push; symmetry and
translation invariance; KKT at converged points; SciPy cross-check on tiny
instances; brute-force enumeration.  Paper: Sec. III-C (fixed-workspace
local solves, stopping and scoring), Eq. mode_nlp, Eq. inexact_mode_value,
Eq. mode_selection."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from _helpers import cost_grad_hess, dense_step, multipliers, to_component, to_interleaved

TIGHT = dict(eps_dual=1e-9, eps_primal=1e-11, eps_comp=1e-11, max_iters=1000, beta_max=1e6)


def _random_point(inst, N, seed):
    rng = np.random.default_rng(seed)
    tr = oracle.cold_start(inst, N)
    tr = tr + rng.normal(size=tr.shape) * 0.02
    lam = rng.normal(size=3 + 11 * N) * 0.1
    return tr, lam


@pytest.mark.parametrize("modes", [[0, 0], [1, 5], [7, 11], [2, 9]])
@pytest.mark.parametrize("curvature", [False, True])
def test_backward_sweep_equals_dense_solve(modes, curvature):
    inst = W.push_l2_instance(5)
    N = 6 if curvature else 16
    tr, lam = _random_point(inst, N, sum(modes))
    # with the curvature term the model may be indefinite at a random point:
    # a larger damping keeps every local S_k positive definite
    pairs = [(100.0, 1.0), (1e4, 1.0)] if curvature else [(100.0, 1e-4), (1e4, 1e-2)]
    for beta, rho in pairs:
        while True:
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


def test_al_merit_matches_definition():
    inst = W.push_l2_instance(1)
    N = 16
    tr, lam = _random_point(inst, N, 3)
    beta = 300.0
    L, J = oracle.al_merit(inst, [4, 8], N, tr, lam, beta)
    z = to_interleaved(tr, N)
    Jref = inst["w_terminal"] * np.sum((z[7 * N: 7 * N + 3] - inst["goal"]) ** 2) + inst["w_control"] * sum(
        np.sum(z[7 * k + 4: 7 * k + 7] ** 2) for k in range(N))
    assert J == pytest.approx(Jref, rel=1e-13)
    c, mask, _, ci = oracle.rows(inst, [4, 8], N, tr)
    cc = np.concatenate([ci, c.ravel()])
    mk = np.concatenate([np.ones(3, bool), mask.ravel().astype(bool)])
    ineq = np.zeros_like(mk); ineq[3:] = np.tile(np.arange(11) >= 5, N)
    t = np.where(ineq, (np.maximum(0, lam + beta * cc) ** 2 - lam ** 2) / (2 * beta), lam * cc + 0.5 * beta * cc ** 2)
    assert L == pytest.approx(Jref + np.sum(t[mk]), rel=1e-13)


@pytest.mark.parametrize("d", [0.05, 0.1, -0.08])
def test_straight_sticking_push_closed_form(d):
    # goal (d, 0, 0), face 0 sticking on every interval: by symmetry s = f_t = 0
    # and constant f_n; min W (N dt k f - d)^2 + R N f^2  =>  J* = W R d^2 / (R + W N dt^2 k^2)
    inst = W.push_l2_straight(abs(d)) if d > 0 else None
    if d < 0:  # push from the +x face (face 2) toward -x
        inst = W.push_l2_straight(0.1)
        inst["goal"] = [d, 0.0, 0.0]
    face_mode = 0 if d > 0 else 6
    N, Wt, R, dt = 16, inst["w_terminal"], inst["w_control"], inst["dt"]
    tr, lam, res = oracle.solve(inst, [face_mode, face_mode], opts=oracle.default_opts(**TIGHT))
    assert res["status"] == oracle.CONVERGED
    Jstar = Wt * R * d * d / (R + Wt * N * dt * dt)
    assert res["cost"] == pytest.approx(Jstar, rel=1e-7)
    fstar = Wt * dt * abs(d) / (Wt * N * dt * dt + R)
    np.testing.assert_allclose(tr[4 * 17: 4 * 17 + N], fstar, rtol=1e-6)
    assert tr[16] == pytest.approx(N * dt * fstar * np.sign(d), rel=1e-6)


def test_straight_push_is_enumeration_argmin():
    # brute force over all 144 two-segment orders (Eq. mode_selection)
    inst = W.push_l2_straight(0.1)
    seqs = W.all_sequences(12, 2)
    res, _ = oracle.solve_batch([inst], np.zeros(144, np.int32), seqs, np.full(144, 2, np.int32))
    feas = res["viol"] <= 1e-5
    order = np.lexsort((np.arange(144), np.where(feas, res["merit"], np.inf)))
    assert tuple(seqs[order[0]]) == (0, 0)
    assert res["cost"][order[0]] == pytest.approx(10 * 0.01 / 17, rel=1e-3)


MIRROR_FACE = [0, 3, 2, 1]
MIRROR_KIND = [0, 2, 1]


def _mirror(m):
    return 3 * MIRROR_FACE[m // 3] + MIRROR_KIND[m % 3]


def test_mirror_symmetry_of_mode_values():
    # reflection y -> -y, theta -> -theta maps face 1 <-> 3, slide+ <-> slide-,
    # s -> -s: the J(m) table is identical under the mode map
    inst = W.push_l2_instance(7)
    mir = dict(inst)
    mir["goal"] = [inst["goal"][0], -inst["goal"][1], -inst["goal"][2]]
    seqs = W.all_sequences(12, 2)[::7]
    mseqs = np.vectorize(_mirror)(seqs).astype(np.uint8)
    n = len(seqs)
    a, _ = oracle.solve_batch([inst], np.zeros(n, np.int32), seqs, np.full(n, 2, np.int32))
    b, _ = oracle.solve_batch([mir], np.zeros(n, np.int32), mseqs, np.full(n, 2, np.int32))
    np.testing.assert_array_equal(a["status"], b["status"])
    np.testing.assert_allclose(a["cost"], b["cost"], rtol=1e-8, atol=1e-12)


def test_translation_invariance():
    inst = W.push_l2_instance(2)
    sh = dict(inst)
    sh["start"] = [0.125, -0.25, 0.0]
    sh["goal"] = [inst["goal"][0] + 0.125, inst["goal"][1] - 0.25, inst["goal"][2]]
    seqs = W.all_sequences(12, 2)[::11]
    n = len(seqs)
    a, _ = oracle.solve_batch([inst], np.zeros(n, np.int32), seqs, np.full(n, 2, np.int32))
    b, _ = oracle.solve_batch([sh], np.zeros(n, np.int32), seqs, np.full(n, 2, np.int32))
    conv = (a["status"] == 0) & (b["status"] == 0)
    assert conv.mean() > 0.8
    np.testing.assert_allclose(a["cost"][conv], b["cost"][conv], rtol=1e-6, atol=1e-10)


@pytest.mark.parametrize("seed", [0, 4])
def test_kkt_at_converged_points(seed):
    # every CONVERGED result is a KKT point of Eq. mode_nlp: feasibility,
    # lambda_I >= 0, stationarity and complementarity, checked on the dense
    # Jacobian independently of the solver's own measures
    inst = W.push_l2_instance(seed)
    N = 16
    for modes in ([0, 4], [3, 3], [10, 2], [8, 6]):
        tr, lam, res = oracle.solve(inst, modes, opts=oracle.default_opts(**TIGHT))
        if res["status"] != oracle.CONVERGED:
            continue
        c, mask, scale, ci = oracle.rows(inst, modes, N, tr)
        cc = np.concatenate([ci, c.ravel()])
        mk = np.concatenate([np.ones(3, bool), mask.ravel().astype(bool)])
        ineq = np.zeros_like(mk); ineq[3:] = np.tile(np.arange(11) >= 5, N)
        assert np.max(np.abs(cc[mk & ~ineq])) <= 1e-9
        assert np.max(np.maximum(cc[mk & ineq], 0)) <= 1e-9
        assert np.all(lam[ineq] >= 0) and np.all(lam[~mk] == 0)
        z = to_interleaved(tr, N)
        gJ, _ = cost_grad_hess(inst, N, z)
        r = gJ + oracle.dense_jacobian(inst, modes, N, tr).T @ lam
        assert np.max(np.abs(r)) <= 1e-7
        assert np.max(np.abs(lam[ineq] * cc[ineq])) <= 1e-9
        # physical checks: friction cone and unilateral force
        fn, ft = tr[4 * 17: 4 * 17 + N], tr[4 * 17 + N: 4 * 17 + 2 * N]
        assert np.all(fn >= -1e-9) and np.all(np.abs(ft) <= inst["mu"] * fn + 1e-9)


def test_nonfinite_warm_start_reports_status():
    inst = W.push_l2_instance(0)
    N = 16
    warm = oracle.cold_start(inst, N)
    warm[5] = np.nan
    _, _, res = oracle.solve(inst, [0, 1], warm=warm)
    assert res["status"] == oracle.NONFINITE


def test_scipy_slsqp_finds_no_better_point_nearby():
    # tiny instance (one segment, N = 4): SciPy's SLSQP on the same NLP
    # (Eq. mode_nlp), started next to the oracle's solution, finds no lower
    # cost (the oracle returns a local minimum, not only a KKT point; the
    # problem is non-convex, so other starts may reach other minima)
    so = pytest.importorskip("scipy.optimize")
    inst = W.push_l2_instance(9)
    inst["knots_per_segment"] = 4
    N = 4
    for mode in (0, 4, 7, 2):
        tr, lam, res = oracle.solve(inst, [mode], opts=oracle.default_opts(**TIGHT))
        assert res["status"] == oracle.CONVERGED

        def fun(z):
            return inst["w_terminal"] * np.sum((z[7 * N: 7 * N + 3] - inst["goal"]) ** 2) + inst["w_control"] * sum(
                np.sum(z[7 * k + 4: 7 * k + 7] ** 2) for k in range(N))

        def cons(z):
            c, mask, _, ci = oracle.rows(inst, [mode], N, to_component(z, N))
            return np.concatenate([ci, c.ravel()]), mask.ravel().astype(bool)

        def eq(z):
            cc, mk = cons(z)
            keep = np.concatenate([np.ones(3, bool), np.tile(np.arange(11) < 5, N) & mk])
            return cc[keep]

        def ineq(z):
            cc, mk = cons(z)
            keep = np.concatenate([np.zeros(3, bool), np.tile(np.arange(11) >= 5, N) & mk])
            return -cc[keep]

        cons_ = [{"type": "eq", "fun": eq}, {"type": "ineq", "fun": ineq}]
        rng = np.random.default_rng(mode)
        zo = to_interleaved(tr, N)
        for _ in range(3):
            r = so.minimize(fun, zo + rng.normal(size=zo.shape) * 1e-4, method="SLSQP", constraints=cons_,
                            options={"maxiter": 1000, "ftol": 1e-14})
            if r.success:
                assert r.fun >= res["cost"] - 1e-7 * max(1.0, res["cost"])
