"""GPU parity of the CUDA evaluator (through the C ABI) against the FP64
oracle.  Paper: Eq. mode_nlp, Eq. inexact_mode_value, Eq. search_merit,
Eq. mode_selection, Sec. III-C.

The TO is a local, non-convex solve (Eq. mode_nlp: "not guaranteed to
attain J*(m)"), run in FP32 on the GPU and in FP64 by the oracle; the two
follow the same iteration but can part ways at a near-tie of a discrete
decision and then reach different local minima, each of them valid.  The
parity bar therefore has two parts:
  * every CONVERGED GPU result is certified by the oracle's own FP64
    residual evaluation (v_hat <= 1e-5, cone / unilateral rows hold);
  * where both converge to the same local solution, costs agree within
    1e-4 relative plus the first-order effect of the stop test's allowed
    infeasibility, |dJ| <= 1e-4 |J| + 2 * sum_i |lambda_i| * eps_primal
    (bounded here through the certified violation), and the fraction of
    such agreements, the status agreement and the enumeration argmin
    (wherever the oracle's cost gap exceeds 1e-3 relative) are checked.
"""
import os

import numpy as np
import pytest

import _parity as PA
import oracle
import workloads as W
from oracle import search as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_21803_gb300 import build as B
    B.build()
    import paper_2609_21803_gb300 as P
    P.lib()
    torch.cuda.set_device(0)
    return P


def gpu_eval(P, insts, seqs, inst_idx=None, lens=None, warm=None, want_traj=False, max_iters=0, opts=None):
    prob = P.Problem(insts, opts=opts)
    packed = P.pack_mode_seqs(seqs, inst_idx, lens)
    d = torch.from_numpy(packed.view(np.uint8).reshape(len(packed), P.MODE_SEQ_BYTES)).cuda()
    w = None if warm is None else torch.from_numpy(np.ascontiguousarray(warm, dtype=np.float32)).cuda()
    r = prob.eval(d, warm=w, want_traj=want_traj, max_iters=max_iters)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in r.items()}
    out["stride"] = prob.stride
    prob.close()
    return out


def certify_fp64(inst, modes, N, traj_f32, Nmax):
    """Physical violation of a GPU trajectory recomputed by the oracle."""
    Np1, Nm1 = N + 1, Nmax + 1
    tr = np.zeros(7 * N + 4)
    for i in range(4):
        tr[i * Np1: (i + 1) * Np1] = traj_f32[i * Nm1: i * Nm1 + Np1]
    for j in range(3):
        tr[4 * Np1 + j * N: 4 * Np1 + (j + 1) * N] = traj_f32[4 * Nm1 + j * Nmax: 4 * Nm1 + j * Nmax + N]
    c, mask, scale, ci = oracle.rows(inst, modes, N, tr)
    ineq = np.arange(11) >= 5
    v = np.where(ineq, np.maximum(c, 0.0), np.abs(c)) / scale * mask
    return max(float(np.max(v)), float(np.max(np.abs(ci)))), tr


def compare(gpu, ref, eps_primal=1e-6):
    cg, co = gpu["status"] == 0, ref["status"] == 0
    both = cg & co
    rel = np.abs(gpu["cost"].astype(np.float64) - ref["cost"]) / np.abs(ref["cost"])
    same = both & (rel < 1e-2)          # same local solution
    return cg, co, both, rel, same


def test_straight_push_closed_form(P):
    # goal (d, 0, 0) with face 0 sticking: J* = W R d^2 / (R + W N dt^2) = 10 d^2 / 17
    inst = W.push_l2_straight(0.1)
    seqs = np.array([[0, 0]], np.uint8)
    g = gpu_eval(P, [inst], seqs, want_traj=True)
    tr, lam, ref = oracle.solve(inst, [0, 0])
    assert g["status"][0] == P.TO_CONVERGED
    assert g["viol"][0] <= 1e-5
    # same algorithm: GPU (FP32) and oracle (FP64) land on the same point
    assert abs(g["cost"][0] - ref["cost"]) <= 1e-4 * ref["cost"]
    # against the closed form, up to the stop test's allowed infeasibility
    Jstar = 10 * 0.01 / 17
    assert abs(g["cost"][0] - Jstar) <= 5e-4 * Jstar
    fn = g["traj"][0][4 * 81: 4 * 81 + 16]
    np.testing.assert_allclose(fn, 0.1 / 1.7, rtol=2e-3)


def _nmax(g):
    return (int(g["stride"]) - 4) // 7


def _parity_asserts(rep, flags, n, label, remaining=None):
    """The acceptance bar on a compare() report (see tests/_parity.py)."""
    print(f"{label}: feasibility flags differ on {len(flags)} of {n} at t_exp: {flags}")
    if remaining is not None:
        print(f"{label}: still differ after the lagging side's refinement budget: {remaining}")
    print(f"{label}: different local solutions {[(d['t'], d['modes']) for d in rep['different']]}")
    print(f"{label}: unresolved {rep['unresolved']}")
    print(f"{label}: state bar exceeded (listed; cost bar, 1e-2 and certified stop hold) {rep['state_excess']}")
    # every converged GPU answer is feasible by the oracle's FP64 rows
    assert not rep["vhat_fail"], rep["vhat_fail"]
    # costs of the same local solution: 1e-4 relative plus the first-order
    # allowance, on the maximum
    assert not rep["cost_excess"], rep["cost_excess"]
    # knot states: within 1e-3 of the exact local solution beyond the
    # oracle's own distance; each listed exception is a certified stop of a
    # weakly determined solve (cost bar, 1e-2 and its FP64 stationarity)
    assert not rep["state_fail"], rep["state_fail"]
    assert len(rep["state_excess"]) <= max(3, 3 * rep["same"] // 100), len(rep["state_excess"])
    # a stop on the tolerances implies feasibility on either side, so a
    # flag disagreement needs one side that ended without the stop test
    assert all(sg != 0 or so != 0 for _, sg, so in flags)
    if remaining is not None:
        assert len(remaining) <= max(3, n // 100), remaining
    assert len(rep["unresolved"]) <= max(3, rep["joint"] // 50), rep["unresolved"]


def _reruns(P, insts, allseq, idx, lens):
    """Re-run functions of the lagging side at the refinement budget."""
    def gpu(ts):
        g = gpu_eval(P, insts, [allseq[t] for t in ts], np.asarray(idx)[ts], max_iters=1500)
        return g["status"], g["viol"]

    def ora(ts):
        seqs = np.asarray([allseq[t] for t in ts], np.uint8)
        r, _, _ = oracle.solve_batch_ex(insts, np.asarray(idx)[ts], seqs, np.asarray(lens)[ts],
                                        opts=oracle.default_opts(max_iters=1500), nthreads=os.cpu_count())
        return r["status"], r["viol"]
    return gpu, ora


def test_two_segment_enumeration_parity(P):
    # the 2-segment workload: every one of the 144 orders x 32 seeded goals
    seeds = range(32)
    insts = [W.push_l2_instance(s) for s in seeds]
    seqs = W.all_sequences(12, 2)
    n = len(seqs) * len(insts)
    allseq = np.tile(seqs, (len(insts), 1))
    idx = np.repeat(np.arange(len(insts)), len(seqs)).astype(np.int32)
    lens, Ns = np.full(n, 2, np.int32), np.full(n, 16)
    g = gpu_eval(P, insts, allseq, idx, want_traj=True)
    g["traj_nmax"] = _nmax(g)
    ref, rtr, _ = oracle.solve_batch_ex(insts, idx, allseq, lens, nthreads=os.cpu_count())
    T = PA.Task(False)
    rep = PA.compare(T, insts, idx, list(allseq), lens, Ns, g, ref, rtr)
    flags = PA.flag_disagreements(g, ref)
    remaining = PA.flags_after_refinement(flags, g, ref, *_reruns(P, insts, allseq, idx, lens))
    _parity_asserts(rep, flags, n, "N=16", remaining)
    # a GPU answer that reached another local solution is a certified one
    assert not PA.certify_different(T, insts, idx, list(allseq), lens, Ns, g, rep)
    # enumeration argmin (Eq. mode_selection) per instance
    out, bad = PA.argmin_parity(T, insts, [slice(144 * i, 144 * (i + 1)) for i in range(len(insts))], idx,
                                list(allseq), lens, Ns, g, ref, rtr)
    assert not bad, bad


def test_full_enumeration_parity_four_segments(P):
    # the benchmarked workload: 4-segment orders, N = 80, both 20,736-order
    # enumerations of two instances in one launch on the GPU and on the
    # oracle; the argmin of each instance is compared, the per-TO bar is
    # taken on a seeded sample of 1,024 orders per instance
    insts = [W.push_l4_instance(s) for s in (0, 1)]
    seqs = W.all_sequences(12, 4)
    m = len(seqs)
    n = 2 * m
    allseq = np.tile(seqs, (2, 1))
    idx = np.repeat(np.arange(2), m).astype(np.int32)
    lens, Ns = np.full(n, 4, np.int32), np.full(n, 80)
    g = gpu_eval(P, insts, allseq, idx, want_traj=True)
    g["traj_nmax"] = _nmax(g)
    ref, rtr, _ = oracle.solve_batch_ex(insts, idx, allseq, lens, nthreads=os.cpu_count())
    print(f"N=80: converged gpu {np.mean(g['status'] == 0):.4f} oracle {np.mean(ref['status'] == 0):.4f}")
    T = PA.Task(False)
    out, bad = PA.argmin_parity(T, insts, [slice(0, m), slice(m, n)], idx, list(allseq), lens, Ns, g, ref, rtr)
    assert not bad, bad
    rng = np.random.default_rng(0)
    sel = np.concatenate([np.sort(rng.choice(m, 1024, replace=False)) + i * m for i in range(2)])
    rep = PA.compare(T, insts, idx, list(allseq), lens, Ns, g, ref, rtr, sel=sel)
    flags = PA.flag_disagreements(g, ref, sel)
    _parity_asserts(rep, flags, len(sel), "N=80")
    assert not PA.certify_different(T, insts, idx, list(allseq), lens, Ns, g, rep)
    # feasibility flags over both whole enumerations, compared again after
    # the lagging side's refinement budget
    flags_all = PA.flag_disagreements(g, ref)
    remaining = PA.flags_after_refinement(flags_all, g, ref, *_reruns(P, insts, allseq, idx, lens))
    print(f"N=80 all orders: feasibility flags differ on {len(flags_all)} of {n} at t_exp, "
          f"{len(remaining)} after refinement: {remaining}")
    assert all(sg != 0 or so != 0 for _, sg, so in flags_all)
    assert len(remaining) <= n // 100


@pytest.mark.parametrize("iters", [1, 2, 5])
def test_iteration_level_parity(P, iters):
    # the GPU runs the oracle's iteration.  After one step from the same cold
    # start the iterates agree to FP32 rounding.  Later steps solve KKT
    # systems whose condition number reaches ~1e7 (beta |A|^2 / rho), so the
    # FP32 step carries relative errors ~1e-3 in its weakly damped directions:
    # the iterates then agree to that level and make the same progress
    # (cost and violation) rather than agreeing bit for bit.
    insts = [W.push_l2_instance(s) for s in range(4)]
    seqs = W.all_sequences(12, 2)
    n = len(seqs) * len(insts)
    allseq = np.tile(seqs, (len(insts), 1))
    idx = np.repeat(np.arange(len(insts)), len(seqs)).astype(np.int32)
    g = gpu_eval(P, insts, allseq, idx, want_traj=True, max_iters=iters)
    ref, tr = oracle.solve_batch(insts, idx, allseq, np.full(n, 2, np.int32), opts=oracle.default_opts(max_iters=iters),
                                 want_traj=True)
    d = np.max(np.abs(g["traj"][:, : 7 * 16 + 4].astype(np.float64) - tr[:, : 7 * 16 + 4]), axis=1)
    scale = np.maximum(1.0, np.max(np.abs(tr[:, : 7 * 16 + 4]), axis=1))
    print(f"iters {iters}: max diff p50 {np.median(d):.2e} p90 {np.percentile(d, 90):.2e}")
    assert np.all(g["iters"] == ref["iters"])
    if iters == 1:
        assert np.mean(d <= 1e-4 * scale) >= 0.99
    else:
        assert np.median(d / scale) <= 3e-3
        dJ = np.abs(g["cost"].astype(np.float64) - ref["cost"])
        assert np.mean(dJ <= 1e-2 * np.abs(ref["cost"]) + 1e-6) >= 0.95


def test_fp64_refinement_at_high_penalty(P):
    # one FP64 iterative-refinement step of the Riccati solve while the
    # penalty exceeds refine_beta.  The cap is raised to 1e5 so that the
    # penalty passes the threshold of 1e4; the run with the threshold at the
    # cap never refines and must equal the run with refinement switched off
    # bit for bit, the refined run must differ (the pass changes the step)
    # and keep the oracle's parity bar at the same options
    insts = [W.push_l2_instance(s) for s in range(6)]
    seqs = W.all_sequences(12, 2)
    n = len(seqs) * len(insts)
    allseq = np.tile(seqs, (len(insts), 1))
    idx = np.repeat(np.arange(len(insts)), len(seqs)).astype(np.int32)
    ref_on = gpu_eval(P, insts, allseq, idx, want_traj=True, opts={"beta_max": 1e5, "refine_beta": 1e4})
    at_cap = gpu_eval(P, insts, allseq, idx, want_traj=True, opts={"beta_max": 1e5, "refine_beta": 1e5})
    off = gpu_eval(P, insts, allseq, idx, want_traj=True, opts={"beta_max": 1e5, "precision_flags": 0})
    for k in ("cost", "status", "iters", "traj"):
        np.testing.assert_array_equal(at_cap[k], off[k])
    changed = (ref_on["iters"] != off["iters"]) | (ref_on["cost"] != off["cost"])
    assert changed.any()
    ref, _ = oracle.solve_batch(insts, idx, allseq, np.full(n, 2, np.int32), opts=oracle.default_opts(beta_max=1e5),
                                nthreads=os.cpu_count())
    cg, co, both, rel, same = compare(ref_on, ref)
    print(f"refined: changed {changed.mean():.3f} conv gpu {cg.mean():.4f} oracle {co.mean():.4f} "
          f"same {same.sum() / max(1, both.sum()):.4f} rel<1e-4 {np.mean(rel[both] < 1e-4):.4f}")
    assert cg.mean() >= 0.9 and abs(cg.mean() - co.mean()) <= 0.05
    assert same.sum() >= 0.85 * both.sum()
    for t in np.flatnonzero(cg)[::13]:
        v, _ = certify_fp64(insts[idx[t]], allseq[t], 16, ref_on["traj"][t], 16)
        assert v <= 1e-5, (t, v)


def test_mixed_lengths_and_instances_one_launch(P):
    # ragged launch: lengths 1..4 (N = 20..80) over three instances, 37 orders
    insts = [W.push_l4_instance(s) for s in (1, 2, 3)]
    rng = np.random.default_rng(3)
    seqs, idx = [], []
    for t in range(37):
        L = 1 + t % 4
        seqs.append(tuple(int(m) for m in rng.integers(0, 12, L)))
        idx.append(t % 3)
    g = gpu_eval(P, insts, seqs, idx)
    modes, lens = W.pad_sequences(seqs, 4)
    ref, _ = oracle.solve_batch(insts, np.array(idx, np.int32), modes, lens)
    cg, co, both, rel, same = compare(g, ref)
    assert cg.mean() >= 0.7
    assert same.sum() >= 0.8 * both.sum()
    assert np.all(g["iters"] <= 300)


def test_mixed_workload_full_launch_sampled(P):
    # the bench's mixed workload as timed: 256 rectangular sliders (length
    # caps 1..6, 10..30 knots per segment, N up to 180) with 512 random
    # orders each, 131,072 TOs in one launch at the autotuned shape; 64
    # seeded samples of its outputs against the oracle.  Trajectories of the
    # sample come from a second launch of those orders alone, which must give
    # the same outputs bit for bit (each TO's arithmetic does not depend on
    # its launch)
    insts = [W.push_mixed_instance(s) for s in range(256)]
    rng = np.random.default_rng(7)
    seqs, idx = [], []
    for i, inst in enumerate(insts):
        for _ in range(512):
            L = int(rng.integers(1, inst["max_segments"] + 1))
            seqs.append(tuple(int(m) for m in rng.integers(0, 12, L)))
            idx.append(i)
    n = len(seqs)
    idx = np.array(idx, np.int32)
    prob = P.Problem(insts)
    d = torch.from_numpy(P.pack_mode_seqs(seqs, idx).view(np.uint8).reshape(n, P.MODE_SEQ_BYTES)).cuda()
    P.comet_autotune(prob.handle, d[:8192], 8192, 40)
    r = prob.eval(d)
    torch.cuda.synchronize()
    full = {k: v.cpu().numpy() for k, v in r.items()}
    prob.close()
    conv = (full["status"] == 0) & (full["viol"] <= 1e-5)
    print(f"mixed workload, one launch: {int(conv.sum())} of {n} converged ({conv.mean():.3f})")
    picks = np.sort(np.random.default_rng(5).choice(n, 64, replace=False))
    ss = [seqs[t] for t in picks]
    si = idx[picks]
    g = gpu_eval(P, insts, ss, si, want_traj=True)
    g["traj_nmax"] = _nmax(g)
    for k in ("status", "cost", "viol", "iters"):
        np.testing.assert_array_equal(g[k], full[k][picks])
    modes, lens = W.pad_sequences(ss, 6)
    Ns = np.array([int(insts[i]["knots_per_segment"]) * int(L) for i, L in zip(si, lens)])
    ref, rtr, _ = oracle.solve_batch_ex(insts, si, modes, lens, nthreads=os.cpu_count())
    T = PA.Task(False)
    rep = PA.compare(T, insts, si, list(modes), lens, Ns, g, ref, rtr)
    flags = PA.flag_disagreements(g, ref)
    # re-runs of the lagging side with each order at its own length (the
    # padded mode array is the oracle's layout)
    _, rerun_oracle = _reruns(P, insts, modes, si, lens)

    def rerun_gpu(ts):
        r2 = gpu_eval(P, insts, [ss[t] for t in ts], si[ts], max_iters=1500)
        return r2["status"], r2["viol"]

    remaining = PA.flags_after_refinement(flags, g, ref, rerun_gpu, rerun_oracle)
    # on these sliders (aspect up to 3, mu up to 0.6, c down to 0.015 m) the
    # FP64 oracle itself often stops at stationary points that are not local
    # minima (its polish descends far), where no exact local solution is
    # attached to compare the GPU with: those are listed, and the GPU is held
    # to the bar wherever the oracle's answer is a local solution
    oracle_nonlocal = [u for u in rep["unresolved"] if not u["oracle_local"]]
    print(f"oracle stops at non-minimum stationary points: "
          f"{[(u['t'], u['modes'], u['gpu_local']) for u in oracle_nonlocal]}")
    rep_gpu = dict(rep, unresolved=[u for u in rep["unresolved"] if u["oracle_local"]])
    _parity_asserts(rep_gpu, flags, len(ss), "mixed workload, sampled", remaining)
    assert not PA.certify_different(T, insts, si, list(modes), lens, Ns, g, rep)


def test_bounded_wait_gives_up_and_reports_timeout(P):
    # failure detection without a fault: with the test hook on, the
    # warm-start staging copy is not issued, so the bounded wait on its
    # barrier runs out (nothing completes it, no copy is in flight); the TO
    # is flagged, the launch reports COMET_ERR_TIMEOUT, and the context stays
    # usable: the same problem then solves the same order from the same
    # warm start
    import time

    prob = P.Problem([W.push_l2_instance(0)])
    d = torch.from_numpy(P.pack_mode_seqs([(0, 3)]).view(np.uint8).reshape(1, P.MODE_SEQ_BYTES)).cuda()
    base = prob.eval(d, want_traj=True)
    warm = base["traj"].clone()
    assert P.comet_eval_check(prob.handle) == 0
    P.comet_debug_stall_staging(prob.handle, True)
    t0 = time.time()
    r = prob.eval(d, warm=warm)
    with pytest.raises(P.CometError, match="status 4"):
        P.comet_eval_check(prob.handle)
    dt = time.time() - t0
    print(f"the stalled launch ended after {dt:.1f} s")
    assert int(r["status"][0]) == P.TO_NONFINITE and np.isnan(float(r["cost"][0]))
    assert dt < 20.0
    P.comet_debug_stall_staging(prob.handle, False)
    r2 = prob.eval(d, warm=warm)
    assert P.comet_eval_check(prob.handle) == 0
    assert int(r2["status"][0]) == P.TO_CONVERGED
    assert float(r2["cost"][0]) == pytest.approx(float(base["cost"][0]), rel=1e-4)
    prob.close()


def test_warm_start_at_oracle_solution(P):
    inst = W.push_l2_instance(4)
    seqs = W.all_sequences(12, 2)[::13]
    n = len(seqs)
    ref, tr = oracle.solve_batch([inst], np.zeros(n, np.int32), seqs, np.full(n, 2, np.int32), want_traj=True)
    warm = np.zeros((n, 7 * 16 + 4), np.float32)
    warm[:] = tr[:, : 7 * 16 + 4]
    g = gpu_eval(P, [inst], seqs, warm=warm)
    # the same restart on the oracle (primal warm start, multipliers at
    # zero): where it converges within t_exp, so does the GPU
    r2, _, _ = oracle.solve_batch_ex([inst], np.zeros(n, np.int32), seqs, np.full(n, 2, np.int32), warm=tr)
    ok = (ref["status"] == 0) & (r2["status"] == 0)
    print("restart statuses: gpu", g["status"].tolist(), "oracle", r2["status"].tolist())
    assert np.all(g["status"][ok] == 0)
    # restarted at the oracle's point the GPU stays in its basin
    rel = np.abs(g["cost"][ok] - ref["cost"][ok]) / np.abs(ref["cost"][ok])
    assert np.all(rel < 1e-3) and np.median(rel) < 1e-4


def test_edge_cases(P):
    inst = W.push_l2_instance(0)
    prob = P.Problem([inst])
    # n = 0 is a no-op
    empty = torch.zeros((0, P.MODE_SEQ_BYTES), dtype=torch.uint8, device="cuda")
    out = prob.eval(empty)
    assert out["cost"].numel() == 0
    # one TO and a partial warp count
    for n in (1, 33):
        seqs = W.random_sequences(n, n, 12, 2)
        g = gpu_eval(P, [inst], seqs)
        assert g["cost"].shape == (n,) and np.all(np.isfinite(g["cost"]))
    # malformed orders from host memory are rejected before any work
    bad = P.pack_mode_seqs(np.array([[0, 12]], np.uint8))
    cost = np.zeros(1, np.float32)
    status = np.zeros(1, np.int32)
    with pytest.raises(P.CometError):
        P.comet_eval_modes(prob.handle, bad, 1, None, cost, None, status)
    bad = P.pack_mode_seqs(np.array([[0, 1, 2]], np.uint8))     # longer than max_segments
    with pytest.raises(P.CometError):
        P.comet_eval_modes(prob.handle, bad, 1, None, cost, None, status)
    # malformed orders in device memory: per-TO status, no call failure
    dbad = torch.from_numpy(P.pack_mode_seqs(np.array([[0, 12]], np.uint8)).view(np.uint8).reshape(1, P.MODE_SEQ_BYTES)).cuda()
    out = prob.eval(dbad)
    torch.cuda.synchronize()
    assert int(out["status"][0]) == P.TO_NONFINITE
    # non-finite warm start -> NONFINITE status
    warm = np.zeros((1, prob.stride), np.float32)
    warm[0, 3] = np.nan
    g = gpu_eval(P, [inst], np.array([[0, 1]], np.uint8), warm=warm)
    assert g["status"][0] == P.TO_NONFINITE
    prob.close()


def test_host_and_device_buffers_agree_and_runs_are_deterministic(P):
    insts = [W.push_l2_instance(6)]
    seqs = W.all_sequences(12, 2)
    n = len(seqs)
    prob = P.Problem(insts)
    packed = P.pack_mode_seqs(seqs)
    h_cost = np.zeros(n, np.float32)
    h_status = np.zeros(n, np.int32)
    h_traj = np.zeros((n, prob.stride), np.float32)
    P.comet_eval_modes(prob.handle, packed, n, None, h_cost, h_traj, h_status)
    d = torch.from_numpy(packed.view(np.uint8).reshape(n, P.MODE_SEQ_BYTES)).cuda()
    a = prob.eval(d, want_traj=True)
    b = prob.eval(d, want_traj=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a["cost"].cpu().numpy(), h_cost)
    np.testing.assert_array_equal(a["status"].cpu().numpy(), h_status)
    np.testing.assert_array_equal(a["traj"].cpu().numpy(), h_traj)
    np.testing.assert_array_equal(a["cost"].cpu().numpy(), b["cost"].cpu().numpy())
    prob.close()


def test_budget_entry_point(P):
    inst = W.push_l4_instance(9)
    seqs = W.all_sequences(12, 4)[:64]
    g5 = gpu_eval(P, [inst], seqs, max_iters=5)
    assert np.all(g5["iters"] <= 5)
    g = gpu_eval(P, [inst], seqs, max_iters=1500)
    assert np.mean(g["status"] == 0) >= np.mean(gpu_eval(P, [inst], seqs)["status"] == 0)


def test_long_horizon_parity(P):
    # mixed-workload sliders with N = 126..174: the forward pass gives each
    # lane 4..6 consecutive stages (ragged last lane at N = 126) and one
    # launch holds four horizons
    insts = [W.push_mixed_instance(s) for s in (8, 38, 39, 46)]
    Ns = [i["knots_per_segment"] * i["max_segments"] for i in insts]
    Nm = max(Ns)
    rng = np.random.default_rng(5)
    seqs, idx = [], []
    for i, inst in enumerate(insts):
        for _ in range(24):
            seqs.append(tuple(int(m) for m in rng.integers(0, 12, inst["max_segments"])))
            idx.append(i)
    idx = np.array(idx, np.int32)
    modes, lens = W.pad_sequences(seqs, 6)

    def xu(traj, N, stride_n):
        # x[4][stride_n + 1] then u[3][stride_n]: the GPU pads every TO to
        # N_max, the oracle writes each at its own N
        x = traj[: 4 * (stride_n + 1)].reshape(4, stride_n + 1)[:, : N + 1]
        u = traj[4 * (stride_n + 1): 4 * (stride_n + 1) + 3 * stride_n].reshape(3, stride_n)[:, :N]
        return np.concatenate([x.ravel(), u.ravel()]).astype(np.float64)

    # one iteration from the same cold start agrees to the FP32 error of the
    # first Newton step.  Over 126..174 stages that step's relative error
    # reaches a few 1e-4 (the KKT system at beta = 100, rho = 1e-4 is far
    # worse conditioned than at N = 16, where 1e-4 holds); the sequential
    # and the lane-split forward passes give identical iterates here, so the
    # bar is 1e-3 relative (max measured 2.7e-4)
    g1 = gpu_eval(P, insts, seqs, idx, want_traj=True, max_iters=1)
    r1, t1 = oracle.solve_batch(insts, idx, modes, lens, opts=oracle.default_opts(max_iters=1), want_traj=True)
    assert g1["stride"] == t1.shape[1]
    ok = []
    for t in range(len(seqs)):
        N = Ns[idx[t]]
        a, b = xu(g1["traj"][t], N, Nm), xu(t1[t], N, N)
        ok.append(np.max(np.abs(a - b)) <= 1e-3 * max(1.0, np.max(np.abs(b))))
    assert np.mean(ok) >= 0.99, np.mean(ok)
    # full solves: same convergence, same local solutions, certified
    g = gpu_eval(P, insts, seqs, idx, want_traj=True)
    ref, _ = oracle.solve_batch(insts, idx, modes, lens)
    cg, co, both, rel, same = compare(g, ref)
    print(f"N 126..174: converged gpu {cg.mean():.3f} oracle {co.mean():.3f}; same {same.sum()}/{both.sum()}")
    assert abs(cg.mean() - co.mean()) <= 0.1
    assert same.sum() >= 0.8 * both.sum()
    for t in np.flatnonzero(cg & (g["viol"] <= 1e-5))[::5]:
        assert certify_fp64(insts[idx[t]], seqs[t], Ns[idx[t]], g["traj"][t], Nm)[0] <= 1e-5, t


def test_free_motion_closed_form_and_grammar_parity(P):
    # free motion (mode 12 of the 13-mode pushing alphabet): free then a
    # straight sticking push from face 0 equals the straight push over the
    # contact intervals alone, J* = W R d^2 / (R + W K dt^2)
    inst = dict(W.push_l2_straight(0.1), n_modes=13)
    K, Wt, R, dt, d = inst["knots_per_segment"], inst["w_terminal"], inst["w_control"], inst["dt"], 0.1
    g = gpu_eval(P, [inst], np.array([[12, 0]], np.uint8), want_traj=True)
    assert g["status"][0] == 0 and g["viol"][0] <= 1e-5
    Jstar = Wt * R * d * d / (R + Wt * K * dt * dt)
    assert abs(g["cost"][0] - Jstar) <= 5e-4 * Jstar
    U = g["traj"][0][4 * 17: 4 * 17 + 3 * 16].reshape(3, 16)
    assert np.max(np.abs(U[:, :K])) <= 1e-4
    # every admissible order of 2..4 segments (start in free motion, faces
    # change through free motion or to an adjacent face) on three instances
    insts = [dict(W.push_l4_instance(s), n_modes=13) for s in range(3)]
    orders = [s for s in S.admissible_orders(4) if len(s) >= 2]
    seqs = [s for s in orders for _ in range(3)]
    idx = np.array([i for _ in orders for i in range(3)], np.int32)
    modes, lens = W.pad_sequences(seqs, 4)
    Ns = [20 * len(s) for s in seqs]
    # first iterate: FP32 rounding of the same step (1e-3: N up to 80)
    g1 = gpu_eval(P, insts, seqs, idx, want_traj=True, max_iters=1)
    r1, t1 = oracle.solve_batch(insts, idx, modes, lens, opts=oracle.default_opts(max_iters=1), want_traj=True)
    ok = []
    for t in range(len(seqs)):
        N = Ns[t]
        a = np.concatenate([g1["traj"][t][: 4 * 81].reshape(4, 81)[:, : N + 1].ravel(),
                            g1["traj"][t][4 * 81: 4 * 81 + 240].reshape(3, 80)[:, :N].ravel()])
        b = t1[t][: 7 * N + 4]
        ok.append(np.max(np.abs(a - b)) <= 1e-3 * max(1.0, np.max(np.abs(b))))
    assert np.mean(ok) >= 0.99
    # full solves.  Orders with free motion converge a little less often in
    # FP32 than in FP64 (measured at the 300-iteration budget: 89 % against
    # the oracle's 93 %; 77 % before the theta row was evaluated in
    # double-float): where both converge they reach the same solutions, and
    # with a 1,500-iteration budget the GPU converges as often as the oracle
    # at 300
    g = gpu_eval(P, insts, seqs, idx, want_traj=True)
    ref, _ = oracle.solve_batch(insts, idx, modes, lens)
    cg, co, both, rel, same = compare(g, ref)
    g_long = gpu_eval(P, insts, seqs, idx, max_iters=1500)
    cl = g_long["status"] == 0
    print(f"grammar orders: converged gpu {cg.mean():.3f} (1,500 iterations {cl.mean():.3f}) "
          f"oracle {co.mean():.3f}; same {same.sum()}/{both.sum()}")
    assert cg.mean() >= co.mean() - 0.1
    assert abs(cl.mean() - co.mean()) <= 0.08
    assert same.sum() >= 0.9 * both.sum()
    for t in np.flatnonzero(cg & (g["viol"] <= 1e-5))[::4]:
        v, tr = certify_fp64(insts[idx[t]], seqs[t], Ns[t], g["traj"][t], 80)
        assert v <= 1e-5, t
        # no contact force during free motion: f_n = 0 is a row (feasibility
        # 1e-5), f_t is set by the effort cost alone (stationarity 1e-4 over
        # 2 w_control = 0.2, i.e. 5e-4)
        seg = [oracle.segment_of(k, len(seqs[t]), Ns[t]) for k in range(Ns[t])]
        Uf = tr[4 * (Ns[t] + 1):].reshape(3, Ns[t])[:2, [seqs[t][q] == 12 for q in seg]]
        assert np.max(np.abs(Uf[0]), initial=0.0) <= 1e-5 and np.max(np.abs(Uf[1]), initial=0.0) <= 5e-4, t
