"""GPU parity of the bimanual evaluator (one CTA per TO) against the FP64
bimanual oracle, through the C ABI.

Same bar as the pushing evaluator (tests/_parity.py): the TO is local and
non-convex and runs in FP32 on the GPU, so the two sides can reach different
local solutions, which are listed and certified one by one; where both reach
the same local solution, costs agree within 1e-4 relative plus the
first-order allowance and knot states within 1e-3 of the exact local
solution beyond the oracle's own distance, on the maximum.  v_hat is scored
in physical units (N, N m, m, m/s, W) on both sides, and both use the
library's default stop test (stationarity relative to max(1, |J|)).
"""
import numpy as np
import pytest

import _parity as PA
import oracle
import workloads as W
from oracle import search as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

G = oracle.GRAVITY


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


def _ev(P, insts, seqs, idx=None, warm=None, want_traj=True, max_iters=0):
    prob = P.Problem(insts)
    packed = P.pack_mode_seqs(seqs, idx)
    d = torch.from_numpy(packed.view(np.uint8).reshape(len(seqs), P.MODE_SEQ_BYTES)).cuda()
    w = None if warm is None else torch.from_numpy(np.ascontiguousarray(warm, np.float32)).cuda()
    r = prob.eval(d, warm=w, want_traj=want_traj, max_iters=max_iters)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in r.items()}
    out["stride"] = prob.stride
    prob.close()
    return out


def _opts(**kw):
    return oracle.default_opts(**kw)


def _to_oracle(traj, N, Nmax):
    """GPU layout x[5][Nmax+1], u[12][Nmax] -> oracle x[5][N+1], u[12][N]."""
    x = traj[: 5 * (Nmax + 1)].reshape(5, Nmax + 1)[:, : N + 1]
    u = traj[5 * (Nmax + 1): 5 * (Nmax + 1) + 12 * Nmax].reshape(12, Nmax)[:, :N]
    return np.concatenate([x.ravel(), u.ravel()]).astype(np.float64)


def _certify(inst, modes, N, tr):
    c, mask, scale, ci = oracle.bim_rows(inst, modes, N, tr)
    ineq = np.zeros(32, bool)
    ineq[11:16] = ineq[19:24] = ineq[27:] = True
    v = np.where(ineq[None, :], np.maximum(c, 0), np.abs(c)) / scale * mask
    return max(float(v.max()), float(np.abs(ci).max()))


def test_box_at_rest_closed_form(P):
    inst = W.bimanual_instance(2)
    inst["goal"] = list(inst["start"])
    g = _ev(P, [inst], [(W.bimanual_mode(0, 0, 0),)])
    assert g["status"][0] == 0
    assert g["cost"][0] == pytest.approx(15 * inst["w_control"], rel=1e-4)
    u = g["traj"][0][5 * 91: 5 * 91 + 12 * 90].reshape(12, 90)[:, :15]
    np.testing.assert_allclose(u[9], inst["mass"] * G, rtol=1e-5)


def test_sliding_push_closed_form(P):
    inst = W.bimanual_instance(3)
    ax = 0.5 * inst["side_x"]
    inst["side_y"] = min(inst["side_y"], 2.5 * ax)
    az = 0.5 * inst["side_y"]
    inst["start"] = [0.0, az, 0.0]
    inst["goal"] = [0.05, az, 0.0]
    # at the refinement budget t_ref: on this heavy box with a small cost the
    # FP32 stationarity floor sits near the tolerance (the solution below is
    # reached well within t_exp, the stop test later)
    g = _ev(P, [inst], [(W.bimanual_mode(1, 1, 0),)], max_iters=1500)
    assert g["status"][0] == 0 and g["viol"][0] <= 1e-5
    mg = inst["mass"] * G
    u = g["traj"][0][5 * 91: 5 * 91 + 12 * 90].reshape(12, 90)[:, :15]
    np.testing.assert_allclose(u[3] / mg, 0.4, atol=2e-4)
    np.testing.assert_allclose(u[4] / mg, 0.2, atol=2e-4)
    np.testing.assert_allclose(u[9] / mg, 0.8, atol=2e-4)
    np.testing.assert_allclose(u[10] / mg, -0.4, atol=2e-4)


def test_first_iterate_matches_oracle(P):
    insts = [W.bimanual_instance(0)]
    rng = np.random.default_rng(1)
    seqs = [(int(m),) for m in rng.choice(507, 24, replace=False)]
    g = _ev(P, insts, seqs, max_iters=1)
    ref, tr = oracle.bim_solve_batch(insts, np.zeros(24, np.int32), seqs, np.ones(24, np.int32),
                                     opts=_opts(max_iters=1), want_traj=True)
    for i in range(24):
        got = _to_oracle(g["traj"][i], 15, 90)
        scale = max(1.0, np.abs(tr[i]).max())
        assert np.max(np.abs(got - tr[i])) <= 1e-4 * scale, i


def _bim_asserts(rep, flags, n, label, remaining=None):
    print(f"{label}: feasibility flags differ on {len(flags)} of {n} at t_exp: {flags}")
    if remaining is not None:
        print(f"{label}: still differ after the lagging side's refinement budget: {remaining}")
    print(f"{label}: different local solutions {[(d['t'], d['modes']) for d in rep['different']]}")
    print(f"{label}: unresolved {rep['unresolved']}")
    print(f"{label}: state bar exceeded (listed; cost bar, 1e-2 and certified stop hold) {rep['state_excess']}")
    assert not rep["vhat_fail"], rep["vhat_fail"]
    assert not rep["cost_excess"], rep["cost_excess"]
    assert not rep["state_fail"], rep["state_fail"]
    assert len(rep["state_excess"]) <= max(3, 3 * rep["same"] // 100), len(rep["state_excess"])
    assert all(sg != 0 or so != 0 for _, sg, so in flags)
    if remaining is not None:
        assert len(remaining) <= max(3, n // 100), remaining
    assert len(rep["unresolved"]) <= max(3, rep["joint"] // 50), rep["unresolved"]


def _bim_reruns(P, insts, seqs, idx, lens):
    def gpu(ts):
        g = _ev(P, insts, [seqs[t] for t in ts], np.asarray(idx)[ts], max_iters=1500)
        return g["status"], g["viol"]

    def ora(ts):
        r, _, _ = oracle.bim_solve_batch_ex(insts, np.asarray(idx)[ts], [seqs[t] for t in ts], np.asarray(lens)[ts],
                                            opts=_opts(max_iters=1500))
        return r["status"], r["viol"]
    return gpu, ora


def test_enumeration_parity_one_segment_and_mixed(P):
    insts = [W.bimanual_instance(s) for s in range(2)]
    rng = np.random.default_rng(0)
    seqs = [(m,) for m in range(507)] * 2 + [tuple(int(m) for m in rng.integers(0, 507, rng.integers(2, 4)))
                                             for _ in range(120)]
    idx = np.concatenate([np.repeat([0, 1], 507), rng.integers(0, 2, 120)]).astype(np.int32)
    lens = np.array([len(s) for s in seqs], np.int32)
    Ns = 15 * lens
    g = _ev(P, insts, seqs, idx)
    g["traj_nmax"] = 90
    ref, rtr, _ = oracle.bim_solve_batch_ex(insts, idx, seqs, lens, opts=_opts())
    cg, co = (g["status"] == 0) & (g["viol"] <= 1e-5), (ref["status"] == 0) & (ref["viol"] <= 1e-5)
    print(f"bimanual: feasible gpu {cg.mean():.3f} oracle {co.mean():.3f}")
    T = PA.Task(True)
    rep = PA.compare(T, insts, idx, seqs, lens, Ns, g, ref, rtr)
    flags = PA.flag_disagreements(g, ref)
    remaining = PA.flags_after_refinement(flags, g, ref, *_bim_reruns(P, insts, seqs, idx, lens))
    _bim_asserts(rep, flags, len(seqs), "bimanual 1-3 segments", remaining)
    assert not PA.certify_different(T, insts, idx, seqs, lens, Ns, g, rep)
    # the enumeration argmin over the one-segment orders of each instance
    out, bad = PA.argmin_parity(T, insts, [slice(507 * i, 507 * (i + 1)) for i in range(2)], idx, seqs, lens, Ns,
                                g, ref, rtr)
    assert not bad, bad


def test_warm_start_and_malformed_orders(P):
    inst = W.bimanual_instance(4)
    modes = (358,)
    r, tr, _ = oracle.bim_solve(inst, modes, 15, opts=_opts())
    assert r["status"] == 0
    warm = np.zeros(17 * 90 + 5, np.float32)
    x = tr[: 5 * 16].reshape(5, 16)
    u = tr[5 * 16:].reshape(12, 15)
    warm[: 5 * 91].reshape(5, 91)[:, :16] = x
    warm[5 * 91:].reshape(12, 90)[:, :15] = u
    g = _ev(P, [inst], [modes], warm=warm[None, :])
    assert g["status"][0] == 0 and g["iters"][0] <= 40
    assert g["cost"][0] == pytest.approx(r["cost"], rel=1e-4)
    # a mode index past the alphabet gives the NONFINITE status, not a fault
    prob = P.Problem([inst])
    bad = P.pack_mode_seqs([(507,), (12,)])
    dbad = torch.from_numpy(bad.view(np.uint8).reshape(2, P.MODE_SEQ_BYTES)).cuda()
    rr = prob.eval(dbad)
    st = rr["status"].cpu().numpy()
    assert st[0] == 4 and st[1] in (0, 1, 2)
    prob.close()
    # a problem holds one task; the launch-shape calls reject a bimanual
    # problem (one CTA per TO); the learned proposal takes it (its bimanual
    # layout is tested in tests/test_gpu_learned_bimanual.py)
    with pytest.raises(P.CometError):
        P.Problem([inst, W.push_l4_instance(0)])
    prob = P.Problem([inst])
    with pytest.raises(P.CometError):
        P.comet_set_launch_config(prob.handle, 2, 1)
    prob.close()


def test_expansion_over_507_modes_matches_oracle(P):
    inst = W.bimanual_instance(0)
    prob = P.Problem([inst])
    M, lmax = 507, 6
    rng = np.random.default_rng(7)
    seqs = list({tuple(int(m) for m in rng.integers(0, M, rng.integers(1, 3))) for _ in range(200)})
    merit = (rng.integers(0, 20, len(seqs)) * 0.125 + 0.5).astype(np.float32)
    f = P.comet_frontier_create(prob.handle, 0, 200000, 20000, 16)
    P.comet_frontier_add(f, P.pack_mode_seqs(seqs), len(seqs), merit, np.zeros(len(seqs), np.float32))
    P.comet_expand(prob.handle, f, 4)
    got = P.frontier_next_orders(f, 20000)
    V = {S.encode(s, M): (float(m), s) for s, m in zip(seqs, merit)}
    want = S.expand(V, k=4, batch=20000, n_modes=M, l_max=lmax)
    assert got == want
    P.comet_frontier_destroy(f)
    prob.close()


def test_bimanual_plan(P):
    # Algorithm 1 on one instance: seed = the 507 one-segment orders, beam
    # 16, batch 1,024, two rounds; the refined best is a certified plan
    inst = W.bimanual_instance(6)
    prob = P.Problem([inst])
    seeds = P.pack_mode_seqs([(m,) for m in range(507)])
    traj = np.zeros(prob.stride, np.float32)
    r = P.comet_plan(prob.handle, 0, seeds, 507, dict(k=16, batch=1024, rounds=2, k_ref=64), out_traj=traj)
    print("bimanual plan", r)
    assert r["best_status"] == 0 and r["best_viol"] <= 1e-5
    N = 15 * len(r["best"])
    v = _certify(inst, r["best"], N, _to_oracle(traj, N, 90))
    assert v <= 1e-5
    prob.close()


def test_long_orders_convergence_matches_oracle(P):
    # random orders of 1..6 segments (N up to 90): the GPU's feasible
    # fraction tracks the FP64 oracle's on the same orders; the per-TO bar
    # holds where both are feasible
    insts = [W.bimanual_instance(s) for s in range(8)]
    rng = np.random.default_rng(11)
    seqs, idx = [], []
    for i in range(8):
        for _ in range(32):
            L = int(rng.integers(1, 7))
            seqs.append(tuple(int(m) for m in rng.integers(0, 507, L)))
            idx.append(i)
    idx = np.array(idx, np.int32)
    lens = np.array([len(s) for s in seqs], np.int32)
    g = _ev(P, insts, seqs, idx)
    g["traj_nmax"] = 90
    ref, rtr, _ = oracle.bim_solve_batch_ex(insts, idx, seqs, lens, opts=_opts())
    cg = (g["status"] == 0) & (g["viol"] <= 1e-5)
    co = (ref["status"] == 0) & (ref["viol"] <= 1e-5)
    print(f"1..6 segments: converged gpu {cg.mean():.3f} oracle {co.mean():.3f}")
    assert abs(cg.mean() - co.mean()) <= 0.08
    T = PA.Task(True)
    rep = PA.compare(T, insts, idx, seqs, lens, 15 * lens, g, ref, rtr)
    flags = PA.flag_disagreements(g, ref)
    remaining = PA.flags_after_refinement(flags, g, ref, *_bim_reruns(P, insts, seqs, idx, lens))
    # on these long orders FP32 converges a little less often than FP64
    # (about 59 % against 62 % at t_exp): up to 2 % of the orders may stay
    # unconverged on the GPU at t_ref where the oracle converged (listed)
    print(f"bimanual 1-6 segments: remaining after t_ref {remaining}")
    assert len(remaining) <= max(3, 2 * len(seqs) // 100), remaining
    _bim_asserts(rep, flags, len(seqs), "bimanual 1-6 segments")
    assert not PA.certify_different(T, insts, idx, seqs, lens, 15 * lens, g, rep)


def test_full_size_launch_sampled(P):
    # the bench's bimanual launch as timed: 512 random orders of 1..6
    # segments on each of 8 instances (4,096 TOs, N up to 90) in one launch;
    # 64 seeded samples of its outputs against the oracle's solves of the
    # same orders, on the bar of the tests above
    insts = [W.bimanual_instance(s) for s in range(8)]
    rng = np.random.default_rng(11)
    seqs, idx = [], []
    for i in range(8):
        for _ in range(512):
            L = int(rng.integers(1, 7))
            seqs.append(tuple(int(m) for m in rng.integers(0, 507, L)))
            idx.append(i)
    n = len(seqs)
    idx = np.array(idx, np.int32)
    g = _ev(P, insts, seqs, idx)
    conv = (g["status"] == 0) & (g["viol"] <= 1e-5)
    print(f"full launch: {int(conv.sum())} of {n} converged ({conv.mean():.3f})")
    picks = np.sort(np.random.default_rng(5).choice(n, 64, replace=False))
    ss = [seqs[t] for t in picks]
    si = idx[picks]
    sl = np.array([len(q) for q in ss], np.int32)
    gs = {k: (v[picks] if isinstance(v, np.ndarray) and v.shape[:1] == (n,) else v) for k, v in g.items()}
    gs["traj_nmax"] = 90
    ref, rtr, _ = oracle.bim_solve_batch_ex(insts, si, ss, sl, opts=_opts())
    T = PA.Task(True)
    rep = PA.compare(T, insts, si, ss, sl, 15 * sl, gs, ref, rtr)
    flags = PA.flag_disagreements(gs, ref)
    remaining = PA.flags_after_refinement(flags, gs, ref, *_bim_reruns(P, insts, ss, si, sl))
    _bim_asserts(rep, flags, len(ss), "bimanual full launch, sampled", remaining)
    assert not PA.certify_different(T, insts, si, ss, sl, 15 * sl, gs, rep)
