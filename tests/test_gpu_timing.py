"""GPU timing optimisation (comet_eval_modes_timed, through the C ABI)
against the timing oracle (oracle/timing.py).  Paper: Sec. III-C (with
timing optimised, the interval durations join the controls), Sec. IV-A (an
optimised time step under the benchmark's duration bound).

Workload: 33 orders, 8 two-segment orders (every 18th of the 144) on each
of the push_l2 instances 0..3 plus the straight push, N = 16, under a
duration bound that leaves room (h in [0.05, 0.2], T = 2 s) and one that
binds (h in [0.02, 0.3], T = 1.2 s against the fixed step's 1.6 s).

How the bar is read.  With free durations a TO's solution set is often
not a point: intervals of equal cost can trade duration, so two valid
answers can sit far apart in state and duration at the same cost.  What is
unique, and compared, is the cost of the exact local solution, the
feasibility flags and the certificates:
  * first iterate (one step from the same cold start, before any discrete
    decision): the iterate within 1e-4 of the oracle's with the bound
    slack; within 2e-3 when it binds.  There the step's linear system is
    ill-conditioned along the duration chain (condition number about 1e6,
    the damping 1e-4 against beta = 100): an FP32 solve of that system
    moves the durations by a few 1e-3 from the FP64 one;
  * later iterates are not compared: the step's size along those weakly
    damped directions makes the trial-step choice flip between 2^-5 and
    2^-6 under FP32 rounding, after which the two runs follow different
    paths;
  * converged answers (budget 1500): every TO the oracle converges also
    converges on the GPU, after a second budget from the GPU's own answer
    where the first one ran out, except at most two on which the oracle
    itself needed more than half the budget: there the flag sits at the
    edge of the budget (order (0, 0) on instance 1 under the binding bound
    converges in the oracle on one host and stays at the budget, infeasible
    at the largest penalty, on another host and on the GPU); each converged
    GPU answer is certified in FP64 by
    the oracle's rows (physical violation <= eps_feas) and lies within
    1e-4 |J*| + sum_r |lam*_r| |c_r(z_gpu)| of the exact local solution J*
    reached by the oracle's tight polish of it (the relative bar plus the
    first-order cost of the residual infeasibility the stop test allows);
    where that polish coincides with the polish of the oracle's own answer
    (same local solution, costs within 1e-8), the GPU's cost is therefore
    within the bar of the oracle's exact solution; the other TOs are listed
    with both exact costs.
"""
import numpy as np
import pytest

import _timing_jobs as TJ
import workloads as W
from oracle import timing as TM

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SLACK = dict(h_min=0.05, h_max=0.2, T=2.0)
BIND = dict(h_min=0.02, h_max=0.3, T=1.2)


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


def workload():
    orders = [tuple(int(v) for v in q) for q in W.all_sequences(12, 2)[::18]]
    seqs, idx = [], []
    for i in range(4):
        for q in orders:
            seqs.append(q)
            idx.append(i)
    seqs.append((0, 0))
    idx.append(4)
    return seqs, np.array(idx, np.int32)


def gpu_timed(P, seqs, idx, timing, max_iters, warm=None, insts=None):
    insts = insts or [TJ.instance(i) for i in range(5)]
    prob = P.Problem(insts)
    n = len(seqs)
    d = torch.from_numpy(P.pack_mode_seqs(seqs, idx).view(np.uint8).reshape(n, P.MODE_SEQ_BYTES)).cuda()
    Nmax = max(int(x["knots_per_segment"]) * int(x["max_segments"]) for x in insts)
    stride = 9 * Nmax + 5
    cost = torch.empty(n, dtype=torch.float32, device="cuda")
    status = torch.empty(n, dtype=torch.int32, device="cuda")
    traj = torch.zeros((n, stride), dtype=torch.float32, device="cuda")
    w = None if warm is None else torch.from_numpy(np.ascontiguousarray(warm, np.float32)).cuda()
    tm = dict(h_min=timing["h_min"], h_max=timing["h_max"], T_max=timing["T"])
    P.comet_eval_modes_timed(prob.handle, tm, d, n, w, max_iters, cost, traj, status)
    viol = torch.empty(n, dtype=torch.float32, device="cuda")
    iters = torch.empty(n, dtype=torch.int32, device="cuda")
    P.comet_eval_stats(prob.handle, viol, None, iters, None)
    torch.cuda.synchronize()
    out = dict(cost=cost.cpu().numpy(), status=status.cpu().numpy(), traj=traj.cpu().numpy(),
               viol=viol.cpu().numpy(), iters=iters.cpu().numpy())
    prob.close()
    return out


@pytest.mark.parametrize("timing,tol", [(SLACK, 1e-4), (BIND, 2e-3)], ids=["slack", "binding"])
def test_first_iterate_matches_the_oracle(P, timing, tol):
    seqs, idx = workload()
    g = gpu_timed(P, seqs, idx, timing, 1)
    ref = TJ.run([(int(i), q, timing, 1, None, None) for q, i in zip(seqs, idx)])
    worst = 0.0
    for t, (z, _, r) in enumerate(ref):
        zg = TJ.to_interleaved(g["traj"][t])
        worst = max(worst, np.abs(zg - z).max() / max(1.0, np.abs(z).max()))
        assert int(g["status"][t]) == r["status"]
        assert g["cost"][t] == pytest.approx(r["cost"], rel=1e-4)
    print(f"first iterate: max scaled difference {worst:.2e} (bar {tol:.0e})")
    assert worst <= tol


def test_straight_push_with_free_durations_closed_form(P):
    # J = W R d^2 / (R + W kappa^2 sum h_k^2) falls in every h_k: with room
    # in the bound every h_k sits at h_max
    d, N, hmax = 0.1, TJ.N, 0.15
    inst = W.push_l2_straight(d)
    Wt, R = inst["w_terminal"], inst["w_control"]
    timing = dict(h_min=0.05, h_max=hmax, T=3.0)
    g = gpu_timed(P, [(0, 0)], np.zeros(1, np.int32), timing, 1500, insts=[inst])
    assert int(g["status"][0]) == TM.CONVERGED
    z = TJ.to_interleaved(g["traj"][0])
    L = TM.Layout(N, timing)
    h = np.array([z[L.u(k) + 3] for k in range(N)])
    np.testing.assert_allclose(h, hmax, atol=1e-5)
    assert z[L.x(N) + 4] == pytest.approx(N * hmax, rel=1e-5)
    J = Wt * R * d * d / (R + Wt * N * hmax ** 2)
    assert g["cost"][0] == pytest.approx(J, rel=1e-4)
    fn = np.array([z[L.u(k)] for k in range(N)])
    np.testing.assert_allclose(fn, Wt * hmax * d / (Wt * N * hmax ** 2 + R), rtol=1e-3)


@pytest.mark.parametrize("timing", [SLACK, BIND], ids=["slack", "binding"])
def test_converged_answers_against_the_exact_local_solutions(P, timing):
    seqs, idx = workload()
    _converged_parity(P, seqs, idx, timing, [TJ.instance(i) for i in range(5)])


def test_free_motion_orders(P):
    # the free-motion mode (12) inside timed orders: the pusher off the
    # slider, the slider at rest, the offset moving at the pusher's rate for
    # h_k; first iterate and converged answers as above
    orders = [(12, 0), (0, 12), (12, 3), (7, 12), (12, 12), (12, 9)]
    seqs = [q for _ in range(4) for q in orders]
    idx = np.repeat(np.arange(4, dtype=np.int32), len(orders))
    insts = [dict(TJ.instance(i), n_modes=13) for i in range(4)]
    g = gpu_timed(P, seqs, idx, SLACK, 1, insts=insts)
    ref = TJ.run([(int(i), q, SLACK, 1, None, None) for q, i in zip(seqs, idx)])
    worst = max(np.abs(TJ.to_interleaved(g["traj"][t]) - z).max() / max(1.0, np.abs(z).max())
                for t, (z, _, _) in enumerate(ref))
    print(f"free motion, first iterate: max scaled difference {worst:.2e}")
    assert worst <= 1e-4
    _converged_parity(P, seqs, idx, SLACK, insts)


def _converged_parity(P, seqs, idx, timing, insts):
    n = len(seqs)
    g = gpu_timed(P, seqs, idx, timing, 1500, insts=insts)
    ref = TJ.run([(int(i), q, timing, 1500, None, None) for q, i in zip(seqs, idx)])
    conv_g = g["status"] == TM.CONVERGED
    conv_o = np.array([r["status"] == TM.CONVERGED for _, _, r in ref])
    # flags: a TO the oracle converges that the GPU leaves at the budget is
    # re-run from the GPU's own answer with a second budget (the oracle's
    # flag on such TOs is itself at the edge of the budget: it changes with
    # the host's floating-point library); after it none may remain
    lag = np.nonzero(conv_o & ~conv_g)[0]
    if len(lag):
        r2 = gpu_timed(P, [seqs[t] for t in lag], idx[lag], timing, 1500, warm=g["traj"][lag], insts=insts)
        for j, t in enumerate(lag):
            for k in ("cost", "status", "traj", "viol", "iters"):
                g[k][t] = r2[k][j]
        print(f"re-run from the GPU's answer: TOs {list(lag)} -> status {list(r2['status'])}")
        conv_g = g["status"] == TM.CONVERGED
    lag = np.nonzero(conv_o & ~conv_g)[0]
    for t in lag:
        print(f"  TO {t} {seqs[t]}: oracle converged in {ref[t][2]['iters']} iterations, GPU still at the budget "
              f"(v_hat {float(g['viol'][t]):.2e})")
    # what may remain: the FP32 and FP64 paths part on a few orders of this
    # non-convex problem, whatever the elimination order: over the 576
    # two-segment orders of instances 0..3 the oracle converged within 750
    # iterations on 7 (bound with room) and 10 (binding) orders that the GPU
    # left at the budget, and the GPU converged on 7 and 26 that the oracle
    # did not.  Two of the sample's orders at most, each listed above
    assert len(lag) <= 2, list(lag)
    zg = [TJ.to_interleaved(g["traj"][t]) for t in range(n)]
    sel = [t for t in range(n) if conv_g[t]]
    pol_g = TJ.run([(int(idx[t]), seqs[t], timing, None, zg[t], TJ.POLISH) for t in sel])
    sel_o = [t for t in sel if conv_o[t]]
    pol_o = dict(zip(sel_o, TJ.run([(int(idx[t]), seqs[t], timing, None, ref[t][0], TJ.POLISH) for t in sel_o])))
    worst, same, diff, off = 0.0, 0, [], []
    for t, (zs, lam, rs) in zip(sel, pol_g):
        Pb = TM.Problem(TJ.instance(int(idx[t])), seqs[t], TJ.N, timing)
        z = zg[t]
        # FP64 certificate of the GPU answer by the oracle's rows
        _, _, m = TM.measures(Pb, z, np.zeros(Pb.L.nl), 1.0)
        assert m["vphys"] <= 1e-5, (t, m["vphys"])
        # the kernel's own FP64 certificate (of its compensated iterate) agrees
        # up to the rounding of the FP32 output
        assert abs(float(g["viol"][t]) - m["vphys"]) <= 2e-7, (t, float(g["viol"][t]), m["vphys"])
        J = Pb.cost(z)
        assert float(g["cost"][t]) == pytest.approx(J, rel=1e-6)
        # the exact local solution of the GPU answer's basin
        if rs["status"] != TM.CONVERGED:
            off.append((t, seqs[t], J, None))
            continue
        c, _, _, mask = TM.all_rows(Pb, z)
        bar = 1e-4 * abs(rs["cost"]) + float(np.sum(np.abs(lam) * np.abs(c * mask)))
        if abs(J - rs["cost"]) > bar:
            off.append((t, seqs[t], J, rs["cost"]))
            continue
        worst = max(worst, abs(J - rs["cost"]) / bar)
        if t in pol_o:
            ro = pol_o[t][2]
            if ro["status"] == TM.CONVERGED and abs(ro["cost"] - rs["cost"]) <= 1e-8 * abs(ro["cost"]):
                same += 1
            else:
                diff.append((t, seqs[t], rs["cost"], ro["cost"]))
    print(f"{len(sel)} converged on the GPU ({int(conv_o.sum())} in the oracle); worst cost / bar {worst:.2f}; "
          f"same local solution {same}, different {len(diff)}")
    for t, q, jg, jo in diff:
        print(f"  TO {t} {q}: exact cost of the GPU's basin {jg:.6g}, of the oracle's {jo:.6g} "
              f"({'GPU lower' if jg < jo else 'oracle lower'})")
    for t, q, J, js in off:
        print(f"  TO {t} {q}: GPU answer at cost {J:.6g} is not within the bar of a local solution "
              f"({'the polish from it does not converge' if js is None else f'the polish from it reaches {js:.6g}'})")
    # a stop at a point that is not a local minimum (a saddle or a flat
    # stretch of free durations, which the polish leaves for a lower basin):
    # over the 576 two-segment orders of instances 0..3 about 1 % of the
    # converged answers of either elimination order (sequential sweep 7 and
    # 7 polishes that did not converge of 1,065; the lane-parallel
    # elimination 6 and 7 of 1,070); one of the sample's answers at most
    assert len(off) <= 1, off
    # the two solvers often end in different local solutions of these flat,
    # non-convex problems; the GPU's are not worse: on at least half of the
    # orders both converge, the GPU's basin is the oracle's or a lower one
    gpu_lower = sum(1 for _, _, jg, jo in diff if jg < jo)
    assert same + gpu_lower >= len(sel_o) // 2, (same, gpu_lower, len(sel_o))


def test_full_size_launch_sampled(P):
    # the bench's 4-segment launch as timed: every order of push_l4 instance
    # 3 (20,736 TOs at N = 80) in one launch under its binding bound (h in
    # [dt/5, 3 dt], T = 3/4 of the fixed schedule); 12 sampled outputs
    # against the oracle's solves of the same orders, with the bars of the
    # samples above (one listed flag lag, one listed answer outside the
    # cost bar at most)
    inst = W.push_l4_instance(3)
    orders = [tuple(int(v) for v in q) for q in W.all_sequences(12, 4)]
    n, dt = len(orders), inst["dt"]
    N = int(inst["knots_per_segment"]) * 4
    tm = dict(h_min=0.2 * dt, h_max=3.0 * dt, T=0.75 * N * dt)
    g = gpu_timed(P, orders, np.zeros(n, np.int32), tm, 1500, insts=[inst])
    conv_all = (g["status"] == TM.CONVERGED) & (g["viol"] <= 1e-5)
    print(f"full launch: {int(conv_all.sum())} of {n} converged ({conv_all.mean():.3f})")
    assert conv_all.mean() >= 0.9
    picks = np.random.default_rng(11).choice(n, 12, replace=False)
    ref = TJ.run([(("l4", 3), orders[t], tm, 1500, None, None) for t in picks])
    conv_o = np.array([r["status"] == TM.CONVERGED for _, _, r in ref])
    conv_g = np.array([bool(g["status"][t] == TM.CONVERGED) for t in picks])
    lag = [int(picks[j]) for j in np.nonzero(conv_o & ~conv_g)[0]]
    print(f"sample: oracle converged {int(conv_o.sum())}, GPU {int(conv_g.sum())}, lagging {lag}")
    assert len(lag) <= 1, lag
    sel = [j for j in range(len(picks)) if conv_g[j]]
    zg = {j: TJ.to_interleaved(g["traj"][picks[j]], Nmax=N) for j in sel}
    pol = TJ.run([(("l4", 3), orders[picks[j]], tm, None, zg[j], TJ.POLISH) for j in sel])
    off, worst = [], 0.0
    for j, (zs, lam, rs) in zip(sel, pol):
        t = int(picks[j])
        Pb = TM.Problem(inst, orders[t], N, tm)
        _, _, m = TM.measures(Pb, zg[j], np.zeros(Pb.L.nl), 1.0)
        assert m["vphys"] <= 1e-5, (t, m["vphys"])
        # the kernel certifies its compensated iterate; the oracle's rows
        # see the FP32 output, whose rounding moves a row by up to 2^-24
        # times the magnitudes it differences (tau reaches 6 s here)
        rnd = 2.0 ** -23 * float(np.abs(zg[j]).max()) + 1e-7
        assert abs(float(g["viol"][t]) - m["vphys"]) <= rnd, (t, float(g["viol"][t]), m["vphys"], rnd)
        J = Pb.cost(zg[j])
        assert float(g["cost"][t]) == pytest.approx(J, rel=1e-6)
        if rs["status"] != TM.CONVERGED:
            off.append((t, orders[t], J, None))
            continue
        c, _, _, mask = TM.all_rows(Pb, zg[j])
        bar = 1e-4 * abs(rs["cost"]) + float(np.sum(np.abs(lam) * np.abs(c * mask)))
        if abs(J - rs["cost"]) > bar:
            off.append((t, orders[t], J, rs["cost"]))
            continue
        worst = max(worst, abs(J - rs["cost"]) / bar)
    print(f"{len(sel)} converged answers certified in FP64; worst cost / bar {worst:.2f}; outside the bar {off}")
    assert len(off) <= 1, off


def test_timed_entry_rejects_bad_arguments(P):
    prob = P.Problem([TJ.instance(0)])
    d = torch.from_numpy(P.pack_mode_seqs([(0, 3)]).view(np.uint8).reshape(1, P.MODE_SEQ_BYTES)).cuda()
    cost = torch.empty(1, dtype=torch.float32, device="cuda")
    status = torch.empty(1, dtype=torch.int32, device="cuda")
    with pytest.raises(P.CometError):
        P.comet_eval_modes_timed(prob.handle, dict(h_min=0.2, h_max=0.1, T_max=1.0), d, 1, None, 10, cost, None,
                                 status)
    with pytest.raises(P.CometError):
        P.comet_eval_modes_timed(prob.handle, dict(h_min=0.05, h_max=0.2, T_max=1.0), d, 1, None, 10,
                                 np.zeros(1, np.float32), None, np.zeros(1, np.int32))
    P.comet_eval_modes_timed(prob.handle, dict(h_min=0.05, h_max=0.2, T_max=2.0), d, 0, None, 10, cost, None,
                             status)
    prob.close()
    bim = P.Problem([W.bimanual_instance(0)])
    with pytest.raises(P.CometError):
        P.comet_eval_modes_timed(bim.handle, dict(h_min=0.05, h_max=0.2, T_max=2.0), d, 1, None, 10, cost, None,
                                 status)
    bim.close()
