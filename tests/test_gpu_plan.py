"""The device planner (Algorithm 1): seed batch, expansion rounds replayed
from a CUDA graph, refinement of the K_ref best orders.  Checked against the
same steps driven one call at a time through the C ABI, and against full
enumeration when the budget covers the whole order space."""
import numpy as np
import pytest

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


def _eval(P, prob, seqs, iters=0):
    packed = P.pack_mode_seqs(seqs)
    d = torch.from_numpy(packed.view(np.uint8).reshape(len(seqs), P.MODE_SEQ_BYTES)).cuda()
    r = prob.eval(d, max_iters=iters)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def test_graph_and_stepwise_planner_agree(P):
    inst = W.push_l4_instance(7)
    prob = P.Problem([inst])
    seeds = P.pack_mode_seqs([(m,) for m in range(12)] + [(a, b) for a in range(12) for b in range(12)])
    opts = dict(k=16, batch=256, rounds=3, k_ref=8, ref_iters=300, use_graph=1)
    a = P.comet_plan(prob.handle, 0, seeds, len(seeds), opts)
    b = P.comet_plan(prob.handle, 0, seeds, len(seeds), dict(opts, use_graph=0))
    # a round admits at most B unseen orders (fewer when the beam's
    # neighbourhoods run short)
    assert a["evaluations"] == b["evaluations"] <= 156 + 3 * 256
    assert a["best"] == b["best"] and a["best_cost"] == b["best_cost"]
    # the same rounds driven one call at a time through the frontier API
    f = P.comet_frontier_create(prob.handle, 0, 100000, 256, 16)
    frontier = [tuple(int(x) for x in r["modes"][: r["len"]]) for r in seeds]
    for rnd in range(4):                   # seed batch + 3 expansion rounds
        r = _eval(P, prob, frontier)
        P.comet_frontier_add(f, P.pack_mode_seqs(frontier), len(frontier), r["cost"], r["viol"])
        if rnd == 3:
            break
        P.comet_expand(prob.handle, f, 16)
        frontier = P.frontier_next_orders(f, 256)
    n, err = P.comet_frontier_size(f)
    assert n == a["evaluations"] and err == 0
    codes, _m = P.comet_frontier_best(f, 8)
    top = [P.decode_code(int(c)) for c in codes]
    ref = _eval(P, prob, top, iters=300)
    ok = (ref["status"] == 0) & (ref["viol"] <= 1e-5)
    assert ok.any()
    i = int(np.argmin(np.where(ok, ref["cost"], np.inf)))
    assert top[i] == a["best"] and ref["cost"][i] == pytest.approx(a["best_cost"], rel=1e-6)
    P.comet_frontier_destroy(f)
    prob.close()


def test_budget_truncates_and_planner_returns_trajectory(P):
    inst = W.push_l4_instance(8)
    prob = P.Problem([inst])
    seeds = P.pack_mode_seqs([(m,) for m in range(12)])
    traj = np.zeros(prob.stride, np.float32)
    r = P.comet_plan(prob.handle, 0, seeds, 12, dict(k=8, batch=500, rounds=4, k_ref=4, budget=700), out_traj=traj)
    assert r["evaluations"] == 700
    assert r["best_status"] == 0 and r["best_viol"] <= 1e-5
    L = len(r["best"])
    N = inst["knots_per_segment"] * L
    Nm1 = 81
    # the returned trajectory starts at the instance's start pose
    np.testing.assert_allclose([traj[0], traj[Nm1], traj[2 * Nm1]], inst["start"], atol=1e-5)
    assert np.isfinite(traj[: 4 * Nm1]).all() and N <= 80
    prob.close()


def test_unlimited_expansion_recovers_enumeration(P):
    # walking all of V (beam k >= |V|, as Algorithm 1 does) with enough rounds
    # evaluates every order of length <= 2 (156), so the answer equals full
    # enumeration's (Eq. mode_selection) followed by the same refinement
    for seed in (0, 3):
        inst = W.push_l2_instance(seed)
        prob = P.Problem([inst])
        seeds = P.pack_mode_seqs([(m,) for m in range(12)])
        r = P.comet_plan(prob.handle, 0, seeds, 12, dict(k=256, batch=64, rounds=12, k_ref=16, ref_iters=600))
        assert r["evaluations"] == 156
        allseq = [(m,) for m in range(12)] + [(a, b) for a in range(12) for b in range(12)]
        e = _eval(P, prob, allseq)
        merit = e["cost"] + 100.0 * np.maximum(e["viol"] - 1e-5, 0)
        order = sorted(range(156), key=lambda i: (merit[i], S.encode(allseq[i], 12)))[:16]
        top = [allseq[i] for i in order]
        ref = _eval(P, prob, top, iters=600)
        ok = (ref["status"] == 0) & (ref["viol"] <= 1e-5)
        i = int(np.argmin(np.where(ok, ref["cost"], np.inf)))
        assert r["best"] == top[i]
        prob.close()


def test_grammar_plan_recovers_admissible_enumeration(P):
    # the pushing grammar: every admissible order is reached from (free,) by
    # admissible one-edit steps, so walking all of V with enough rounds
    # evaluates all 57 admissible orders of at most 4 segments and returns
    # the enumeration's answer after the same refinement
    inst = dict(W.push_grammar_instance(3), max_segments=4, knots_per_segment=6)
    prob = P.Problem([inst])
    every = W.admissible_push_orders(4)
    assert len(every) == 57
    seeds = P.pack_mode_seqs([(12,)])
    r = P.comet_plan(prob.handle, 0, seeds, 1, dict(k=256, batch=64, rounds=12, k_ref=8, ref_iters=600, grammar=1))
    assert r["evaluations"] == 57
    e = P.comet_plan(prob.handle, 0, P.pack_mode_seqs(every), 57, dict(rounds=0, k_ref=8, ref_iters=600))
    assert r["best"] == e["best"] and r["best_cost"] == e["best_cost"]
    assert r["best"][0] == 12 and r["best_status"] == 0
    # radius 2 reaches the same set in fewer rounds
    r2 = P.comet_plan(prob.handle, 0, seeds, 1, dict(k=256, batch=256, rounds=6, k_ref=8, ref_iters=600,
                                                     grammar=1, radius=2))
    assert r2["evaluations"] == 57 and r2["best"] == e["best"]
    prob.close()
