"""The MCTS comparison policy (Sec. IV-A) on the GPU evaluator: the native
search driven with the evaluator's results asks for the same pools as the
oracle's MCTS given those results; the planner comet_plan_mcts evaluates the
whole order space when the budget allows and then returns the enumeration's
answer, and it keeps its evaluation budget."""
import numpy as np
import pytest

import workloads as W
from oracle import mcts as T
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


def _eval(P, prob, recs):
    d = torch.from_numpy(np.ascontiguousarray(recs).view(np.uint8).reshape(len(recs), P.MODE_SEQ_BYTES)).cuda()
    r = prob.eval(d)
    torch.cuda.synchronize()
    return r["cost"].cpu().numpy(), r["viol"].cpu().numpy()


def test_native_search_on_gpu_results_matches_oracle(P):
    prob = P.Problem([W.push_l4_instance(2)])
    native = P.Mcts(n_modes=12, l_max=4, seed=17, max_evals=600)
    ref = T.Mcts(n_modes=12, l_max=4, seed=17, max_evals=600)
    pools = 0
    while True:
        rec = native.ask(96)
        orders = [tuple(int(m) for m in r["modes"][: r["len"]]) for r in rec]
        assert orders == ref.ask(96)
        if not orders:
            break
        cost, viol = _eval(P, prob, rec)
        native.tell(cost, viol)
        ref.tell([float(c) for c in cost], [float(v) for v in viol])
        pools += 1
    assert native.stats()["evaluations"] == ref.issued == 600 and pools >= 600 // 96
    codes, _ = native.best(32)
    assert [int(c) for c in codes] == ref.best_orders(32)
    native.close()
    prob.close()


def test_unbounded_plan_recovers_enumeration(P):
    # the search claims every order of at most two segments (156) and, with
    # K_ref covering them all, refines the same set as enumeration does
    for seed in (0, 3):
        inst = W.push_l2_instance(seed)
        prob = P.Problem([inst])
        r = P.comet_plan_mcts(prob.handle, 0, dict(seed=seed), 32, dict(k_ref=156, ref_iters=600))
        assert r["evaluations"] == 156 and r["rounds_run"] >= 156 // 32
        every = [(m,) for m in range(12)] + [(a, b) for a in range(12) for b in range(12)]
        e = P.comet_plan(prob.handle, 0, P.pack_mode_seqs(every), 156, dict(rounds=0, k_ref=156, ref_iters=600))
        assert r["best"] == e["best"] and r["best_cost"] == e["best_cost"]
        assert r["best_status"] == 0 and r["explore_ms"] > 0
        prob.close()


def test_grammar_plan_and_budget(P):
    # the pushing grammar: all 57 admissible orders of at most 4 segments
    inst = dict(W.push_grammar_instance(3), max_segments=4, knots_per_segment=6)
    prob = P.Problem([inst])
    r = P.comet_plan_mcts(prob.handle, 0, dict(grammar=1, seed=4), 16, dict(k_ref=57, ref_iters=600))
    assert r["evaluations"] == 57 and r["best"][0] == 12
    every = W.admissible_push_orders(4)
    e = P.comet_plan(prob.handle, 0, P.pack_mode_seqs(every), 57, dict(rounds=0, k_ref=57, ref_iters=600))
    assert r["best"] == e["best"] and r["best_cost"] == e["best_cost"]
    prob.close()
    # an evaluation budget on the 4-segment space (22,620 orders)
    prob = P.Problem([W.push_l4_instance(5)])
    r = P.comet_plan_mcts(prob.handle, 0, dict(max_evals=300, seed=1), 64, dict(k_ref=16, ref_iters=600))
    assert r["evaluations"] == 300 and r["rounds_run"] == 5
    assert r["best_status"] in (0, 1, 2) and np.isfinite(r["best_cost"])
    prob.close()
    # an unbounded search over 12^7 orders is rejected before any work
    prob = P.Problem([dict(W.push_l4_instance(5), max_segments=7)])
    with pytest.raises(P.CometError):
        P.comet_plan_mcts(prob.handle, 0, dict(seed=1), 64)
    prob.close()
