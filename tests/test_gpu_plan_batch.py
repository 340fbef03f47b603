"""The batched planner (Algorithm 1 for many instances at once): each round
expands every instance's frontier and evaluates all next batches in one
persistent launch.  Every TO is solved by the same arithmetic whatever else
shares its launch, so each instance's plan must equal, bit for bit, the plan
of the single-instance planner on the same seeds and options."""
import numpy as np
import pytest

import workloads as W

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


def _seeds(inst):
    one = [(m,) for m in range(12)]
    two = [(a, b) for a in range(12) for b in range(12)] if inst["max_segments"] >= 2 else []
    return one + two[::5]


@pytest.mark.parametrize("use_graph", [1, 0])
def test_batched_plans_equal_single_instance_plans(P, use_graph):
    insts = [W.push_mixed_instance(s) for s in range(6)]
    prob = P.Problem(insts)
    opts = dict(k=16, batch=256, rounds=3, k_ref=8, ref_iters=300, use_graph=use_graph)
    seeds = [_seeds(i) for i in insts]
    got = P.comet_plan_batch(prob.handle, list(range(6)), seeds, opts)
    assert len(got) == 6
    for i in range(6):
        want = P.comet_plan(prob.handle, i, P.pack_mode_seqs(seeds[i], np.full(len(seeds[i]), i, np.int32)),
                            len(seeds[i]), opts)
        g = got[i]
        assert g["evaluations"] == want["evaluations"], i
        assert g["best"] == want["best"] and g["best_status"] == want["best_status"], i
        if want["best_status"] == 0:
            assert g["best_cost"] == want["best_cost"] and g["best_viol"] == want["best_viol"], i
        assert len(g["best"]) <= insts[i]["max_segments"]
    prob.close()


def test_batched_planner_repeated_instance_and_bad_arguments(P):
    # the same instance twice in one batch: two independent frontiers, same plan
    inst = W.push_l4_instance(7)
    prob = P.Problem([inst])
    s = _seeds(inst)
    opts = dict(k=8, batch=128, rounds=2, k_ref=4, ref_iters=300)
    a, b = P.comet_plan_batch(prob.handle, [0, 0], [s, s], opts)
    assert a == b
    # an empty seed slice or an instance out of range is rejected
    with pytest.raises(P.CometError):
        P.comet_plan_batch(prob.handle, [0, 0], [s, []], opts)
    with pytest.raises(P.CometError):
        P.comet_plan_batch(prob.handle, [1], [s], opts)
    prob.close()
