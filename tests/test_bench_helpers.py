"""Host logic of bench.py that needs no GPU: uniform sampling without
replacement as the first distinct orders of the sampler's stream, and the
MCTS comparison leg's bookkeeping driven by a stand-in library."""
import types

import numpy as np

import bench
import paper_2609_21803_gb300 as P
from oracle import search as S


def test_first_distinct_is_the_stream_without_repeats():
    stream = S.sample_orders(7, 0, 2000, 13, 8, grammar=1)
    recs = P.pack_mode_seqs(stream)
    want = list(dict.fromkeys(stream))
    for k in (1, 100, len(want), len(want) + 50):
        got = [tuple(int(m) for m in r["modes"][: r["len"]]) for r in bench.first_distinct(recs, 13, k)]
        assert got == want[:k]
    # a uniform sample without replacement: every admissible order of at most
    # 3 segments is equally likely to come first
    counts = {}
    for seed in range(3000):
        first = S.sample_orders(seed, 0, 1, 13, 3, grammar=1)[0]
        counts[first] = counts.get(first, 0) + 1
    assert len(counts) == len(S.admissible_orders(3))
    expect = 3000 / len(counts)
    assert max(counts.values()) < 2.0 * expect and min(counts.values()) > 0.3 * expect


def test_mcts_leg_bookkeeping_with_a_stand_in_library():
    calls = []

    class Prob:
        def __init__(self, insts):
            self.handle = len(calls) + 1

        def close(self):
            pass

    def plan(h, i, seqs, n, opts):
        rounds = opts.get("rounds", 0)
        return {"best": (12,), "best_cost": 1.0, "best_viol": 0.0, "best_status": 0, "rounds_run": rounds,
                "evaluations": 3000 if rounds else n, "explore_ms": 10.0, "refine_ms": 5.0}

    def plan_mcts(h, i, mo, pool, opts):
        calls.append((mo["max_evals"], pool, mo["grammar"], opts["k_ref"]))
        ok = pool != 64
        return {"best": (12,), "best_cost": 1.0 if ok else 1.5, "best_viol": 0.0, "best_status": 0,
                "rounds_run": -(-3000 // pool), "evaluations": 3000, "explore_ms": 20.0, "refine_ms": 5.0}

    stub = types.SimpleNamespace(Problem=Prob, comet_plan=plan, comet_plan_mcts=plan_mcts, GRAMMAR_PUSH=1,
                                 pack_mode_seqs=P.pack_mode_seqs)
    out = bench.mcts_times(stub, n_inst=2)
    # every pool size runs on every instance at the expansion's evaluation count
    assert sorted(set(calls)) == [(3000, 64, 1, 256), (3000, 256, 1, 256), (3000, 1024, 1, 256)]
    assert len(calls) == 6
    assert out["pool_1024"]["recovered"] == 2 and out["pool_64"]["recovered"] == 0
    assert out["pool_256"]["pools"] == 12.0 and out["expansion_recovered"] == 2
