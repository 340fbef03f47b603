"""The native tree search of include/comet_mcts.h against the oracle's MCTS
(Sec. IV-A, IV-B): given the same evaluation results the two must ask for
the same pools, order for order, grow trees of the same size and rank the
evaluated orders the same way.  Host code only -- no GPU needed."""
import ctypes

import numpy as np
import pytest

import paper_2609_21803_gb300 as P
import workloads as W
import oracle
from oracle import mcts as T
from oracle import search as S


@pytest.fixture(scope="module")
def lib():
    from paper_2609_21803_gb300 import build as B
    B.build()
    return P.lib()


def records_to_orders(rec):
    return [tuple(int(m) for m in r["modes"][: r["len"]]) for r in rec]


def synthetic(n_modes):
    """A deterministic landscape over codes: float32 costs with ties, about a
    third of the orders infeasible."""
    def f(order):
        code = S.encode(order, n_modes)
        h = (code * 0x9E3779B1) & 0xFFFFFFFF
        cost = np.float32(1.0 + (h % 997) / 64.0)
        viol = np.float32(1e-3 if (h >> 11) % 3 == 0 else 2e-6)
        return cost, viol
    return f


def drive(native, ref, f, pool, instance=0):
    asks = 0
    while True:
        rec = native.ask(pool, instance)
        got = records_to_orders(rec)
        want = ref.ask(pool)
        assert got == want, f"ask {asks}"
        assert all(int(r["instance"]) == instance for r in rec)
        if not want:
            break
        cv = [f(o) for o in want]
        cost = np.array([c for c, _ in cv], np.float32)
        viol = np.array([v for _, v in cv], np.float32)
        native.tell(cost, viol)
        ref.tell([float(c) for c in cost], [float(v) for v in viol])
        st = native.stats()
        assert st["evaluations"] == ref.issued and st["tree_nodes"] == ref.nodes
        assert st["best"] == ref.best and st["pending"] == 0
        asks += 1
    return asks


CASES = [
    dict(n_modes=3, l_max=3, pool=1),
    dict(n_modes=3, l_max=3, pool=5, seed=7),
    dict(n_modes=12, l_max=4, pool=64, max_evals=700, seed=3),
    dict(n_modes=13, l_max=6, pool=16, grammar=1, seed=11),
    dict(n_modes=40, l_max=5, pool=128, max_evals=1000, reward=1, c_uct=1.3, seed=5),
    dict(n_modes=507, l_max=3, pool=256, max_evals=3000, reward=1, seed=2),
]


@pytest.mark.parametrize("case", CASES)
def test_native_search_matches_oracle(lib, case):
    case = dict(case)
    pool = case.pop("pool")
    native = P.Mcts(**case)
    ref = T.Mcts(**case)
    f = synthetic(case["n_modes"])
    asks = drive(native, ref, f, pool)
    assert asks >= 1
    st = native.stats()
    assert st["exhausted"] == ref.root.exhausted
    codes, merits = native.best(40)
    assert [int(c) for c in codes] == ref.best_orders(40)
    native.close()


def test_native_search_on_oracle_solves(lib):
    # real values: every order of two segments on a 2-segment pushing
    # instance solved by the FP64 oracle, rounded to FP32 as the evaluator
    # returns them
    inst = W.push_l2_instance(1)
    every = [(m,) for m in range(12)] + [(a, b) for a in range(12) for b in range(12)]
    modes, lens = W.pad_sequences(every, 2)
    res, _ = oracle.solve_batch([inst], np.zeros(len(every), np.int32), modes, lens)
    table = {o: (np.float32(res["cost"][i]), np.float32(res["viol"][i])) for i, o in enumerate(every)}
    for pool, seed in ((16, 0), (3, 9)):
        native = P.Mcts(n_modes=12, l_max=2, seed=seed)
        ref = T.Mcts(n_modes=12, l_max=2, seed=seed)
        drive(native, ref, lambda o: table[o], pool)
        assert native.stats()["evaluations"] == 156 and native.stats()["exhausted"]
        codes, _ = native.best(8)
        assert [int(c) for c in codes] == ref.best_orders(8)
        # the ranking is Eq. search_merit over the enumeration
        m = [S.merit(float(table[o][0]), float(table[o][1])) for o in every]
        order = sorted(range(len(every)), key=lambda i: (m[i], S.encode(every[i], 12)))
        assert [S.decode(int(c), 12) for c in codes] == [every[i] for i in order[:8]]
        native.close()


def test_struct_layouts():
    assert ctypes.sizeof(P.MctsOpts) == 64
    assert ctypes.sizeof(P.MctsStats) == 40


def test_defaults_and_errors(lib):
    o = P.comet_mcts_default_opts()
    assert (o.n_modes, o.l_max, o.grammar, o.reward, o.max_evals, o.c_uct, o.eps_feas, o.merit_mu, o.max_ms) == \
        (12, 4, 0, 0, 0, 0.8, 1e-5, 100.0, 0.0)
    for bad in (dict(grammar=1), dict(l_max=17), dict(l_max=0), dict(n_modes=507, l_max=7), dict(reward=2),
                dict(c_uct=-1.0), dict(max_evals=-1), dict(n_modes=0), dict(n_modes=65536, l_max=1),
                dict(max_ms=-1.0), dict(max_ms=float("inf"))):
        with pytest.raises(P.CometError):
            P.Mcts(**bad)
    t = P.Mcts(n_modes=3, l_max=2)
    rec = t.ask(4)
    assert len(rec) == 4
    with pytest.raises(P.CometError):
        t.ask(4)                      # the pool was not told
    with pytest.raises(P.CometError):
        t.tell(np.ones(3), np.zeros(3))  # wrong size
    assert t.stats()["pending"] == 4
    t.tell(np.ones(4), np.zeros(4))
    assert t.stats()["evaluations"] == 4
    with pytest.raises(P.CometError):
        t.ask(0)
    # non-finite results are infeasible and rank last
    t.ask(2)
    t.tell(np.array([np.nan, 0.5], np.float32), np.array([0.0, np.inf], np.float32))
    codes, merits = t.best(6)
    assert np.isinf(merits[-2:]).all() and np.isfinite(merits[:-2]).all()
    t.close()


def test_plan_mcts_rejects_bad_arguments_before_any_gpu_work(lib):
    # validated on the host: no problem, no options or an empty pool
    with pytest.raises(P.CometError):
        P.comet_plan_mcts(None, 0, dict(seed=1), 16)
    r = P.PlanResult()
    o = P.comet_mcts_default_opts()
    assert lib.comet_plan_mcts(None, 0, ctypes.byref(o), 16, None, ctypes.byref(r), None) == 1
    assert lib.comet_plan_mcts(None, 0, None, 16, None, ctypes.byref(r), None) == 1
    t = P.Mcts(n_modes=3, l_max=2)
    codes, merits = t.best(0)
    assert len(codes) == 0 and len(merits) == 0
    t.close()
