"""Pins of the MCTS comparison policy of the oracle (Sec. IV-A, IV-B): order
coverage against the enumeration, the evaluation budget, the bookkeeping of
virtual loss and backed-up rewards, the reward definitions, and that UCT
exploits (finds a planted best order far more often than uniform sampling
with the same budget)."""
import math

import numpy as np
import pytest

from oracle import mcts as T
from oracle import search as S


def table_eval(cost_of, viol_of=lambda o: 0.0):
    seen = []

    def evaluate(orders):
        seen.extend(orders)
        return [cost_of(o) for o in orders], [viol_of(o) for o in orders]

    return evaluate, seen


def every_order(n_modes, l_max):
    return [S.unrank_order(i, n_modes, l_max) for i in range(sum(n_modes ** L for L in range(1, l_max + 1)))]


@pytest.mark.parametrize("pool", [1, 5, 64])
def test_unlimited_budget_evaluates_every_order_once(pool):
    ev, seen = table_eval(lambda o: 1.0 + sum(o) + 0.1 * len(o))
    t = T.run(ev, pool, n_modes=3, l_max=3, seed=11)
    assert len(seen) == len(set(seen)) == 3 + 9 + 27
    assert set(seen) == set(every_order(3, 3))
    assert t.root.exhausted and t.issued == 39


def test_grammar_visits_exactly_the_admissible_orders():
    ev, seen = table_eval(lambda o: 1.0 + len(o))
    t = T.run(ev, 16, n_modes=13, l_max=4, grammar=1, seed=5)
    assert sorted(seen) == sorted(S.admissible_orders(4)) and len(seen) == 57
    assert all(S.admissible_push(o) for o in seen)
    # the paper's count of admissible box orders of at most 6 segments
    ev6, seen6 = table_eval(lambda o: 1.0)
    T.run(ev6, 256, n_modes=13, l_max=6, grammar=1, seed=1)
    assert len(set(seen6)) == len(seen6) == 601


@pytest.mark.parametrize("budget,pool", [(50, 8), (37, 64), (1, 3)])
def test_budget_and_pool_bounds(budget, pool):
    sizes = []

    def ev(orders):
        sizes.append(len(orders))
        return [1.0] * len(orders), [0.0] * len(orders)

    t = T.run(ev, pool, n_modes=4, l_max=4, seed=3, max_evals=budget)
    assert sum(sizes) == t.issued == budget
    assert all(1 <= s <= pool for s in sizes)


def _walk(node):
    yield node
    for c in node.children.values():
        yield from _walk(c)


def test_virtual_loss_and_backup_conservation():
    # visits: every attempt creates one node and counts once on each node of
    # its path, so n(X) = 1 + sum n(children) below the root
    rng = np.random.default_rng(0)
    cost = {o: float(rng.uniform(1, 3)) for o in every_order(4, 3)}
    viol = {o: (0.0 if rng.uniform() < 0.7 else 1e-3) for o in cost}
    t = T.Mcts(n_modes=4, l_max=3, seed=9)
    while True:
        pool = t.ask(6)
        if not pool:
            break
        assert len(set(pool)) == len(pool)
        # virtual loss: the waiting paths carry visits, their rewards are not in yet
        pending = sum(len(p) for p in t.waiting.values())
        assert pending >= len(pool)
        t.tell([cost[o] for o in pool], [viol[o] for o in pool])
        assert not t.waiting
    assert t.root.exhausted and t.issued == len(cost)
    assert t.root.n == sum(c.n for c in t.root.children.values()) == t.nodes - 1
    for v in _walk(t.root):
        if v is not t.root:
            assert v.n == 1 + sum(c.n for c in v.children.values())
        assert -1e-12 <= v.w <= v.n + 1e-12
    # rewards: with every order feasible at one cost each reward is 1, so
    # every visit is backed up exactly once: w = n on every node; with every
    # order infeasible nothing is backed up
    for viol_all, expect in ((0.0, "n"), (1.0, "zero")):
        t = T.run(lambda os: ([2.0] * len(os), [viol_all] * len(os)), 5, n_modes=3, l_max=3, seed=4)
        for v in _walk(t.root):
            assert v.w == (v.n if expect == "n" else 0.0)


def test_reward_definitions():
    t = T.Mcts(n_modes=3, l_max=2, reward=T.REWARD_FEASIBLE)
    t.best = 2.0
    assert t.reward(2.0, 0.0) == 1.0 and t.reward(4.0, 0.0) == 0.5
    assert t.reward(1.0, 1e-3) == 0.0 and t.reward(float("nan"), 0.0) == 0.0
    m = T.Mcts(n_modes=3, l_max=2, reward=T.REWARD_MERIT, eps_feas=1e-5, mu=100.0)
    m.best = 2.0
    # M_hat = J_hat + mu max(v_hat - eps, 0) (Eq. search_merit)
    assert m.reward(3.0, 1e-2 + 1e-5) == pytest.approx(2.0 / 4.0)
    assert m.reward(2.0, 0.0) == 1.0


def test_told_rewards_use_the_pool_best():
    # one pool holding the best feasible order: J_best is updated before the
    # backup, so that order's path receives exactly 1 and the others J_best/J
    t = T.Mcts(n_modes=2, l_max=1, seed=0)
    pool = t.ask(8)
    assert sorted(pool) == [(0,), (1,)]
    costs = {(0,): 4.0, (1,): 2.0}
    t.tell([costs[o] for o in pool], [0.0, 0.0])
    # each one-segment child is reached twice (its creation and its "stop"
    # leaf), both paths waiting on the same pool entry
    ch = {c.prefix: c for c in t.root.children.values()}
    assert ch[(1,)].n == ch[(0,)].n == 2
    assert ch[(1,)].w == 2 * 1.0 and ch[(0,)].w == 2 * 0.5
    assert t.root.w == 3.0 and t.best == 2.0


def test_uct_exploits_a_planted_best_order():
    target = (2, 5, 1, 3)

    def cost(o):
        d = sum(1 for i, m in enumerate(o) if i >= len(target) or m != target[i]) + abs(len(o) - len(target))
        return 1.0 + 2.0 * d

    budget, found_mcts = 200, 0
    for seed in range(20):
        ev, seen = table_eval(cost)
        T.run(ev, 8, n_modes=6, l_max=4, seed=seed, max_evals=budget)
        found_mcts += target in seen
    # uniform sampling with the same budget finds it with probability
    # about 200 / 1554 = 0.13 per run
    found_uniform = 0
    for seed in range(20):
        sample = S.sample_orders(seed, 0, budget, 6, 4)
        found_uniform += target in sample
    assert found_mcts >= 14 and found_uniform <= 8 and found_mcts > 2 * found_uniform


def test_seeded_runs_repeat_and_seeds_differ():
    def ev(orders):
        return [1.0 + (S.encode(o, 5) % 7) for o in orders], [0.0] * len(orders)

    a = T.run(ev, 4, n_modes=5, l_max=3, seed=21, max_evals=60)
    b = T.run(ev, 4, n_modes=5, l_max=3, seed=21, max_evals=60)
    c = T.run(ev, 4, n_modes=5, l_max=3, seed=22, max_evals=60)
    assert list(a.results) == list(b.results) and a.best_orders(10) == b.best_orders(10)
    assert list(a.results) != list(c.results)


def test_best_orders_rank_by_merit_then_code():
    t = T.Mcts(n_modes=3, l_max=2, seed=0)
    orders = t.ask(12)
    vals = {o: (1.0, 0.0) if len(o) == 1 else (0.5, 1.0) for o in orders}
    t.tell([vals[o][0] for o in orders], [vals[o][1] for o in orders])
    codes = t.best_orders(3)
    # the one-segment orders (merit 1.0) beat the infeasible ones (merit ~100.5)
    assert [S.decode(c, 3) for c in codes] == [(0,), (1,), (2,)]


@pytest.mark.parametrize("wa,pick", [(0.8, "A"), (0.0, "B"), (1.0, "A")])
def test_uct_selection_textbook_cases(wa, pick):
    # UCT = UCB1 at every node (Kocsis and Szepesvari 2006): mean reward plus
    # c sqrt(ln N / n), c = 0.8 (Sec. IV-A).  Parent visits 10; child A
    # visited once, child B nine times with mean 0.85:
    #   wa = 0.8: A scores 0.8 + 0.8 sqrt(ln 10) = 2.01 > B's 0.85 + 0.8
    #             sqrt(ln 10 / 9) = 1.25 (exploration picks A, pure
    #             exploitation would pick B);
    #   wa = 0.0: A scores 1.21 < 1.25 (the mean decides: B)
    t = T.Mcts(n_modes=2, l_max=2, seed=0, c_uct=0.8)
    A = T.Node((0,), False, t.slots((0,)))
    B = T.Node((1,), False, t.slots((1,)))
    A.n, A.w, B.n, B.w = 1, wa, 9, 9 * 0.85
    t.root.untried, t.root.children, t.root.n = [], {1: A, 2: B}, 10
    t.attempt()
    assert (A.n, B.n) == ((2, 9) if pick == "A" else (1, 10))


def test_uct_ties_go_to_the_lowest_slot():
    t = T.Mcts(n_modes=3, l_max=2, seed=0)
    kids = {}
    for slot, m in ((3, 2), (1, 0), (2, 1)):
        kids[slot] = T.Node((m,), False, t.slots((m,)))
        kids[slot].n, kids[slot].w = 2, 1.0
    t.root.untried, t.root.children, t.root.n = [], kids, 6
    t.attempt()
    assert [kids[s].n for s in (1, 2, 3)] == [3, 2, 2]


def test_policies_on_oracle_solves_order_as_in_the_paper():
    # every order of <= 2 segments on 16 instances solved by the FP64 oracle;
    # each policy searches those results with the same budget, counted by the
    # instances on which it evaluates the enumeration's feasible argmin
    # (Eq. mode_selection).  The paper's ordering: expansion, MCTS, uniform
    import oracle
    import workloads as W
    every = [(m,) for m in range(12)] + [(a, b) for a in range(12) for b in range(12)]
    modes, lens = W.pad_sequences(every, 2)
    found = {"expansion": [0, 0], "mcts": [0, 0], "uniform": [0, 0]}
    for s in range(16):
        res, _ = oracle.solve_batch([W.push_l2_instance(s)], np.zeros(len(every), np.int32), modes, lens)
        tab = {o: (float(np.float32(res["cost"][i])), float(np.float32(res["viol"][i]))) for i, o in enumerate(every)}
        feas = [o for o in every if tab[o][1] <= 1e-5]
        target = min(feas, key=lambda o: (S.merit(*tab[o]), S.encode(o, 12)))
        for j, budget in enumerate((48, 96)):
            V, _ = S.run_expansion(lambda q: [S.merit(*tab[o]) for o in q], [(m,) for m in range(12)], 8, 12, 12,
                                   2, 100, budget=budget)
            found["expansion"][j] += any(seq == target for _, seq in V.values())
            seen = []

            def ev(q):
                seen.extend(q)
                return [tab[o][0] for o in q], [tab[o][1] for o in q]

            T.run(ev, 8, n_modes=12, l_max=2, seed=s, max_evals=budget)
            found["mcts"][j] += target in seen
            first = list(dict.fromkeys(S.sample_orders(s, 0, 4 * budget, 12, 2)))[:budget]
            found["uniform"][j] += target in first
    for j in range(2):
        assert found["expansion"][j] >= found["mcts"][j] > found["uniform"][j], found
    assert found["mcts"][1] >= 12, found
