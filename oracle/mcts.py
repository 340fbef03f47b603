"""Monte Carlo tree search over mode orders -- TEST INFRASTRUCTURE ONLY
(plain Python; imported by tests/, never by the product path).

The comparison policy of Sec. IV-A and IV-B of the paper: UCT with
exploration constant c = 0.8, virtual loss and random rollouts, a pool of P
orders handed to the evaluator at a time, and the reward J_best / J_hat for a
feasible order (0 otherwise; Sec. IV-A) or M_best / M_hat (Sec. IV-B), with
M_hat the merit of Eq. search_merit.

The paper names these ingredients and nothing more; the readings below are
this implementation's (the native search in csrc/mcts.cu follows the same
ones, so that the two agree order for order):
  * tree: a node is a prefix of an order; its actions, in slot order, are
    "stop" (slot 0: the prefix itself is the order; prefixes of length >= 1)
    and "append mode a_j" (slot 1 + j, j over the alphabet in ascending
    order; length < l_max and, under the pushing grammar, the extended prefix
    admissible).  The root is the empty prefix;
  * selection: from the root, while the node has no untried action, go to
    the child of largest UCT score  w / n + c sqrt(ln n_parent / n)  among
    children that are not exhausted (ties: lowest slot);
  * expansion: one untried action of the node, drawn uniformly (draw mod the
    number of untried actions, in slot order), becomes a child;
  * rollout: from the child, one draw per step picks uniformly among the
    available actions until "stop"; a "stop" child rolls out to its prefix;
  * virtual loss: every node on the path gets its visit at selection time
    with reward 0; the reward is added when the order's result is known --
    at once when the order was evaluated before, else when the pool that
    holds it is told;
  * pool: distinct orders not evaluated before, at most P per ask and at
    most the evaluation budget in total; an order already waiting in the
    pool adds its path to that entry;
  * exhaustion: a "stop" child is exhausted when created (its order is
    claimed), any other node once it has no untried action and all its
    children are exhausted; selection never enters an exhausted child, so
    with enough budget every order is evaluated exactly once;
  * reward at tell time: J_best (or M_best) is first updated with the whole
    pool, then each waiting path receives its order's reward, pool entries
    in order and paths in arrival order;
  * random numbers: draw_i = SplitMix64 output i from the seed (the
    generator of oracle.search.splitmix64), one counter for the whole run.
"""
from __future__ import annotations

import math
from typing import Callable, Sequence

from .search import PUSH_FREE, _ok, encode, merit, push_alphabet, splitmix64

REWARD_FEASIBLE = 0  # J_best / J_hat for a feasible order, 0 otherwise (Sec. IV-A)
REWARD_MERIT = 1     # M_best / M_hat (Sec. IV-B)


class Node:
    __slots__ = ("prefix", "stop", "n", "w", "untried", "children", "exhausted")

    def __init__(self, prefix: tuple, stop: bool, slots: list):
        self.prefix = prefix
        self.stop = stop
        self.n = 0
        self.w = 0.0
        self.untried = [] if stop else slots
        self.children: dict[int, Node] = {}
        self.exhausted = stop


def uct_score(w: float, n: int, n_parent: int, c: float) -> float:
    """UCT of a child with total reward w over n visits under a parent with
    n_parent visits."""
    return w / n + c * math.sqrt(math.log(n_parent) / n)


class Mcts:
    def __init__(self, n_modes: int, l_max: int, grammar: int = 0, seed: int = 0, c_uct: float = 0.8,
                 max_evals: int = 0, reward: int = REWARD_FEASIBLE, eps_feas: float = 1e-5, mu: float = 100.0):
        self.n_modes, self.l_max, self.grammar = n_modes, l_max, grammar
        self.alpha = push_alphabet() if grammar == 1 else tuple(range(n_modes))
        self.seed, self.ctr = seed, 0
        self.c, self.max_evals, self.reward_kind = c_uct, max_evals, reward
        self.eps, self.mu = eps_feas, mu
        self.root = Node((), False, self.slots(()))
        self.nodes = 1
        self.results: dict[int, tuple[float, float]] = {}  # code -> (cost, viol)
        self.best = math.inf  # J_best (feasible) or M_best
        self.issued = 0
        self.pool: list[tuple] = []
        self.waiting: dict[int, list] = {}

    # -- the order space ---------------------------------------------------
    def slots(self, prefix: tuple) -> list[int]:
        """Available actions of a prefix, in slot order."""
        out = [0] if prefix else []
        if len(prefix) < self.l_max:
            for j, m in enumerate(self.alpha):
                if self.grammar == 1:
                    ok = (m == PUSH_FREE) if not prefix else _ok(prefix[-1], m)
                else:
                    ok = True
                if ok:
                    out.append(1 + j)
        return out

    def draw(self) -> int:
        d = splitmix64(self.seed, self.ctr)
        self.ctr += 1
        return d

    def child_prefix(self, prefix: tuple, slot: int) -> tuple:
        return prefix if slot == 0 else prefix + (self.alpha[slot - 1],)

    # -- rewards ------------------------------------------------------------
    def value(self, cost: float, viol: float) -> float:
        """The quantity J_best or M_best ranks (inf when it does not count)."""
        if not (math.isfinite(cost) and math.isfinite(viol)):
            return math.inf
        if self.reward_kind == REWARD_MERIT:
            return merit(cost, viol, self.eps, self.mu)
        return cost if viol <= self.eps else math.inf

    def reward(self, cost: float, viol: float) -> float:
        v = self.value(cost, viol)
        if v == math.inf:
            return 0.0
        if v <= 0.0:
            return 1.0
        return self.best / v

    # -- one search step ------------------------------------------------------
    def ask(self, pool: int) -> list[tuple]:
        """The next pool of at most `pool` orders to evaluate."""
        assert not self.pool, "tell the pending pool first"
        while (len(self.pool) < pool and not self.root.exhausted
               and (self.max_evals <= 0 or self.issued + len(self.pool) < self.max_evals)):
            self.attempt()
        return list(self.pool)

    def attempt(self) -> None:
        node, path = self.root, [self.root]
        while not node.untried:
            best, best_s = None, -math.inf
            for slot in sorted(node.children):
                ch = node.children[slot]
                if ch.exhausted:
                    continue
                s = uct_score(ch.w, ch.n, node.n, self.c)
                if s > best_s:
                    best, best_s = ch, s
            assert best is not None, "selection reached an exhausted node"
            node = best
            path.append(node)
        # expansion
        i = self.draw() % len(node.untried)
        slot = node.untried.pop(i)
        prefix = self.child_prefix(node.prefix, slot)
        child = Node(prefix, slot == 0, [] if slot == 0 else self.slots(prefix))
        node.children[slot] = child
        self.nodes += 1
        path.append(child)
        # rollout
        order = prefix
        if slot != 0:
            while True:
                acts = self.slots(order)
                a = acts[self.draw() % len(acts)]
                if a == 0:
                    break
                order = order + (self.alpha[a - 1],)
        # virtual loss, then the reward now or when the pool is told
        for v in path:
            v.n += 1
        code = encode(order, self.n_modes)
        if code in self.results:
            r = self.reward(*self.results[code])
            for v in path:
                v.w += r
        elif code in self.waiting:
            self.waiting[code].append(path)
        else:
            self.pool.append(order)
            self.waiting[code] = [path]
        # exhaustion, bottom up
        for v in reversed(path):
            if v.untried or any(not ch.exhausted for ch in v.children.values()):
                break
            v.exhausted = True

    def tell(self, costs: Sequence[float], viols: Sequence[float]) -> None:
        """Results of the pending pool, in pool order."""
        assert len(costs) == len(self.pool) == len(viols)
        codes = [encode(o, self.n_modes) for o in self.pool]
        for code, c, v in zip(codes, costs, viols):
            self.results[code] = (float(c), float(v))
            self.best = min(self.best, self.value(float(c), float(v)))
        for code in codes:
            r = self.reward(*self.results[code])
            for path in self.waiting.pop(code):
                for v in path:
                    v.w += r
        self.issued += len(self.pool)
        self.pool = []

    def best_orders(self, k: int) -> list[int]:
        """Codes of the k evaluated orders of least (M_hat, code)."""
        keys = []
        for code, (c, v) in self.results.items():
            m = merit(c, v, self.eps, self.mu)
            keys.append((m if m == m else math.inf, code))  # a non-finite result ranks last
        keys.sort()
        return [code for _, code in keys[:k]]


def run(evaluate: Callable[[list], tuple], pool: int, **kw) -> Mcts:
    """Ask / evaluate / tell until the budget is spent or every order is
    evaluated; evaluate(orders) -> (costs, viols)."""
    t = Mcts(**kw)
    while True:
        orders = t.ask(pool)
        if not orders:
            return t
        costs, viols = evaluate(orders)
        t.tell(costs, viols)
