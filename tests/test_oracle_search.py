"""Pins of the discrete-search oracle (no GPU): mode code, neighbourhood,
Algorithm 1 invariants, and the admissible-order counts the paper prints
(Sec. III-A transition rules, Sec. III-B, Sec. IV-A)."""
import itertools
import os

import numpy as np
import pytest

from oracle import search as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_admissible_counts_match_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "admissible_counts.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 4
    for f, cap, count in rows:
        assert S.count_admissible_push(int(f), int(cap)) == int(count)


def test_admissible_count_brute_force_small():
    # the DP equals explicit enumeration on a small alphabet
    F, cap = 4, 5
    FREE = F

    def ok(s):
        if s[0] != FREE:
            return False
        for a, b in zip(s, s[1:]):
            if a == b:
                return False
            if a != FREE and b != FREE and (a - b) % F not in (1, F - 1):
                return False
        return True

    n = sum(ok(s) for L in range(1, cap + 1) for s in itertools.product(range(F + 1), repeat=L))
    assert n == S.count_admissible_push(F, cap)


def test_code_roundtrip_and_injective():
    seen = set()
    for L in range(1, 4):
        for s in itertools.product(range(12), repeat=L):
            c = S.encode(s, 12)
            assert S.decode(c, 12) == s
            seen.add(c)
    assert len(seen) == 12 + 144 + 1728
    assert S.encode([11] * 16, 12) < 2 ** 64


def test_neighbourhood_counts_and_order():
    M, Lmax = 12, 6
    s = (3, 7, 1)
    nb = S.neighbours(s, M, Lmax)
    assert len(nb) == 3 * 11 + 4 * 12 + 3
    assert nb[0] == (0, 7, 1) and nb[10] == (11, 7, 1)           # substitutions first
    assert nb[33] == (0, 3, 7, 1)                                 # then insertions
    assert nb[-3:] == [(7, 1), (3, 1), (3, 7)]                    # then deletions
    assert all(len(x) <= Lmax for x in nb)
    assert S.neighbours((5,), M, 1) == [(m,) for m in range(12) if m != 5]   # no insert/delete
    assert S.neighbour_slots(M, Lmax) >= max(len(S.neighbours(s, M, Lmax)) for s in [(0,) * 6, (1, 2)])


def test_expand_invariants():
    rng = np.random.default_rng(0)
    M, Lmax = 12, 4
    V = {}
    for s in itertools.product(range(M), repeat=2):
        V[S.encode(s, M)] = (float(rng.uniform()), s)
    out = S.expand(V, k=8, batch=500, n_modes=M, l_max=Lmax)
    codes = [S.encode(s, M) for s in out]
    assert len(out) <= 500 and len(set(codes)) == len(codes)
    assert not set(codes) & set(V)
    # walked in merit order: the first admitted orders are neighbours of the best one
    best = min(V.items(), key=lambda kv: (kv[1][0], kv[0]))[1][1]
    first = list(dict.fromkeys(x for x in S.neighbours(best, M, Lmax) if S.encode(x, M) not in V))
    assert out[: len(first)] == first


def test_expansion_recovers_enumeration_argmin_unlimited_budget():
    # Algorithm 1 invariant: with an unlimited budget (and a merit whose best
    # order is reachable by single edits) expansion finds enumeration's best
    M, Lmax = 5, 3
    allseq = [s for L in range(1, Lmax + 1) for s in itertools.product(range(M), repeat=L)]
    target = (4, 1, 3)

    def f(batch):
        return [sum(a != b for a, b in itertools.zip_longest(s, target, fillvalue=-1)) + 0.01 * len(s)
                for s in batch]

    V, sizes = S.run_expansion(f, [(m,) for m in range(M)], k=4, batch=20, n_modes=M, l_max=Lmax, rounds=100)
    best_enum = allseq[int(np.argmin(f(allseq)))]
    best_exp = min(V.values(), key=lambda v: v[0])[1]
    assert best_exp == best_enum == target
    assert all(sz <= 20 for sz in sizes[1:])
    assert len(V) == sum(sizes)                    # no order evaluated twice


def test_budget_truncates_last_batch():
    M, Lmax = 4, 3
    V, sizes = S.run_expansion(lambda b: [float(sum(s)) for s in b], [(m,) for m in range(M)], k=2, batch=10,
                               n_modes=M, l_max=Lmax, rounds=50, budget=23)
    assert sum(sizes) == 23 and len(V) == 23


def test_enumeration_argmin_prefers_feasible_then_index():
    costs = [1.0, 0.5, 0.5, 0.1]
    viols = [0.0, 0.0, 0.0, 1e-3]
    assert S.enumeration_argmin(costs, viols) == 1


# ------------------------------------------------ grammar (admissible orders)

def _lev(a, b):
    """Edit distance over segments (insert, delete, substitute one mode)."""
    d = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        prev, d[0] = d[0], i
        for j in range(1, len(b) + 1):
            cur = d[j]
            d[j] = min(d[j] + 1, d[j - 1] + 1, prev + (a[i - 1] != b[j - 1]))
            prev = cur
    return d[len(b)]


def test_admissible_orders_match_brute_force_and_the_paper():
    import itertools
    alpha = S.push_alphabet(4)
    brute = [s for L in range(1, 6) for s in itertools.product(alpha, repeat=L) if S.admissible_push(s)]
    assert S.admissible_orders(5) == brute          # same set and order (length, then lexicographic)
    # the paper's counts for the four-faced box (golden file)
    assert len(S.admissible_orders(6)) == S.count_admissible_push(4, 6) == 601
    assert len(S.admissible_orders(8)) == S.count_admissible_push(4, 8) == 6297


@pytest.mark.parametrize("seq", [(12,), (12, 0), (12, 3, 12, 9), (12, 0, 3, 6, 12)])
def test_grammar_neighbourhoods_by_edit_distance(seq):
    l_max = 6
    pool = S.admissible_orders(l_max)
    n1 = S.grammar_neighbours(seq, l_max, 1)
    assert set(n1) == {t for t in pool if _lev(seq, t) == 1}
    assert len(n1) == len(set(n1))
    n2 = S.grammar_neighbours(seq, l_max, 2)
    # every intermediate admissible: t is one edit from an admissible order
    # that is itself one edit from seq
    want = {t for t in pool if t != seq and any(_lev(t, u) <= 1 for u in n1)}
    assert set(n2) == want
    assert n2[: len(n1)] == n1                      # one-edit orders first, in order
    assert all(_lev(seq, t) <= 2 for t in n2)


def test_grammar_expansion_round():
    rng = np.random.default_rng(3)
    seeds = S.admissible_orders(3)
    V = {S.encode(s, 13): (float(rng.uniform()), s) for s in seeds}
    out = S.expand_grammar(V, k=4, batch=60, l_max=5, r=2)
    assert 0 < len(out) <= 60 and len(set(out)) == len(out)
    assert all(S.admissible_push(s) and S.encode(s, 13) not in V for s in out)
    # the first admitted orders come from the best-ranked parent
    best = min(V.values(), key=lambda v: (v[0], S.encode(v[1], 13)))[1]
    nb = [t for t in S.grammar_neighbours(best, 5, 2) if S.encode(t, 13) not in V]
    assert out[: len(nb)] == nb[: len(out)]


@pytest.mark.parametrize("seq", [(3,), (0, 7), (11, 2, 5)])
def test_two_edit_neighbourhood_by_edit_distance(seq):
    # N_2 over every order of 1..3 segments = the orders at edit distance 1
    # or 2 (any intermediate of length 1..l_max is an order), one-edit first
    l_max, M = 3, 12
    pool = [s for L in range(1, l_max + 1) for s in itertools.product(range(M), repeat=L)]
    n1 = S.neighbours_r(seq, M, l_max, 1)
    n2 = S.neighbours_r(seq, M, l_max, 2)
    assert set(n1) == {t for t in pool if _lev(seq, t) == 1}
    assert n2[: len(n1)] == n1
    # with l_max = 3 an intermediate may not exceed 3 segments
    want = {t for t in pool if t != seq and any(_lev(t, u) <= 1 for u in n1)}
    assert set(n2) == want and len(n2) == len(set(n2))


def test_workload_seed_orders_match_the_oracle_grammar():
    # the bench's seed generator (workloads) is written apart from the
    # oracle's grammar; both give the same orders in the same order
    import workloads as W
    for cap in (1, 4, 6):
        assert W.admissible_push_orders(cap) == S.admissible_orders(cap)
    assert len(W.admissible_push_orders(8)) == 6297


# ------------------------------------------------ uniform sampling of orders

def test_splitmix64_published_outputs():
    # the generator's first outputs from seed 0 (Steele, Lea and Flood 2014)
    assert [S.splitmix64(0, i) for i in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_unranking_follows_the_enumerations():
    pool = [s for L in range(1, 4) for s in itertools.product(range(5), repeat=L)]
    assert [S.unrank_order(i, 5, 3) for i in range(len(pool))] == pool
    A = S.admissible_orders(6)
    assert [S.unrank_admissible(i, 6) for i in range(len(A))] == A


def test_uniform_sample_frequencies():
    # 12 orders (3 modes, up to 2 segments), 24,000 draws: every count within
    # 5 standard deviations of 2,000
    from collections import Counter
    c = Counter(S.sample_orders(11, 0, 24000, 3, 2))
    assert len(c) == 12
    sd = (24000 * (1 / 12) * (11 / 12)) ** 0.5
    assert all(abs(v - 2000) <= 5 * sd for v in c.values())
    g = Counter(S.sample_orders(5, 0, 20000, 13, 4, grammar=1))
    assert set(g) == set(S.admissible_orders(4)) and all(S.admissible_push(s) for s in g)
