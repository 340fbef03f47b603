"""Discrete-search oracle -- TEST INFRASTRUCTURE ONLY (plain Python).

Follows Sec. III-B of the paper:
  * Eq. mode_selection: full enumeration picks argmin of the merit over the
    evaluated orders (feasible first; ties go to the lower enumeration index);
  * Eq. search_merit:   M_hat = J_hat + mu * max(v_hat - eps_feas, 0);
  * "Neighborhood expansion": N_1(m) = one insertion, deletion or
    substitution of a mode segment;
  * Algorithm 1: walk the evaluated set V in increasing merit and admit unseen
    neighbours (not in V or the next batch) until the batch holds B orders.

Readings where the paper is silent:
  * enumeration order of a neighbourhood: substitutions (position, then mode
    ascending), then insertions (position 0..L, mode ascending), then
    deletions (position ascending); lengths outside [1, L_max] are skipped;
  * only the k best orders of V are walked (beam k);
  * rank key (M_hat, code) -- the u64 mode code breaks ties;
  * mode code: code = L + sum_i (m_i + 1) (M + 1)^(i + 1).
"""
from __future__ import annotations

from typing import Iterable, Sequence


def encode(seq: Sequence[int], n_modes: int) -> int:
    """u64 mode code of a sequence (length in the lowest digit)."""
    base = n_modes + 1
    code = len(seq)
    p = base
    for m in seq:
        code += (int(m) + 1) * p
        p *= base
    assert code < 2 ** 64
    return code


def decode(code: int, n_modes: int) -> tuple[int, ...]:
    base = n_modes + 1
    L = code % base
    code //= base
    out = []
    for _ in range(L):
        out.append(code % base - 1)
        code //= base
    return tuple(out)


def merit(cost: float, viol: float, eps_feas: float = 1e-5, mu: float = 100.0) -> float:
    """Eq. search_merit."""
    return cost + mu * max(viol - eps_feas, 0.0)


def enumeration_argmin(costs, viols, eps_feas: float = 1e-5, mu: float = 100.0) -> int:
    """Eq. mode_selection over an enumerated list: the feasible order of least
    merit (lowest index on ties); if none is feasible, the least merit."""
    best, best_key = -1, None
    for i, (c, v) in enumerate(zip(costs, viols)):
        key = (0 if v <= eps_feas else 1, merit(c, v, eps_feas, mu), i)
        if best_key is None or key < best_key:
            best, best_key = i, key
    return best


def neighbours(seq: Sequence[int], n_modes: int, l_max: int) -> list[tuple[int, ...]]:
    """N_1(m) in the enumeration order stated in the module docstring
    (duplicates kept; the caller skips orders already seen)."""
    s = tuple(int(m) for m in seq)
    L = len(s)
    out: list[tuple[int, ...]] = []
    for i in range(L):                       # substitutions
        for m in range(n_modes):
            if m != s[i]:
                out.append(s[:i] + (m,) + s[i + 1:])
    if L + 1 <= l_max:                       # insertions
        for i in range(L + 1):
            for m in range(n_modes):
                out.append(s[:i] + (m,) + s[i:])
    if L - 1 >= 1:                           # deletions
        for i in range(L):
            out.append(s[:i] + s[i + 1:])
    return out


def neighbour_slots(n_modes: int, l_max: int) -> int:
    """Upper bound on |N_1(m)| for any m of length <= l_max: the number of
    neighbour slots per parent used to order candidates."""
    L = l_max
    return L * (n_modes - 1) + (L + 1) * n_modes + L


def neighbours_r(seq: Sequence[int], n_modes: int, l_max: int, r: int = 1) -> list[tuple[int, ...]]:
    """N_r(m) over every order of 1..l_max segments (r <= 2): the one-edit
    neighbours in the order of `neighbours`, then with r = 2 the one-edit
    neighbours of each of them in that order; first occurrences kept, m
    excluded."""
    s = tuple(int(m) for m in seq)
    first = neighbours(s, n_modes, l_max)
    out, seen = [], {s}
    for t in first:
        if t not in seen:
            seen.add(t)
            out.append(t)
    if r >= 2:
        for t in first:
            for u in neighbours(t, n_modes, l_max):
                if u not in seen:
                    seen.add(u)
                    out.append(u)
    return out


def expand(evaluated: dict, k: int, batch: int, n_modes: int, l_max: int, r: int = 1) -> list[tuple[int, ...]]:
    """One round of Algorithm 1 (lines 5-10) on the evaluated set
    V = {code: (merit, seq)}: walk the k best orders by (merit, code) and
    admit unseen orders of each r-edit neighbourhood until `batch` orders
    are collected."""
    ranked = sorted(evaluated.items(), key=lambda kv: (kv[1][0], kv[0]))[:k]
    seen = set(evaluated)
    out: list[tuple[int, ...]] = []
    for _, (_, seq) in ranked:
        for nb in (neighbours(seq, n_modes, l_max) if r == 1 else neighbours_r(seq, n_modes, l_max, r)):
            c = encode(nb, n_modes)
            if c in seen:
                continue
            seen.add(c)
            out.append(nb)
            if len(out) == batch:
                return out
    return out


def run_expansion(evaluate, seed_batch: Iterable[Sequence[int]], k: int, batch: int, n_modes: int,
                  l_max: int, rounds: int, budget: int | None = None):
    """Algorithm 1's loop: evaluate F_s, add to V, expand; stops after
    `rounds` expansions, when no unseen neighbour remains, or at the budget
    (the last batch is truncated to fit).  evaluate(list_of_seqs) returns a
    list of merits.  Returns V = {code: (merit, seq)} and the batch sizes."""
    V: dict = {}
    frontier = [tuple(int(m) for m in s) for s in seed_batch]
    sizes = []
    s = 0
    while frontier and s <= rounds:
        if budget is not None:
            frontier = frontier[: max(0, budget - len(V))]
            if not frontier:
                break
        merits = evaluate(frontier)
        for seq, mval in zip(frontier, merits):
            V[encode(seq, n_modes)] = (float(mval), seq)
        sizes.append(len(frontier))
        frontier = expand(V, k, batch, n_modes, l_max)
        s += 1
    return V, sizes


# ---------------------------------------------------------------- grammar

def count_admissible_push(n_faces: int, cap: int) -> int:
    """Number of admissible pushing orders of at most `cap` segments over the
    alphabet {free} + faces (Sec. III-A: no two consecutive segments share a
    mode; a contact changes faces through free motion).  Reading fixed by the
    counts the paper prints (Sec. IV-A): orders start in free, and a direct
    contact-to-contact switch is allowed only between adjacent faces of the
    cyclic face list.  Counted by brute-force dynamic programming over the
    last mode."""
    FREE = n_faces

    def ok(a, b):
        if a == b:
            return False
        if a == FREE or b == FREE:
            return True
        return (a - b) % n_faces in (1, n_faces - 1)

    counts = {FREE: 1}   # sequences of length 1 that start in free
    total = 1
    for _ in range(2, cap + 1):
        nxt: dict = {}
        for last, c in counts.items():
            for m in range(n_faces + 1):
                if ok(last, m):
                    nxt[m] = nxt.get(m, 0) + c
        counts = nxt
        total += sum(counts.values())
    return total


# ------------------------------------------- grammar over the 13-mode alphabet
#
# The paper's pushing modes are sticking contact on a face or free motion
# (Sec. III-A, IV-A).  In the 13-mode pushing alphabet (faces x {stick,
# slide+, slide-} = 0..11, free motion = 12) they are the modes 3 f and 12.
# Admissible orders follow the rules of count_admissible_push: start in free
# motion, no two consecutive segments share a mode, and a direct
# contact-to-contact switch joins adjacent faces of the cyclic face list.

PUSH_FREE = 12


def push_alphabet(n_faces: int = 4) -> tuple[int, ...]:
    """The task alphabet in ascending mode order: stick on each face, free."""
    return tuple(3 * f for f in range(n_faces)) + (PUSH_FREE,)


def admissible_push(seq: Sequence[int], n_faces: int = 4) -> bool:
    s = tuple(int(m) for m in seq)
    if not s or s[0] != PUSH_FREE:
        return False
    alpha = set(push_alphabet(n_faces))
    if any(m not in alpha for m in s):
        return False
    for a, b in zip(s, s[1:]):
        if a == b:
            return False
        if a != PUSH_FREE and b != PUSH_FREE and (a // 3 - b // 3) % n_faces not in (1, n_faces - 1):
            return False
    return True


def admissible_orders(cap: int, n_faces: int = 4) -> list[tuple[int, ...]]:
    """All admissible orders of 1..cap segments, by length, then
    lexicographically in alphabet order (the seed batch F_0 of Sec. III-B)."""
    alpha = push_alphabet(n_faces)
    out: list[tuple[int, ...]] = []
    level = [(PUSH_FREE,)]
    for _ in range(cap):
        out += level
        level = [s + (m,) for s in level for m in alpha if admissible_push(s + (m,), n_faces)]
    return out


def alphabet_neighbours(seq: Sequence[int], alpha: Sequence[int], l_max: int) -> list[tuple[int, ...]]:
    """One-edit neighbours over `alpha` in the enumeration order of
    `neighbours`: substitutions, insertions, deletions, by position and then
    by alphabet position."""
    s = tuple(int(m) for m in seq)
    L = len(s)
    out: list[tuple[int, ...]] = []
    for i in range(L):
        for m in alpha:
            if m != s[i]:
                out.append(s[:i] + (m,) + s[i + 1:])
    if L + 1 <= l_max:
        for i in range(L + 1):
            for m in alpha:
                out.append(s[:i] + (m,) + s[i:])
    if L - 1 >= 1:
        for i in range(L):
            out.append(s[:i] + s[i + 1:])
    return out


def grammar_neighbours(seq: Sequence[int], l_max: int, r: int = 1, n_faces: int = 4) -> list[tuple[int, ...]]:
    """N_r(m) (Sec. III-B): orders within r <= 2 edits of m with every
    intermediate order admissible, in enumeration order: the admissible
    one-edit neighbours of m, then (r = 2) for each of them in that order its
    own admissible one-edit neighbours; first occurrences kept, m excluded."""
    alpha = push_alphabet(n_faces)
    s = tuple(int(m) for m in seq)

    def n1(t):
        return [u for u in alphabet_neighbours(t, alpha, l_max) if admissible_push(u, n_faces)]

    out, seen = [], {s}
    first = n1(s)
    for t in first:
        if t not in seen:
            seen.add(t)
            out.append(t)
    if r >= 2:
        for t in first:
            for u in n1(t):
                if u not in seen:
                    seen.add(u)
                    out.append(u)
    return out


def expand_grammar(evaluated: dict, k: int, batch: int, l_max: int, r: int = 1, n_faces: int = 4,
                   n_modes: int = 13) -> list[tuple[int, ...]]:
    """One round of Algorithm 1 over admissible orders: walk the k best
    orders of V by (merit, code) and admit unseen orders of each r-edit
    neighbourhood until `batch` are collected."""
    ranked = sorted(evaluated.items(), key=lambda kv: (kv[1][0], kv[0]))[:k]
    seen = set(evaluated)
    out: list[tuple[int, ...]] = []
    for _, (_, seq) in ranked:
        for nb in grammar_neighbours(seq, l_max, r, n_faces):
            c = encode(nb, n_modes)
            if c in seen:
                continue
            seen.add(c)
            out.append(nb)
            if len(out) == batch:
                return out
    return out


# ------------------------------------------------- uniform sampling of orders
#
# The uniform-sampling search policy (a comparison policy on the same
# evaluator): order i of a sample is drawn from a counter-based generator,
# SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
# generators", 2014): state_i = seed + (i + 1) * 0x9E3779B97F4A7C15 (mod
# 2^64), draw_i = mix(state_i).  The draw modulo the number T of orders picks
# the order at that index of the (length, lexicographic) enumeration.

_M64 = (1 << 64) - 1


def splitmix64(seed: int, i: int) -> int:
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def unrank_order(index: int, n_modes: int, l_max: int) -> tuple[int, ...]:
    """Order number `index` among every order of 1..l_max segments over
    n_modes modes, by length and then lexicographically."""
    for L in range(1, l_max + 1):
        cnt = n_modes ** L
        if index < cnt:
            digits = []
            for _ in range(L):
                digits.append(index % n_modes)
                index //= n_modes
            return tuple(reversed(digits))
        index -= cnt
    raise ValueError("index past the order space")


def _ok(a: int, b: int, n_faces: int = 4) -> bool:
    if a == b:
        return False
    if a == PUSH_FREE or b == PUSH_FREE:
        return True
    return (a // 3 - b // 3) % n_faces in (1, n_faces - 1)


def unrank_admissible(index: int, cap: int, n_faces: int = 4) -> tuple[int, ...]:
    """Admissible order number `index` in the order of admissible_orders(cap)
    (by length, then lexicographically), built left to right from the
    number of admissible completions after each candidate mode."""
    alpha = push_alphabet(n_faces)
    comp = [{m: 1 for m in alpha}]
    for r in range(1, cap):
        comp.append({m: sum(comp[r - 1][b] for b in alpha if _ok(m, b, n_faces)) for m in alpha})
    for L in range(1, cap + 1):
        cnt = comp[L - 1][PUSH_FREE]
        if index < cnt:
            seq = [PUSH_FREE]
            for pos in range(1, L):
                rem = L - 1 - pos
                for b in alpha:
                    if not _ok(seq[-1], b, n_faces):
                        continue
                    c = comp[rem][b]
                    if index < c:
                        seq.append(b)
                        break
                    index -= c
            return tuple(seq)
        index -= cnt
    raise ValueError("index past the admissible orders")


def sample_orders(seed: int, first: int, n: int, n_modes: int, l_max: int, grammar: int = 0) -> list:
    """Orders first .. first + n - 1 of the uniform sample (grammar 0: every
    order; 1: the admissible pushing orders)."""
    if grammar == 1:
        total = len(admissible_orders(l_max))
        return [unrank_admissible(splitmix64(seed, i) % total, l_max) for i in range(first, first + n)]
    total = sum(n_modes ** L for L in range(1, l_max + 1))
    return [unrank_order(splitmix64(seed, i) % total, n_modes, l_max) for i in range(first, first + n)]
