"""GPU expansion (Sec. III-B, Algorithm 1) against the oracle's search, bit
for bit: the same evaluated set V with the same merits must produce the same
next batch F_{s+1}, in the same order (rank key (M_hat, code), neighbourhood
enumeration order, deduplication against V and within the round)."""
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


def _problem(P, lmax):
    inst = W.push_l4_instance(0)
    inst["max_segments"] = lmax
    inst["knots_per_segment"] = 4
    return P.Problem([inst]), inst


def _add(P, f, seqs, merit):
    """Add orders with merit = cost (viol 0) from host arrays."""
    packed = P.pack_mode_seqs(seqs)
    cost = np.asarray(merit, dtype=np.float32)
    viol = np.zeros(len(seqs), np.float32)
    P.comet_frontier_add(f, packed, len(seqs), cost, viol)


def _next(P, f):
    return P.frontier_next_orders(f, 8192)


@pytest.mark.parametrize("seed,lmax,k,batch", [(0, 4, 8, 300), (1, 4, 64, 4096), (2, 6, 16, 100), (3, 3, 5, 50)])
def test_expand_matches_oracle(P, seed, lmax, k, batch):
    prob, inst = _problem(P, lmax)
    M = 12
    rng = np.random.default_rng(seed)
    # V: random orders of every length, merits drawn from a few values so that
    # ties (broken by the mode code) are frequent
    seqs = list({tuple(int(m) for m in rng.integers(0, M, rng.integers(1, lmax + 1))) for _ in range(400)})
    merit = rng.integers(0, 20, len(seqs)).astype(np.float32) * np.float32(0.125) + np.float32(0.5)
    f = P.comet_frontier_create(prob.handle, 0, 100000, batch, 64)
    _add(P, f, seqs, merit)
    P.comet_expand(prob.handle, f, k)
    got = _next(P, f)
    V = {S.encode(s, M): (float(m), s) for s, m in zip(seqs, merit)}
    want = S.expand(V, k=k, batch=batch, n_modes=M, l_max=lmax)
    assert got == want
    n, err = P.comet_frontier_size(f)
    assert n == len(seqs) and err == 0
    # top-k of V by (merit, code)
    codes, merits = P.comet_frontier_best(f, 10)
    ranked = sorted(V.items(), key=lambda kv: (kv[1][0], kv[0]))[:10]
    assert [int(c) for c in codes] == [c for c, _ in ranked]
    np.testing.assert_array_equal(merits, np.array([m for _, (m, _) in ranked], np.float32))
    P.comet_frontier_destroy(f)
    prob.close()


def test_rounds_of_algorithm_1_match_oracle(P):
    # several rounds with a synthetic merit (a function of the order only):
    # evaluate F_s, add to V, expand -- both sides must walk the same path
    prob, inst = _problem(P, 4)
    M = 12
    target = (3, 8, 1, 10)

    def merit_of(batch):
        return [np.float32(sum(a != b for a, b in zip(s + (-1,) * 4, target)) + 0.01 * len(s)) for s in batch]

    seeds = [(m,) for m in range(M)]
    f = P.comet_frontier_create(prob.handle, 0, 20000, 200, 16)
    V = {}
    frontier = seeds
    for _ in range(5):
        mer = merit_of(frontier)
        _add(P, f, frontier, mer)
        for s, m in zip(frontier, mer):
            V[S.encode(s, M)] = (float(m), s)
        P.comet_expand(prob.handle, f, 16)
        got = _next(P, f)
        want = S.expand(V, k=16, batch=200, n_modes=M, l_max=4)
        assert got == want
        frontier = got
        if not frontier:
            break
    best = min(V.values(), key=lambda v: (v[0], S.encode(v[1], M)))[1]
    assert best == target
    P.comet_frontier_destroy(f)
    prob.close()


def test_frontier_edge_cases(P):
    prob, inst = _problem(P, 3)
    with pytest.raises(P.CometError):
        P.comet_frontier_create(prob.handle, 5, 100, 10, 8)       # no such instance
    with pytest.raises(P.CometError):
        P.comet_frontier_create(prob.handle, 0, 100, 200, 8)      # batch > capacity
    f = P.comet_frontier_create(prob.handle, 0, 40, 40, 8)
    # empty V: expansion yields nothing
    P.comet_expand(prob.handle, f, 8)
    assert _next(P, f) == []
    # k larger than |V|
    _add(P, f, [(1,), (2, 3)], [0.5, 0.25])
    P.comet_expand(prob.handle, f, 8)
    got = _next(P, f)
    V = {S.encode((1,), 12): (0.5, (1,)), S.encode((2, 3), 12): (0.25, (2, 3))}
    assert got == S.expand(V, k=8, batch=40, n_modes=12, l_max=3)
    # an order of another instance from host memory is rejected
    bad = P.pack_mode_seqs([(1, 2)], inst_idx=[1])
    with pytest.raises(P.CometError):
        P.comet_frontier_add(f, bad, 1, np.zeros(1, np.float32), np.zeros(1, np.float32))
    # capacity overflow on the device is flagged, never written out of bounds
    many = [(a, b) for a in range(12) for b in range(12)][:60]
    _add(P, f, many[:38], np.ones(38, np.float32))
    _add(P, f, many[38:48], np.ones(10, np.float32))
    n, err = P.comet_frontier_size(f)
    assert n == 40 and err == 2
    P.comet_expand(prob.handle, f, 8)               # still safe to expand
    assert len(_next(P, f)) <= 40
    with pytest.raises(P.CometError):               # one call larger than the capacity
        _add(P, f, many, np.ones(60, np.float32))
    P.comet_frontier_destroy(f)
    prob.close()


@pytest.mark.parametrize("seed,lmax,k,batch,r", [(0, 4, 8, 20000, 2), (1, 3, 16, 500, 2), (2, 5, 4, 20000, 1)])
def test_two_edit_expansion_matches_oracle(P, seed, lmax, k, batch, r):
    # N_r over every order (Sec. III-B "at most r edits"): the one-edit orders
    # of a parent first, then the one-edit orders of each of them in order
    prob, inst = _problem(P, lmax)
    M = 12
    rng = np.random.default_rng(seed)
    seqs = list({tuple(int(m) for m in rng.integers(0, M, rng.integers(1, lmax + 1))) for _ in range(200)})
    merit = rng.integers(0, 20, len(seqs)).astype(np.float32) * np.float32(0.125) + np.float32(0.5)
    f = P.comet_frontier_create(prob.handle, 0, 2000000, batch, 64, radius=r)
    _add(P, f, seqs, merit)
    P.comet_expand(prob.handle, f, k)
    got = P.frontier_next_orders(f, batch)
    V = {S.encode(s, M): (float(m), s) for s, m in zip(seqs, merit)}
    assert got == S.expand(V, k=k, batch=batch, n_modes=M, l_max=lmax, r=r)
    P.comet_frontier_destroy(f)
    prob.close()


@pytest.mark.parametrize("r,batch", [(1, 20000), (2, 20000), (2, 300)])
def test_grammar_expansion_matches_oracle(P, r, batch):
    # the pushing grammar over the 13-mode alphabet (stick on a face, free
    # motion): only admissible orders, every intermediate admissible
    inst = dict(W.push_l4_instance(0), n_modes=13, max_segments=6, knots_per_segment=4)
    prob = P.Problem([inst])
    rng = np.random.default_rng(5 + r)
    seqs = S.admissible_orders(3)
    merit = rng.integers(0, 10, len(seqs)).astype(np.float32) * np.float32(0.25) + np.float32(1.0)
    f = P.comet_frontier_create(prob.handle, 0, 200000, batch, 64, radius=r, grammar=P.GRAMMAR_PUSH)
    _add(P, f, seqs, merit)
    P.comet_expand(prob.handle, f, 8)
    got = P.frontier_next_orders(f, batch)
    V = {S.encode(s, 13): (float(m), s) for s, m in zip(seqs, merit)}
    want = S.expand_grammar(V, k=8, batch=batch, l_max=6, r=r)
    assert got == want and all(S.admissible_push(s) for s in got)
    P.comet_frontier_destroy(f)
    # the rule is checked: the grammar needs the 13-mode alphabet
    prob12, _ = _problem(P, 4)
    with pytest.raises(P.CometError):
        P.comet_frontier_create(prob12.handle, 0, 1000, 100, 8, radius=1, grammar=P.GRAMMAR_PUSH)
    with pytest.raises(P.CometError):
        P.comet_frontier_create(prob12.handle, 0, 1000, 100, 8, radius=3)
    prob12.close()
    prob.close()


@pytest.mark.parametrize("grammar", [0, 1])
def test_uniform_sampler_matches_oracle(P, grammar):
    # the uniform-sampling policy's orders, bit for bit: SplitMix64 draws and
    # the unranking of the (length, lexicographic) enumeration
    inst = W.push_grammar_instance(0) if grammar else W.push_l4_instance(0)
    prob = P.Problem([inst])
    for seed in (0, 7, 2 ** 63 + 5):
        rec = P.comet_sample_orders(prob.handle, 0, seed, 100, 3000, grammar)
        got = [tuple(int(m) for m in r["modes"][: r["len"]]) for r in rec]
        assert all(int(r["instance"]) == 0 for r in rec)
        assert got == S.sample_orders(seed, 100, 3000, inst["n_modes"], inst["max_segments"], grammar)
    prob.close()


def test_frontier_checkpoint_resumes_the_rounds(P, tmp_path):
    # Algorithm 1's rounds with a synthetic merit, interrupted after two
    # rounds: the frontier saved there and loaded into a new frontier walks
    # the same remaining rounds as the uninterrupted one (same batches, same
    # best orders); mismatched frontiers and foreign files are refused
    prob, inst = _problem(P, 4)
    M = 12
    target = (3, 8, 1, 10)

    def merit_of(batch):
        return [np.float32(sum(a != b for a, b in zip(s + (-1,) * 4, target)) + 0.01 * len(s)) for s in batch]

    def rounds(f, frontier, n):
        seen = []
        for _ in range(n):
            _add(P, f, frontier, merit_of(frontier))
            P.comet_expand(prob.handle, f, 16)
            frontier = _next(P, f)
            seen.append(frontier)
        return frontier, seen

    seeds = [(m,) for m in range(M)]
    fa = P.comet_frontier_create(prob.handle, 0, 20000, 200, 16)
    mid, _ = rounds(fa, seeds, 2)
    path = str(tmp_path / "frontier.ckpt")
    P.comet_frontier_save(fa, path)
    fb = P.comet_frontier_create(prob.handle, 0, 20000, 200, 16)
    P.comet_frontier_load(fb, path)
    assert P.comet_frontier_size(fb)[0] == P.comet_frontier_size(fa)[0]
    assert _next(P, fb) == mid
    ca, ma = P.comet_frontier_best(fa, 16)
    cb, mb = P.comet_frontier_best(fb, 16)
    np.testing.assert_array_equal(ca, cb)
    np.testing.assert_array_equal(ma, mb)
    _, seen_a = rounds(fa, mid, 3)
    _, seen_b = rounds(fb, mid, 3)
    assert seen_a == seen_b
    np.testing.assert_array_equal(P.comet_frontier_best(fa, 16)[0], P.comet_frontier_best(fb, 16)[0])
    # another neighbourhood rule, a smaller frontier, a foreign file
    fr = P.comet_frontier_create(prob.handle, 0, 20000, 200, 16, radius=2)
    with pytest.raises(P.CometError):
        P.comet_frontier_load(fr, path)
    fs = P.comet_frontier_create(prob.handle, 0, 100, 50, 16)
    with pytest.raises(P.CometError):
        P.comet_frontier_load(fs, path)
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"\0" * 200)
    with pytest.raises(P.CometError):
        P.comet_frontier_load(fb, str(bad))
    # a truncated file, and a pending order with a mode outside the alphabet
    # (the last 40-byte record's first mode: int32 instance, u8 len, 3 pad
    # bytes, then u16 modes)
    raw = bytearray(open(path, "rb").read())
    bad.write_bytes(bytes(raw[:-10]))
    with pytest.raises(P.CometError):
        P.comet_frontier_load(fb, str(bad))
    raw[len(raw) - 40 + 8: len(raw) - 40 + 10] = (M).to_bytes(2, "little")
    bad.write_bytes(bytes(raw))
    with pytest.raises(P.CometError):
        P.comet_frontier_load(fb, str(bad))
    for f in (fa, fb, fr, fs):
        P.comet_frontier_destroy(f)
    prob.close()
