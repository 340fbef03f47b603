"""The GPU-vs-oracle parity harness (tests/_parity.py) checked on the CPU.

Two FP64 oracle runs of the same orders that take different penalty paths
(beta_0 = 100 and 300) are both valid answers of the evaluator: the harness
must accept the second against the first at the acceptance bar, and it must
catch a planted cost error of 1e-3 relative and a planted state error of
5e-3 on TOs that reach the same local solution."""
import os

import numpy as np

import _parity as PA
import oracle
import workloads as W


def _runs():
    insts = [W.push_l2_instance(s) for s in range(8)]
    seqs = W.all_sequences(12, 2)
    allseq = np.tile(seqs, (len(insts), 1))
    n = len(allseq)
    idx = np.repeat(np.arange(len(insts)), len(seqs)).astype(np.int32)
    lens, Ns = np.full(n, 2, np.int32), np.full(n, 16)
    ref, rtr, _ = oracle.solve_batch_ex(insts, idx, allseq, lens, nthreads=os.cpu_count())
    g, gtr, _ = oracle.solve_batch_ex(insts, idx, allseq, lens, opts=oracle.default_opts(beta0=300.0),
                                      nthreads=os.cpu_count())
    other = dict(status=g["status"], cost=g["cost"].copy(), viol=g["viol"], traj=gtr.copy(), traj_nmax=16)
    return insts, allseq, idx, lens, Ns, ref, rtr, other


def test_two_fp64_runs_meet_the_bar():
    insts, allseq, idx, lens, Ns, ref, rtr, other = _runs()
    T = PA.Task(False)
    rep = PA.compare(T, insts, idx, list(allseq), lens, Ns, other, ref, rtr)
    assert rep["same"] >= 0.7 * rep["joint"]
    assert not rep["vhat_fail"]
    assert not rep["cost_excess"]
    assert len(rep["state_excess"]) <= max(2, rep["same"] // 100)
    assert not PA.certify_different(T, insts, idx, list(allseq), lens, Ns, other, rep)
    flags = PA.flag_disagreements(other, ref)
    assert all(a != 0 or b != 0 for _, a, b in flags)
    out, bad = PA.argmin_parity(T, insts, [slice(144 * i, 144 * (i + 1)) for i in range(len(insts))], idx,
                                list(allseq), lens, Ns, other, ref, rtr)
    assert not bad


def test_planted_errors_are_caught():
    insts, allseq, idx, lens, Ns, ref, rtr, other = _runs()
    T = PA.Task(False)
    rep = PA.compare(T, insts, idx, list(allseq), lens, Ns, other, ref, rtr, verbose=False)
    # pick TOs that reach the same local solution with a clean margin
    same = [t for t in range(len(idx)) if other["status"][t] == 0 and ref["status"][t] == 0
            and abs(other["cost"][t] - ref["cost"][t]) <= 1e-6 * abs(ref["cost"][t])][:12]
    assert len(same) >= 8
    a, b = same[:4], same[4:8]
    for t in a:
        other["cost"][t] *= 1.001                       # cost off by 1e-3 relative
    for t in b:
        other["traj"][t][17 + 8] += 5e-3                # y at knot 8 off by 5e-3
    rep = PA.compare(T, insts, idx, list(allseq), lens, Ns, other, ref, rtr, sel=np.array(same), verbose=False)
    assert {e[0] for e in rep["cost_excess"]} >= set(a)
    assert {e[0] for e in rep["state_excess"]} >= set(b)


def test_padded_orders_of_mixed_lengths():
    # orders of 1..4 segments passed as a zero-padded mode array with their
    # lengths: every order is compared at its own length (a padded order read
    # whole would be another order, with other rows and v_hat)
    insts = [W.push_l4_instance(s) for s in (0, 1)]
    rng = np.random.default_rng(4)
    seqs = [tuple(int(m) for m in rng.integers(0, 12, 1 + t % 4)) for t in range(24)]
    idx = (np.arange(24) % 2).astype(np.int32)
    modes, lens = W.pad_sequences(seqs, 4)
    Ns = 20 * lens
    ref, rtr, _ = oracle.solve_batch_ex(insts, idx, modes, lens, nthreads=os.cpu_count())
    g, gtr, _ = oracle.solve_batch_ex(insts, idx, modes, lens, opts=oracle.default_opts(beta0=300.0),
                                      nthreads=os.cpu_count())
    # the answers in the GPU's layout, padded to the longest order (N = 80)
    Nm = int(Ns.max())
    tr = np.zeros((24, 7 * Nm + 4))
    for t in range(24):
        N = int(Ns[t])
        for i in range(4):
            tr[t, i * (Nm + 1): i * (Nm + 1) + N + 1] = gtr[t][i * (N + 1): (i + 1) * (N + 1)]
        for j in range(3):
            tr[t, 4 * (Nm + 1) + j * Nm: 4 * (Nm + 1) + j * Nm + N] = gtr[t][4 * (N + 1) + j * N: 4 * (N + 1) + (j + 1) * N]
    other = dict(status=g["status"], cost=g["cost"], viol=g["viol"], traj=tr, traj_nmax=Nm)
    T = PA.Task(False)
    rep = PA.compare(T, insts, idx, list(modes), lens, Ns, other, ref, rtr, verbose=False)
    assert rep["joint"] >= 12
    assert not rep["vhat_fail"], rep["vhat_fail"]
    assert not rep["cost_excess"], rep["cost_excess"]
    assert not PA.certify_different(T, insts, idx, list(modes), lens, Ns, other, rep)
