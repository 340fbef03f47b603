"""The allocation-free entry point, comet_eval_modes_noalloc.

It exists for callers that must not allocate device memory: code running
inside a pool or arena that owns all device memory of the process, real-time
loops where cudaMalloc / cudaFree (and the synchronisation they can imply) are
not allowed after start-up, or hosts that forbid the CUDA allocator.  It runs
the same evaluator as comet_eval_modes with its scratch in a fixed device
array of the library, so its results must match the problem-based entry
point; two calls in a row check that the shared scratch is reset between
calls.  The file is named so that pytest collects it last.
"""
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


def _orders(seed, n, insts):
    rng = np.random.default_rng(seed)
    seqs, idx = [], []
    for t in range(n):
        i = t % len(insts)
        L = 1 + int(rng.integers(0, insts[i]["max_segments"]))
        seqs.append(tuple(int(m) for m in rng.integers(0, 12, L)))
        idx.append(i)
    return seqs, idx


def _reference(P, insts, packed_dev, n, stride_expected, warm=None):
    # the existing, allocating entry point on the same orders
    prob = P.Problem(insts)
    assert prob.stride == stride_expected
    cost = torch.empty(n, dtype=torch.float32, device="cuda")
    status = torch.empty(n, dtype=torch.int32, device="cuda")
    traj = torch.empty((n, prob.stride), dtype=torch.float32, device="cuda")
    P.comet_eval_modes(prob.handle, packed_dev, n, warm, cost, traj, status)
    torch.cuda.synchronize()
    out = cost.cpu().numpy(), status.cpu().numpy(), traj.cpu().numpy()
    prob.close()
    return out


def test_noalloc_matches_allocating_entry_point_twice(P):
    insts = [W.push_l4_instance(21), W.push_l4_instance(22)]
    Nmax = 80
    stride = 7 * Nmax + 4
    stream = torch.cuda.current_stream()
    for call, (seed, n) in enumerate([(1, 700), (2, 257)]):
        seqs, idx = _orders(seed, n, insts)
        packed = P.pack_mode_seqs(seqs, idx)
        d = torch.from_numpy(packed.view(np.uint8).reshape(n, P.MODE_SEQ_BYTES)).cuda()
        cost = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
        status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        traj = torch.zeros((n, stride), dtype=torch.float32, device="cuda")
        P.comet_eval_modes_noalloc(insts, None, stream.cuda_stream, d, n, None, cost, traj, status)
        torch.cuda.synchronize()
        c, s, tr = cost.cpu().numpy(), status.cpu().numpy(), traj.cpu().numpy()
        rc, rs, rtr = _reference(P, insts, d, n, stride)
        # each TO is solved by one warp independently of the others, so the
        # two entry points agree to the bit; the comparison uses the cost and
        # state tolerances of the parity tests (1e-4 relative, 1e-3 absolute)
        np.testing.assert_array_equal(s, rs, err_msg=f"call {call}")
        np.testing.assert_allclose(c, rc, rtol=1e-4, atol=1e-7, err_msg=f"call {call}")
        np.testing.assert_allclose(tr, rtr, rtol=0, atol=1e-3, err_msg=f"call {call}")
        assert np.mean(s == P.TO_CONVERGED) > 0.5


def test_noalloc_rejects_what_it_cannot_hold(P):
    inst = W.push_l2_instance(0)
    n = 4
    packed = P.pack_mode_seqs(np.zeros((n, 2), np.uint8))
    d = torch.from_numpy(packed.view(np.uint8).reshape(n, P.MODE_SEQ_BYTES)).cuda()
    cost = torch.empty(n, dtype=torch.float32, device="cuda")
    status = torch.empty(n, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(P.CometError, match="64 instances"):
        P.comet_eval_modes_noalloc([inst] * 65, None, s, d, n, None, cost, None, status)
    with pytest.raises(P.CometError, match="device memory"):
        P.comet_eval_modes_noalloc([inst], None, s, packed, n, None, cost, None, status)


def test_noalloc_many_tos_per_warp_and_warm_starts(P):
    """4,000 TOs at N = 80 exceed the 1,308 warps whose stage records fit the
    fixed array, so warps take several TOs each from the work counter (the
    launch shape only this entry point uses).  Each TO is still solved by one
    warp with the same arithmetic, so the results equal the allocating entry
    point's bit for bit, cold and then warm-started from the first results."""
    insts = [W.push_l4_instance(23), W.push_l4_instance(24)]
    stride = 7 * 80 + 4
    n = 4000
    seqs, idx = _orders(3, n, insts)
    packed = P.pack_mode_seqs(seqs, idx)
    d = torch.from_numpy(packed.view(np.uint8).reshape(n, P.MODE_SEQ_BYTES)).cuda()
    s = torch.cuda.current_stream().cuda_stream
    warm = None
    for call in range(2):
        cost = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
        status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        traj = torch.zeros((n, stride), dtype=torch.float32, device="cuda")
        P.comet_eval_modes_noalloc(insts, None, s, d, n, warm, cost, traj, status)
        torch.cuda.synchronize()
        c, st, tr = cost.cpu().numpy(), status.cpu().numpy(), traj.cpu().numpy()
        rc, rs, rtr = _reference(P, insts, d, n, stride, warm)
        np.testing.assert_array_equal(st, rs, err_msg=f"call {call}")
        np.testing.assert_array_equal(c.view(np.uint32), rc.view(np.uint32), err_msg=f"call {call}")
        np.testing.assert_array_equal(tr.view(np.uint32), rtr.view(np.uint32), err_msg=f"call {call}")
        assert np.mean(st == P.TO_CONVERGED) > 0.5
        warm = traj  # the second call starts from the first call's solutions


def test_noalloc_rejects_too_large_n_max(P):
    """An instance whose N_max needs more shared memory per warp than a block
    can have is rejected with INVALID_ARG before anything runs."""
    inst = dict(W.push_l4_instance(25))
    inst["knots_per_segment"] = 256
    inst["max_segments"] = 16  # N_max = 4,096
    n = 2
    packed = P.pack_mode_seqs(np.zeros((n, 1), np.uint8))
    d = torch.from_numpy(packed.view(np.uint8).reshape(n, P.MODE_SEQ_BYTES)).cuda()
    cost = torch.empty(n, dtype=torch.float32, device="cuda")
    status = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(P.CometError, match="shared memory|too large"):
        P.comet_eval_modes_noalloc([inst], None, s, d, n, None, cost, None, status)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [-7, -7]  # nothing was launched
