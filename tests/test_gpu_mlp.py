"""The learned proposal's BF16 tensor-core kernels against the FP64 oracle
(oracle/mlp.py), through the C ABI (include/comet_proposal.h).

* The GEMM (tcgen05 + TMA + TMEM) against an FP64 matmul of the same BF16
  operands, for ragged M, N and K (partial tiles, N > 256, K not a multiple
  of 64) and every fused epilogue.  Bound: FP32 accumulation of K products,
  |D - D64| <= 2^-22 sum_k |a_k b_k| + 1e-30 (K terms, each rounding at most
  one FP32 ulp of the running sum), and BF16 outputs within one BF16 ulp.
* Forward, loss and gradients of the 4-layer MLP against the oracle run on
  the same BF16 operands with the GPU's BF16 storage of activations and
  layer gradients mirrored (round_hidden): outputs within 1e-2 relative
  (floor: the output's RMS),
  gradients with cosine >= 0.999 and relative L2 error <= 1e-2 per tensor.
* One AdamW step against the oracle's AdamW applied to the GPU's gradient.
* Features and training targets bit for bit / to FP32 rounding.
"""
import numpy as np
import pytest

import workloads as W
from oracle import mlp as O

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


def _bf16_dev(x):
    """(device uint16 tensor of bf16 bits, fp64 values)"""
    bits = O.bf16_bits(x)
    return torch.from_numpy(bits.view(np.int16)).cuda(), O.from_bf16_bits(bits)


def _to_np_bf16(t):
    return O.from_bf16_bits(t.cpu().numpy().view(np.uint16))


GEMM_SHAPES = [(128, 256, 64), (1, 16, 64), (300, 256, 256), (257, 48, 100), (4096, 256, 256), (1000, 544, 64),
               (20736, 256, 64), (129, 200, 320)]


@pytest.mark.parametrize("M,N,K", GEMM_SHAPES)
def test_gemm_store_bias(P, M, N, K):
    # rows start on 16-byte boundaries: the leading dimension is K rounded up
    # to 8 elements, the padding holds NaN (never read)
    rng = np.random.default_rng(M * 7 + N + K)
    ld = (K + 7) // 8 * 8
    A = np.full((M, ld), np.nan)
    A[:, :K] = rng.normal(size=(M, K))
    B = np.full((N, ld), np.nan)
    B[:, :K] = rng.normal(size=(N, K))
    a, a64 = _bf16_dev(A)
    b, b64 = _bf16_dev(B)
    a64, b64 = a64[:, :K], b64[:, :K]
    bias = rng.normal(size=N).astype(np.float32)
    out = torch.full((M, N), np.nan, dtype=torch.float32, device="cuda")
    P.comet_gemm_bf16(a, ld, b, ld, M, N, K, kind=P.GEMM_STORE, bias=torch.from_numpy(bias).cuda(), out_f32=out,
                      ld_f32=N)
    got = out.cpu().numpy().astype(np.float64)
    want = a64 @ b64.T + bias
    bound = 2.0 ** -22 * (np.abs(a64) @ np.abs(b64).T) * K ** 0.5 + 2.0 ** -23 * np.abs(bias) + 1e-30
    assert np.all(np.abs(got - want) <= bound + 1e-6 * np.abs(want)), np.max(np.abs(got - want) / (bound + 1e-30))


def test_gemm_leading_dimensions_and_padding_never_read(P):
    # operands inside larger buffers whose padding holds NaN: a GEMM that
    # reads past K or past the rows would return NaN
    M, N, K, lda, ldb = 200, 96, 72, 136, 80
    rng = np.random.default_rng(3)
    A = np.full((M + 5, lda), np.nan)
    A[:M, :K] = rng.normal(size=(M, K))
    B = np.full((N + 3, ldb), np.nan)
    B[:N, :K] = rng.normal(size=(N, K))
    a, a64 = _bf16_dev(A)
    b, b64 = _bf16_dev(B)
    out = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    P.comet_gemm_bf16(a, lda, b, ldb, M, N, K, kind=P.GEMM_STORE, out_f32=out, ld_f32=N)
    got = out.cpu().numpy()
    want = a64[:M, :K] @ b64[:N, :K].T
    assert np.all(np.isfinite(got))
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-4)


@pytest.mark.parametrize("M,N,K", [(300, 256, 64), (130, 64, 256)])
def test_gemm_bias_gelu_epilogue(P, M, N, K):
    rng = np.random.default_rng(11)
    a, a64 = _bf16_dev(rng.normal(size=(M, K)) * 0.3)
    b, b64 = _bf16_dev(rng.normal(size=(N, K)) * 0.3)
    bias = (rng.normal(size=N) * 0.1).astype(np.float32)
    ldt = 384
    z = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    h = torch.zeros((M, N), dtype=torch.int16, device="cuda")
    ht = torch.zeros((N, ldt), dtype=torch.int16, device="cuda")
    P.comet_gemm_bf16(a, K, b, K, M, N, K, kind=P.GEMM_BIAS_GELU, bias=torch.from_numpy(bias).cuda(), out_f32=z,
                      ld_f32=N, out_bf16=h, ld_bf16=N, out_bf16_t=ht, ld_bf16_t=ldt)
    z_want = a64 @ b64.T + bias
    np.testing.assert_allclose(z.cpu().numpy(), z_want, rtol=1e-5, atol=1e-5)
    hv = _to_np_bf16(h)
    # H = bf16(GELU(Z)) of the GPU's own Z: one bf16 ulp (2^-8 relative)
    # plus the hardware tanh's error (relative 2^-10.987 on t, so at most
    # 0.5 |z| 2^-10.9 on GELU)
    zz = z.cpu().numpy().astype(np.float64)
    hw = O.gelu(zz)
    assert np.all(np.abs(hv - hw) <= 2.0 ** -8 * np.abs(hw) + 0.5 * np.abs(zz) * 2.0 ** -10.9 + 1e-6)
    np.testing.assert_array_equal(ht.cpu().numpy()[:, :M], h.cpu().numpy().T)


def test_gemm_gelu_grad_epilogue(P):
    M, N, K = 257, 256, 256
    rng = np.random.default_rng(12)
    a, a64 = _bf16_dev(rng.normal(size=(M, K)) * 0.1)
    b, b64 = _bf16_dev(rng.normal(size=(N, K)) * 0.1)
    zin = rng.normal(size=(M, N)).astype(np.float32)
    g = torch.zeros((M, N), dtype=torch.int16, device="cuda")
    gt = torch.zeros((N, 384), dtype=torch.int16, device="cuda")
    P.comet_gemm_bf16(a, K, b, K, M, N, K, kind=P.GEMM_GELU_GRAD, out_bf16=g, ld_bf16=N, out_bf16_t=gt, ld_bf16_t=384,
                      z_in=torch.from_numpy(zin).cuda(), ld_z=N)
    z64 = zin.astype(np.float64)
    acc = a64 @ b64.T
    want = acc * O.gelu_grad(z64)
    got = _to_np_bf16(g)
    scale = np.abs(a64) @ np.abs(b64).T * np.abs(O.gelu_grad(z64))
    # GELU' from the hardware tanh (relative 2^-10.9 on t):
    # |d GELU'| <= |dt| (0.5 + |z| |t| a (1 + 3 b z^2)) with |t| <= 1
    dgrad = 2.0 ** -10.9 * (0.5 + np.abs(z64) * O.GELU_A * (1 + 3 * O.GELU_B * z64 ** 2))
    assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 1e-5 * scale + np.abs(acc) * dgrad + 1e-7)
    np.testing.assert_array_equal(gt.cpu().numpy()[:, :M], g.cpu().numpy().T)


@pytest.mark.parametrize("splits", [1, 4, 16])
def test_gemm_split_k_atomic(P, splits):
    M, N, K = 256, 64, 4096
    rng = np.random.default_rng(splits)
    a, a64 = _bf16_dev(rng.normal(size=(M, K)))
    b, b64 = _bf16_dev(rng.normal(size=(N, K)))
    base = rng.normal(size=(M, N)).astype(np.float32)
    out = torch.from_numpy(base.copy()).cuda()
    P.comet_gemm_bf16(a, K, b, K, M, N, K, kind=P.GEMM_ATOMIC_ADD, k_splits=splits, out_f32=out, ld_f32=N)
    want = base + a64 @ b64.T
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-5, atol=2e-3)


def test_gemm_rejects_bad_arguments(P):
    a = torch.zeros((128, 64), dtype=torch.int16, device="cuda")
    out = torch.zeros((128, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(P.CometError):
        P.comet_gemm_bf16(a, 60, a, 64, 128, 16, 64, out_f32=out, ld_f32=16)   # lda not a multiple of 8
    with pytest.raises(P.CometError):
        P.comet_gemm_bf16(a, 64, a, 64, 128, 16, 64, kind=P.GEMM_STORE, k_splits=2, out_f32=out, ld_f32=16)
    with pytest.raises(P.CometError):
        P.comet_gemm_bf16(a.cpu(), 64, a, 64, 128, 16, 64, out_f32=out, ld_f32=16)  # host operand


# ---------------------------------------------------------------- the MLP

def _problem(P, lmax=4, K=20):
    inst = W.push_l4_instance(0)
    inst["max_segments"] = lmax
    inst["knots_per_segment"] = K
    return P.Problem([inst, W.push_l4_instance(1)]), [inst, W.push_l4_instance(1)]


def _params(P, q, seed, bias_scale=0.1):
    din, width, dout, n = P.comet_proposal_dims(q)
    ps = W.mlp_params(din, width, dout, seed, bias_scale=bias_scale)
    flat = O.flatten(ps).astype(np.float32)
    assert flat.size == n
    P.comet_proposal_set_params(q, flat)
    return O.unflatten(flat.astype(np.float64), din, width, dout), (din, width, dout)


def test_features_bit_exact(P):
    prob, insts = _problem(P)
    q = P.comet_proposal_create(prob.handle)
    din, width, dout, _ = P.comet_proposal_dims(q)
    assert (din, width, dout) == (64, 256, 256)
    rng = np.random.default_rng(0)
    seqs = [tuple(int(m) for m in rng.integers(0, 12, rng.integers(1, 5))) for _ in range(333)]
    idx = rng.integers(0, 2, len(seqs)).astype(np.int32)
    packed = P.pack_mode_seqs(seqs, idx)
    x = torch.zeros((len(seqs), din), dtype=torch.int16, device="cuda")
    P.comet_proposal_features(q, packed, len(seqs), x)
    want = np.stack([O.features(insts[i], s, 4, din) for s, i in zip(seqs, idx)])
    np.testing.assert_array_equal(x.cpu().numpy().view(np.uint16), O.bf16_bits(want))
    P.comet_proposal_destroy(q)
    prob.close()


@pytest.mark.parametrize("M", [1, 200, 4096])
def test_forward_matches_oracle(P, M):
    prob, insts = _problem(P)
    q = P.comet_proposal_create(prob.handle)
    params, (din, width, dout) = _params(P, q, seed=M)
    rng = np.random.default_rng(M)
    X = rng.normal(size=(M, din))
    xb = O.bf16_bits(X)
    y = np.zeros((M, dout), np.float32)
    P.comet_proposal_forward(q, xb, M, y)
    want, _ = O.forward(params, X, round_hidden=True)
    # 1e-2 relative, with the output's RMS as the floor: a hidden activation
    # whose FP32 and FP64 pre-activations straddle a BF16 rounding boundary
    # is stored one BF16 ulp (2^-8) apart, which moves outputs near zero by
    # about 2^-8 of a typical output
    rms = np.sqrt(np.mean(want ** 2))
    err = np.abs(y - want) / (np.abs(want) + rms)
    assert np.max(err) <= 1e-2, np.max(err)
    assert np.median(np.abs(y - want) / (np.abs(want) + 1e-2)) <= 1e-3
    P.comet_proposal_destroy(q)
    prob.close()


def _cos(a, b):
    return float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))


@pytest.mark.parametrize("M", [64, 1000, 4096])
def test_gradients_match_oracle(P, M):
    prob, insts = _problem(P)
    q = P.comet_proposal_create(prob.handle)
    params, (din, width, dout) = _params(P, q, seed=100 + M)
    rng = np.random.default_rng(M + 1)
    X = rng.normal(size=(M, din))
    T = rng.normal(size=(M, dout))
    Om = rng.uniform(0, 1, size=(M, dout)) * (rng.uniform(size=(M, dout)) < 0.5)
    Om[:, 0] = 1.0
    loss = P.comet_proposal_train_batch(q, O.bf16_bits(X), T.astype(np.float32), Om.astype(np.float32), M,
                                        {"lr": 0.0})
    n = sum(W_.size + b_.size for W_, b_ in params)
    flat, grad = np.zeros(n, np.float32), np.zeros(n, np.float32)
    P.comet_proposal_get_params(q, flat, grad)
    Yw, cache = O.forward(params, X, round_hidden=True)
    want_loss = O.loss(Yw, T, Om)
    assert loss == pytest.approx(want_loss, rel=1e-2)
    grads = O.backward(params, cache, Yw, T, Om, round_hidden=True)
    got = O.unflatten(grad.astype(np.float64), din, width, dout)
    for l in range(4):
        for g_got, g_want in zip(got[l], grads[l]):
            rel = np.linalg.norm(g_got - g_want) / np.linalg.norm(g_want)
            assert _cos(g_got, g_want) >= 0.999 and rel <= 1e-2, (l, rel)
    # lr = 0 leaves the parameters unchanged
    np.testing.assert_array_equal(flat, O.flatten(params).astype(np.float32))
    P.comet_proposal_destroy(q)
    prob.close()


def test_adamw_step_matches_oracle(P):
    prob, insts = _problem(P)
    q = P.comet_proposal_create(prob.handle)
    params, (din, width, dout) = _params(P, q, seed=7)
    M = 512
    rng = np.random.default_rng(9)
    X, T = rng.normal(size=(M, din)), rng.normal(size=(M, dout))
    Om = np.ones((M, dout)) * 0.01
    n = sum(W_.size + b_.size for W_, b_ in params)
    p0 = O.flatten(params)
    opts = {"lr": 1e-3, "weight_decay": 0.01}
    m = v = np.zeros(n)
    p = p0.copy()
    for t in (1, 2, 3):
        P.comet_proposal_train_batch(q, O.bf16_bits(X), T.astype(np.float32), Om.astype(np.float32), M, opts)
        flat, grad = np.zeros(n, np.float32), np.zeros(n, np.float32)
        P.comet_proposal_get_params(q, flat, grad)
        # the oracle's AdamW on the GPU's gradient of this step
        p, m, v = O.adamw(p, grad.astype(np.float64), m, v, t, 1e-3, wd=0.01)
        np.testing.assert_allclose(flat, p, rtol=0, atol=1e-6)
        p = flat.astype(np.float64)
    P.comet_proposal_destroy(q)
    prob.close()


def test_targets_from_evaluator_results(P):
    prob, insts = _problem(P)
    q = P.comet_proposal_create(prob.handle, {"dataset_cap": 1000})
    din, width, dout, _ = P.comet_proposal_dims(q)
    rng = np.random.default_rng(5)
    n = 300
    seqs = [tuple(int(m) for m in rng.integers(0, 12, rng.integers(1, 5))) for _ in range(n)]
    idx = rng.integers(0, 2, n).astype(np.int32)
    packed = P.pack_mode_seqs(seqs, idx)
    stride = prob.stride
    cost = rng.uniform(0.01, 2.0, n).astype(np.float32)
    viol = (rng.uniform(0, 1, n) ** 4 * 1e-3).astype(np.float32)
    status = rng.choice([0, 0, 0, 1, 2, 4], n).astype(np.int32)
    traj = rng.normal(size=(n, stride)).astype(np.float32)
    P.comet_proposal_add_samples(q, packed, n, cost, viol, status, traj)
    assert P.comet_proposal_dataset_size(q) == n
    Tw = np.zeros((n, dout))
    Ow = np.zeros((n, dout))
    Nmax = 80
    for i in range(n):
        N = 20 * len(seqs[i])
        ctrl = traj[i, 4 * (Nmax + 1):].reshape(3, Nmax).astype(np.float64)
        Tw[i], Ow[i] = O.targets(float(cost[i]), float(viol[i]), int(status[i]), ctrl, N, Nmax, dout)
    got_T, got_O, got_X = P.proposal_dataset_rows(q, n)
    np.testing.assert_allclose(got_T, Tw, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(got_O, Ow, rtol=1e-6, atol=0)
    Xw = np.stack([O.features(insts[i], s, 4, din) for s, i in zip(seqs, idx)])
    np.testing.assert_array_equal(got_X, O.bf16_bits(Xw))
    P.comet_proposal_add_samples(q, packed, n, cost, viol, status, traj)
    P.comet_proposal_add_samples(q, packed, n, cost, viol, status, traj)
    with pytest.raises(P.CometError):       # 1,200 > dataset_cap
        P.comet_proposal_add_samples(q, packed, n, cost, viol, status, traj)
    assert P.comet_proposal_dataset_size(q) == 3 * n
    P.comet_proposal_destroy(q)
    prob.close()


def test_fused_forward_agrees_with_the_layered_training_pass(P):
    # inference runs the four layers in one persistent tcgen05 kernel;
    # training runs them as separate GEMMs: the loss of the fused outputs
    # equals the training step's loss on the same batch
    prob, insts = _problem(P)
    q = P.comet_proposal_create(prob.handle)
    params, (din, width, dout) = _params(P, q, seed=31)
    M = 3000
    rng = np.random.default_rng(31)
    X = rng.normal(size=(M, din))
    T = rng.normal(size=(M, dout)).astype(np.float32)
    Om = (rng.uniform(size=(M, dout)) < 0.3).astype(np.float32)
    y = np.zeros((M, dout), np.float32)
    P.comet_proposal_forward(q, O.bf16_bits(X), M, y)
    loss_fused = float(np.sum(Om.astype(np.float64) * (y.astype(np.float64) - T) ** 2) / M)
    loss_layered = P.comet_proposal_train_batch(q, O.bf16_bits(X), T, Om, M, {"lr": 0.0})
    assert loss_layered == pytest.approx(loss_fused, rel=1e-5)
    P.comet_proposal_destroy(q)
    prob.close()


def test_fused_forward_at_pruning_size(P):
    # 20,736 rows (162 tiles over the SMs, several tiles per CTA): sampled
    # rows against the oracle
    prob, insts = _problem(P)
    q = P.comet_proposal_create(prob.handle)
    params, (din, width, dout) = _params(P, q, seed=32)
    M = 20736
    rng = np.random.default_rng(32)
    X = rng.normal(size=(M, din))
    y = np.zeros((M, dout), np.float32)
    P.comet_proposal_forward(q, O.bf16_bits(X), M, y)
    rows = np.sort(rng.choice(M, 300, replace=False))
    want, _ = O.forward(params, X[rows], round_hidden=True)
    rms = np.sqrt(np.mean(want ** 2))
    assert np.max(np.abs(y[rows] - want) / (np.abs(want) + rms)) <= 1e-2
    assert np.all(np.isfinite(y))
    P.comet_proposal_destroy(q)
    prob.close()


def test_checkpoint_resumes_training_exactly(P, tmp_path):
    # two proposals over the same training set: the second loads the first's
    # checkpoint after some training steps, and both then continue with the
    # same batches; parameters, moments and step count were all restored, so
    # the two stay together up to the order of the training step's atomic
    # sums (about 1e-6 relative), far below what restarting the optimiser
    # moves (asserted last)
    prob, insts = _problem(P)
    rng = np.random.default_rng(7)
    n = 600
    seqs = [tuple(int(m) for m in rng.integers(0, 12, rng.integers(1, 5))) for _ in range(n)]
    idx = rng.integers(0, 2, n).astype(np.int32)
    packed = P.pack_mode_seqs(seqs, idx)
    stride = prob.stride
    cost = rng.uniform(0.01, 2.0, n).astype(np.float32)
    viol = (rng.uniform(0, 1, n) ** 4 * 1e-3).astype(np.float32)
    status = rng.choice([0, 0, 0, 1, 2], n).astype(np.int32)
    traj = rng.normal(size=(n, stride)).astype(np.float32)
    qa = P.comet_proposal_create(prob.handle, {"dataset_cap": n})
    qb = P.comet_proposal_create(prob.handle, {"dataset_cap": n})
    for q in (qa, qb):
        P.comet_proposal_add_samples(q, packed, n, cost, viol, status, traj)
    P.comet_proposal_train(qa, 40, 256, {"lr": 1e-3}, seed=1)
    path = str(tmp_path / "proposal.ckpt")
    P.comet_proposal_save(qa, path)
    P.comet_proposal_load(qb, path)
    _, _, _, npar = P.comet_proposal_dims(qa)
    a, b = np.zeros(npar, np.float32), np.zeros(npar, np.float32)
    P.comet_proposal_get_params(qa, a)
    P.comet_proposal_get_params(qb, b)
    np.testing.assert_array_equal(a, b)
    la = P.comet_proposal_train(qa, 25, 256, {"lr": 1e-3}, seed=2)
    lb = P.comet_proposal_train(qb, 25, 256, {"lr": 1e-3}, seed=2)
    np.testing.assert_allclose(lb, la, rtol=1e-5)
    P.comet_proposal_get_params(qa, a)
    P.comet_proposal_get_params(qb, b)
    np.testing.assert_allclose(b, a, rtol=1e-4, atol=1e-6)
    # a proposal whose moments were reset takes a different step
    qc = P.comet_proposal_create(prob.handle, {"dataset_cap": n})
    P.comet_proposal_add_samples(qc, packed, n, cost, viol, status, traj)
    P.comet_proposal_load(qc, path)
    P.comet_proposal_get_params(qc, b)
    P.comet_proposal_set_params(qc, b)   # same weights, optimiser reset
    lc = P.comet_proposal_train(qc, 25, 256, {"lr": 1e-3}, seed=2)
    assert np.max(np.abs(lc - la) / np.abs(la)) > 1e-3
    # files that are not checkpoints of this layout are refused
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"not a checkpoint" * 8)
    with pytest.raises(P.CometError):
        P.comet_proposal_load(qb, str(bad))
    raw = open(path, "rb").read()
    (tmp_path / "short.ckpt").write_bytes(raw[: len(raw) // 2])
    with pytest.raises(P.CometError):
        P.comet_proposal_load(qb, str(tmp_path / "short.ckpt"))
    for q in (qa, qb, qc):
        P.comet_proposal_destroy(q)
    prob.close()
