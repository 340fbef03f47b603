"""The learned proposal on the bimanual task (507 modes per segment, 12
controls per interval), through the C ABI (include/comet_proposal.h), against
the FP64 oracle's restatement of its layout (oracle/mlp.py: bim_features,
bim_targets, bim_warm) and in use in front of Algorithm 1.

* Features bit for bit (factored one-hot of the 507 modes), training targets
  to FP32 rounding (forces in units of m g), the forward pass on the bimanual
  widths (in_dim 192, out_dim 1,088: the layered tensor-core GEMMs) within
  the bound of tests/test_gpu_mlp.py, and warm starts built from the
  predicted controls as the oracle builds them from the same outputs.
* Trained on evaluator results of training instances, the proposal ranks
  orders of held-out instances by merit better than an untrained network,
  and the learned planner returns certified plans from fewer evaluations
  than plain expansion with the same beam and rounds.
"""
import numpy as np
import pytest

import workloads as W
from oracle import mlp as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
spearmanr = pytest.importorskip("scipy.stats").spearmanr


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


def _dev(P, packed):
    return torch.from_numpy(packed.view(np.uint8).reshape(len(packed), P.MODE_SEQ_BYTES)).cuda()


def _orders(rng, n, lmax=6):
    return [tuple(int(m) for m in rng.integers(0, 507, rng.integers(1, lmax + 1))) for _ in range(n)]


def test_bimanual_dims_features_and_targets(P):
    insts = [W.bimanual_instance(0), W.bimanual_instance(1)]
    prob = P.Problem(insts)
    q = P.comet_proposal_create(prob.handle, {"dataset_cap": 400})
    din, width, dout, _ = P.comet_proposal_dims(q)
    n_max = max(i["knots_per_segment"] * i["max_segments"] for i in insts)
    assert (din, width, dout) == O.bim_dims(6, n_max)
    rng = np.random.default_rng(0)
    n = 333
    seqs = _orders(rng, n)
    idx = rng.integers(0, 2, n).astype(np.int32)
    packed = P.pack_mode_seqs(seqs, idx)
    x = torch.zeros((n, din), dtype=torch.int16, device="cuda")
    P.comet_proposal_features(q, packed, n, x)
    want = np.stack([O.bim_features(insts[i], s, 6, din) for s, i in zip(seqs, idx)])
    np.testing.assert_array_equal(x.cpu().numpy().view(np.uint16), O.bf16_bits(want))
    # targets of evaluator-shaped results
    stride = prob.stride
    assert stride == 17 * n_max + 5
    cost = rng.uniform(1.0, 40.0, n).astype(np.float32)
    viol = (rng.uniform(0, 1, n) ** 4 * 1e-3).astype(np.float32)
    status = rng.choice([0, 0, 0, 1, 2, 4], n).astype(np.int32)
    traj = (rng.normal(size=(n, stride)) * 5.0).astype(np.float32)
    P.comet_proposal_add_samples(q, packed, n, cost, viol, status, traj)
    got_T, got_O, got_X = P.proposal_dataset_rows(q, n)
    for i in range(n):
        N = insts[idx[i]]["knots_per_segment"] * len(seqs[i])
        ctrl = traj[i, 5 * (n_max + 1):].reshape(12, n_max).astype(np.float64)
        Tw, Ow = O.bim_targets(float(cost[i]), float(viol[i]), int(status[i]), ctrl, N, n_max, dout,
                               insts[idx[i]]["mass"])
        np.testing.assert_allclose(got_T[i], Tw, rtol=2e-6, atol=1e-7)
        np.testing.assert_allclose(got_O[i], Ow, rtol=1e-6, atol=0)
    np.testing.assert_array_equal(got_X, O.bf16_bits(want))
    P.comet_proposal_destroy(q)
    prob.close()


def test_bimanual_forward_and_warm_starts_match_the_oracle(P):
    insts = [W.bimanual_instance(2), W.bimanual_instance(3)]
    prob = P.Problem(insts)
    q = P.comet_proposal_create(prob.handle)
    din, width, dout, npar = P.comet_proposal_dims(q)
    ps = W.mlp_params(din, width, dout, 7, bias_scale=0.1)
    flat = O.flatten(ps).astype(np.float32)
    assert flat.size == npar
    P.comet_proposal_set_params(q, flat)
    params = O.unflatten(flat.astype(np.float64), din, width, dout)
    rng = np.random.default_rng(1)
    M = 300
    seqs = _orders(rng, M)
    idx = rng.integers(0, 2, M).astype(np.int32)
    packed = P.pack_mode_seqs(seqs, idx)
    X = np.stack([O.bim_features(insts[i], s, 6, din) for s, i in zip(seqs, idx)])
    y = np.zeros((M, dout), np.float32)
    P.comet_proposal_forward(q, O.bf16_bits(X), M, y)
    want, _ = O.forward(params, X, round_hidden=True)
    rms = np.sqrt(np.mean(want ** 2))
    err = np.abs(y - want) / (np.abs(want) + rms)
    assert np.max(err) <= 1e-2, np.max(err)
    # warm starts: the oracle's construction from the GPU's own outputs
    stride = prob.stride
    n_max = (stride - 5) // 17
    merit = np.zeros(M, np.float32)
    warm = np.zeros((M, stride), np.float32)
    P.comet_proposal_predict(q, packed, M, merit, warm)
    np.testing.assert_allclose(merit, np.exp(y[:, 0].astype(np.float64)), rtol=1e-5)
    for i in range(M):
        N = insts[idx[i]]["knots_per_segment"] * len(seqs[i])
        w = O.bim_warm(insts[idx[i]], N, n_max, y[i].astype(np.float64))
        np.testing.assert_allclose(warm[i], w, rtol=1e-5, atol=1e-6)
    P.comet_proposal_destroy(q)
    prob.close()


@pytest.fixture(scope="module")
def trained(P):
    """Trained on 64 bimanual instances (seeds 1000..1063, disjoint from the
    held-out seeds 40..), 768 random orders of 1..4 segments each, evaluated
    by the GPU evaluator."""
    n_inst, per = 64, 768
    insts = [W.bimanual_instance(1000 + s) for s in range(n_inst)]
    prob = P.Problem(insts)
    q = P.comet_proposal_create(prob.handle, {"dataset_cap": n_inst * per})
    rng = np.random.default_rng(2)
    seqs = _orders(rng, n_inst * per, lmax=4)
    idx = np.repeat(np.arange(n_inst, dtype=np.int32), per)
    packed = P.pack_mode_seqs(seqs, idx)
    for a in range(0, len(packed), 16384):
        d = _dev(P, packed[a:a + 16384])
        r = prob.eval(d, want_traj=True)
        P.comet_proposal_add_samples(q, d, len(d), r["cost"], r["viol"], r["status"], r["traj"])
    losses = np.concatenate([P.comet_proposal_train(q, 600, 2048, {"lr": 1e-3}, seed=1),
                             P.comet_proposal_train(q, 400, 2048, {"lr": 3e-4}, seed=2)])
    _, _, _, n = P.comet_proposal_dims(q)
    flat = np.zeros(n, np.float32)
    P.comet_proposal_get_params(q, flat)
    P.comet_proposal_destroy(q)
    prob.close()
    return flat, losses


def test_bimanual_training_and_ranking(P, trained):
    flat, losses = trained
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.5 * losses[:10].mean(), (losses[:10].mean(), losses[-50:].mean())
    # rank correlation of predicted and evaluated merit on a held-out
    # instance, trained against untrained parameters of the same shape
    inst = W.bimanual_instance(40)
    prob = P.Problem([inst])
    rng = np.random.default_rng(9)
    seqs = _orders(rng, 2048, lmax=4)
    packed = P.pack_mode_seqs(seqs)
    r = prob.eval(_dev(P, packed))
    m_true = r["cost"].cpu().numpy() + 100.0 * np.maximum(r["viol"].cpu().numpy() - 1e-5, 0.0)
    rho = {}
    for name, params in (("trained", flat), ("untrained", None)):
        q = P.comet_proposal_create(prob.handle)
        if params is not None:
            P.comet_proposal_set_params(q, params)
        m = np.zeros(len(seqs), np.float32)
        P.comet_proposal_predict(q, packed, len(seqs), m)
        P.comet_proposal_destroy(q)
        rho[name] = spearmanr(m, m_true).correlation
    prob.close()
    print(f"Spearman rank correlation with evaluated merit: {rho}")
    assert rho["trained"] > 0.5 and rho["trained"] > rho["untrained"] + 0.3


def test_bimanual_learned_planner(P, trained):
    flat, _ = trained
    seeds = P.pack_mode_seqs([(m,) for m in range(507)])
    rows = []
    for seed in range(40, 44):
        prob = P.Problem([W.bimanual_instance(seed)])
        plain = P.comet_plan(prob.handle, 0, seeds, 507, dict(k=16, batch=1024, rounds=3, k_ref=64))
        q = P.comet_proposal_create(prob.handle)
        P.comet_proposal_set_params(q, flat)
        learned = P.comet_plan(prob.handle, 0, seeds, 507, dict(k=16, batch=256, rounds=3, k_ref=64), proposal=q)
        P.comet_proposal_destroy(q)
        prob.close()
        rows.append((plain["best_cost"], learned["best_cost"], plain["evaluations"], learned["evaluations"],
                     plain["best_status"] == 0 and plain["best_viol"] <= 1e-5,
                     learned["best_status"] == 0 and learned["best_viol"] <= 1e-5))
        print(f"instance {seed}: plain {plain['best_cost']:.4f} ({plain['evaluations']} evaluations, "
              f"{plain['explore_ms'] + plain['refine_ms']:.0f} ms), learned {learned['best_cost']:.4f} "
              f"({learned['evaluations']}, {learned['explore_ms'] + learned['refine_ms']:.0f} ms)")
    rows = np.array(rows, dtype=float)
    assert np.all(rows[:, 5] >= rows[:, 4])          # a certified plan wherever plain expansion finds one
    assert np.all(rows[:, 3] < 0.6 * rows[:, 2])     # from far fewer evaluations


def test_batched_learned_planner_equals_one_instance_at_a_time(P, trained):
    # the batched planner runs the same algorithm: per instance the same
    # evaluated set, plan and cost as the single-instance learned planner
    flat, _ = trained
    insts = [W.bimanual_instance(s) for s in range(44, 48)]
    prob = P.Problem(insts)
    q = P.comet_proposal_create(prob.handle)
    P.comet_proposal_set_params(q, flat)
    one = [(m,) for m in range(507)]
    opts = dict(k=16, batch=256, rounds=3, k_ref=64)
    batched = P.comet_plan_batch(prob.handle, list(range(4)), [one] * 4, opts, proposal=q)
    for i in range(4):
        r = P.comet_plan(prob.handle, i, P.pack_mode_seqs(one, np.full(507, i, np.int32)), 507, opts, proposal=q)
        assert r["evaluations"] == batched[i]["evaluations"]
        assert r["best"] == batched[i]["best"] and r["best_cost"] == batched[i]["best_cost"]
    P.comet_proposal_destroy(q)
    prob.close()
