"""The learned proposal in use: trained on the GPU on evaluator results, it
orders and prunes the expansion of Algorithm 1 and warm-starts the TOs; the
evaluator still solves and certifies every returned plan.

The ablation (the same planner with and without the proposal, on held-out
instances) checks what the trained network buys: plans as good as plain
expansion with far fewer evaluations, warm starts that save solver
iterations, and a ranking of orders by predicted merit that an untrained
network of the same shape does not have.  The pruning step itself is
checked against the oracle's forward pass of the same parameters.
"""
import numpy as np
import pytest

import workloads as W
from oracle import mlp as O
from oracle import search as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
spearmanr = pytest.importorskip("scipy.stats").spearmanr

EVERY = [(m,) for m in range(12)] + [tuple(s) for s in W.all_sequences(12, 2)] + \
    [tuple(s) for s in W.all_sequences(12, 3)] + [tuple(s) for s in W.all_sequences(12, 4)]
SEEDS = [(m,) for m in range(12)] + [tuple(s) for s in W.all_sequences(12, 2)]


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


@pytest.fixture(scope="module")
def trained(P):
    """Parameters trained on 256 random 4-segment pushing instances (seeds
    1000..1255, disjoint from the held-out seeds 48..63), 1,024 random
    orders each, evaluated by the GPU evaluator."""
    n_inst, per = 256, 1024
    insts = [W.push_l4_instance(1000 + s) for s in range(n_inst)]
    prob = P.Problem(insts)
    q = P.comet_proposal_create(prob.handle, {"dataset_cap": n_inst * per})
    rng = np.random.default_rng(0)
    pick = rng.integers(0, len(EVERY), size=n_inst * per)
    idx = np.repeat(np.arange(n_inst, dtype=np.int32), per)
    packed = P.pack_mode_seqs([EVERY[j] for j in pick], idx)
    for a in range(0, len(packed), 65536):
        d = _dev(P, packed[a:a + 65536])
        r = prob.eval(d, want_traj=True)
        P.comet_proposal_add_samples(q, d, len(d), r["cost"], r["viol"], r["status"], r["traj"])
    assert P.comet_proposal_dataset_size(q) == n_inst * per
    losses = np.concatenate([P.comet_proposal_train(q, 1000, 4096, {"lr": 1e-3}, seed=1),
                             P.comet_proposal_train(q, 500, 4096, {"lr": 3e-4}, seed=2),
                             P.comet_proposal_train(q, 500, 4096, {"lr": 1e-4}, seed=3)])
    _, _, _, n = P.comet_proposal_dims(q)
    flat = np.zeros(n, np.float32)
    P.comet_proposal_get_params(q, flat)
    P.comet_proposal_destroy(q)
    prob.close()
    return flat, losses


def test_training_reduces_the_loss(trained):
    _, losses = trained
    assert np.all(np.isfinite(losses))
    print(f"loss: first 10 {losses[:10].mean():.3f}, last 100 {losses[-100:].mean():.3f}")
    assert losses[-100:].mean() < 0.15 * losses[:10].mean()


def _ranking(P, flat, inst):
    prob = P.Problem([inst])
    packed = P.pack_mode_seqs(EVERY)
    d = _dev(P, packed)
    r = prob.eval(d)
    merit = r["merit"].cpu().numpy()
    q = P.comet_proposal_create(prob.handle)
    if flat is not None:
        P.comet_proposal_set_params(q, flat)
    pm = np.zeros(len(EVERY), np.float32)
    P.comet_proposal_predict(q, packed, len(EVERY), pm, None)
    P.comet_proposal_destroy(q)
    prob.close()
    ok = np.isfinite(merit)
    return spearmanr(np.log(pm[ok]), np.log(np.maximum(merit[ok], 1e-12))).correlation


def test_trained_ranking_beats_untrained(P, trained):
    flat, _ = trained
    for seed in (60, 61):
        inst = W.push_l4_instance(seed)
        rho_t = _ranking(P, flat, inst)
        rho_u = _ranking(P, None, inst)
        print(f"instance {seed}: Spearman trained {rho_t:.3f}, untrained {rho_u:.3f}")
        assert rho_t >= 0.4 and rho_t >= rho_u + 0.3


def test_warm_starts_save_iterations(P, trained):
    flat, _ = trained
    inst = W.push_l4_instance(60)
    prob = P.Problem([inst])
    d = _dev(P, P.pack_mode_seqs(EVERY))
    cold = {k: v.cpu().numpy() for k, v in prob.eval(d).items()}
    q = P.comet_proposal_create(prob.handle)
    P.comet_proposal_set_params(q, flat)
    warm = torch.empty((len(EVERY), prob.stride), dtype=torch.float32, device="cuda")
    P.comet_proposal_predict(q, d, len(EVERY), None, warm)
    w = {k: v.cpu().numpy() for k, v in prob.eval(d, warm=warm).items()}
    P.comet_proposal_destroy(q)
    prob.close()
    print(f"iterations cold {cold['iters'].mean():.1f}, warm {w['iters'].mean():.1f}; converged cold "
          f"{np.mean(cold['status'] == 0):.3f}, warm {np.mean(w['status'] == 0):.3f}")
    assert w["iters"].mean() < 0.95 * cold["iters"].mean()
    assert np.mean(w["status"] == 0) >= np.mean(cold["status"] == 0) - 0.01
    # the enumeration argmin (Eq. mode_selection) is the same order
    assert S.enumeration_argmin(w["cost"], w["viol"]) == S.enumeration_argmin(cold["cost"], cold["viol"])


def test_learned_planner_ablation(P, trained):
    # plain expansion (B = 4096) against the learned planner (the 512 best
    # neighbours by predicted merit, warm-started) on held-out instances
    flat, _ = trained
    ps = P.pack_mode_seqs(SEEDS)
    same, rows = 0, []
    for seed in range(48, 56):
        prob = P.Problem([W.push_l4_instance(seed)])
        plain = P.comet_plan(prob.handle, 0, ps, len(ps), dict(k=64, batch=4096, rounds=3, k_ref=256))
        q = P.comet_proposal_create(prob.handle)
        P.comet_proposal_set_params(q, flat)
        learned = P.comet_plan(prob.handle, 0, ps, len(ps), dict(k=64, batch=512, rounds=3, k_ref=256), proposal=q)
        P.comet_proposal_destroy(q)
        prob.close()
        assert learned["best_status"] == 0 and learned["best_viol"] <= 1e-5
        ok = learned["best_cost"] <= plain["best_cost"] * (1 + 1e-3) + 1e-9
        same += ok
        rows.append((plain["evaluations"], learned["evaluations"], plain["explore_ms"] + plain["refine_ms"],
                     learned["explore_ms"] + learned["refine_ms"]))
        print(f"instance {seed}: plain {plain['best_cost']:.5f} ({plain['evaluations']} evaluations, "
              f"{rows[-1][2]:.1f} ms), learned {learned['best_cost']:.5f} ({learned['evaluations']}, {rows[-1][3]:.1f} ms)")
    rows = np.array(rows)
    assert same >= 7, same                                   # same plan (within 1e-3) on >= 7 of 8
    assert np.all(rows[:, 1] < 0.6 * rows[:, 0])             # far fewer evaluations
    assert np.median(rows[:, 3]) < np.median(rows[:, 2])     # lower plan time


def test_prune_matches_the_oracle_ranking(P):
    # untrained (seeded) parameters: the kept batch is the `keep` best of the
    # frontier's candidates by the oracle's forward pass of the same
    # parameters, up to swaps of near-ties (BF16 arithmetic)
    inst = W.push_l4_instance(3)
    prob = P.Problem([inst])
    q = P.comet_proposal_create(prob.handle)
    din, width, dout, n = P.comet_proposal_dims(q)
    params = W.mlp_params(din, width, dout, 5, bias_scale=0.2)
    P.comet_proposal_set_params(q, O.flatten(params).astype(np.float32))
    f = P.comet_frontier_create(prob.handle, 0, 20000, 8192, 64)
    rng = np.random.default_rng(1)
    V = list({tuple(int(m) for m in rng.integers(0, 12, rng.integers(1, 4))) for _ in range(300)})
    merit = rng.uniform(0, 1, len(V)).astype(np.float32)
    P.comet_frontier_add(f, P.pack_mode_seqs(V), len(V), merit, np.zeros(len(V), np.float32))
    P.comet_expand(prob.handle, f, 16)
    cand = P.frontier_next_orders(f, 8192)
    keep = 200
    P.comet_proposal_prune(q, f, keep)
    kept = P.frontier_next_orders(f, 8192)
    assert len(kept) == min(keep, len(cand)) and len(set(kept)) == len(kept) and set(kept) <= set(cand)
    X = np.stack([O.features(inst, s, 4, din) for s in cand])
    y, _ = O.forward(params, X)
    pred = y[:, 0]
    order = sorted(range(len(cand)), key=lambda i: (pred[i], S.encode(cand[i], 12)))
    want = [cand[i] for i in order[:keep]]
    # in the order of the proposal's own predictions (ties by mode code)
    pm = np.zeros(len(kept), np.float32)
    P.comet_proposal_predict(q, P.pack_mode_seqs(kept), len(kept), pm, None)
    keys = [(float(np.log(m)), S.encode(s, 12)) for m, s in zip(pm, kept)]
    assert all(keys[i][0] <= keys[i + 1][0] + 1e-6 for i in range(len(keys) - 1))
    # identical except where the oracle's scores are within BF16 noise
    thresh = pred[order[keep - 1]]
    for s in set(want) ^ set(kept):
        assert abs(pred[cand.index(s)] - thresh) <= 2e-2 * (abs(thresh) + 1), s
    P.comet_frontier_destroy(f)
    P.comet_proposal_destroy(q)
    prob.close()
