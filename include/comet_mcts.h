/* comet_mcts.h -- Monte Carlo tree search over mode orders (C ABI).
 *
 * A comparison search policy on the same evaluator (Sec. IV-A and IV-B of
 * the paper): UCT with exploration constant c = 0.8, virtual loss and random
 * rollouts; P orders at a time go to the evaluator; the reward of an order is
 * J_best / J_hat when it is feasible (v_hat <= eps_feas) and 0 otherwise
 * (Sec. IV-A), or M_best / M_hat with M_hat the merit of Eq. search_merit
 * (Sec. IV-B), where J_best (M_best) is the least over the orders evaluated
 * so far.
 *
 * The search itself is host code (a tree of order prefixes); the evaluator
 * solves each pool of orders on the GPU.  It runs in two forms:
 *   - ask / tell: comet_mcts_ask returns the next pool, the caller evaluates
 *     it by any means (comet_eval_modes, or a batch of several searches) and
 *     reports the results with comet_mcts_tell;
 *   - comet_plan_mcts: the whole plan for one instance of a problem -- ask,
 *     evaluate, tell until the evaluation budget is spent or every order has
 *     been evaluated, then the K_ref best orders by merit are refined as in
 *     Algorithm 1 (comet_plan with those orders as seeds and no expansion
 *     round).
 *
 * The tree (the paper gives only the ingredients above; these are this
 * library's readings):
 *   - a node is a prefix of an order.  Its actions, in slot order, are
 *     "stop" (slot 0: the prefix is the order; prefixes of length >= 1) and
 *     "append mode a_j" (slot 1 + j, j over the alphabet in ascending order;
 *     when the prefix is shorter than l_max and, under COMET_GRAMMAR_PUSH,
 *     the extended prefix is admissible).  The alphabet is 0..n_modes-1, or
 *     {0, 3, 6, 9, 12} (sticking on each face, free motion) under the
 *     pushing grammar, whose admissible orders start in free motion, never
 *     repeat a mode and switch contact only between adjacent faces;
 *   - selection: from the root, while the node has no untried action, move
 *     to the child of largest  w / n + c sqrt(ln n_parent / n)  among the
 *     children that are not exhausted (ties: the lowest slot);
 *   - expansion: the untried action at index draw mod (number untried), in
 *     slot order, becomes a child;
 *   - rollout: from that child, each step takes the available action at
 *     index draw mod (number available) until "stop"; a "stop" child is its
 *     own order;
 *   - virtual loss: each node on the path gets its visit at selection time
 *     and its reward when the order's result is known: at once for an order
 *     evaluated before, else when the pool holding it is told (an order
 *     already waiting in the pool adds its path to that entry);
 *   - a pool holds distinct orders not evaluated before, at most P, and the
 *     evaluations never exceed max_evals;
 *   - exhaustion: a "stop" child is exhausted when created, any other node
 *     once it has no untried action and all its children are exhausted;
 *     selection never enters an exhausted child, so with a large enough
 *     budget every order is evaluated exactly once;
 *   - at tell time J_best (M_best) is first updated with the whole pool,
 *     then the waiting paths receive their rewards (pool order, then arrival
 *     order);
 *   - draws: draw_i = output i of SplitMix64 (Steele, Lea and Flood 2014)
 *     from `seed` (state seed + (i + 1) * 0x9E3779B97F4A7C15), one counter
 *     for the whole search, in the order expansion, then rollout steps.
 * Arithmetic is IEEE double throughout (no contraction), so a search is a
 * deterministic function of its options and the told results.
 *
 * Errors: functions return a comet_status and set comet_last_error().
 */
#ifndef COMET_MCTS_H
#define COMET_MCTS_H

#include <stdint.h>

#include "comet.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct comet_mcts comet_mcts;

enum {
    COMET_MCTS_REWARD_FEASIBLE = 0, /* J_best / J_hat if v_hat <= eps_feas, else 0 (Sec. IV-A) */
    COMET_MCTS_REWARD_MERIT = 1     /* M_best / M_hat (Sec. IV-B) */
};

typedef struct {
    int32_t n_modes;   /* size of the mode alphabet (13 under COMET_GRAMMAR_PUSH); (n_modes + 1)^(l_max + 1)
                          must stay below 2^64 (the mode code) */
    int32_t l_max;     /* longest order, 1..COMET_MAX_SEGMENTS */
    int32_t grammar;   /* COMET_GRAMMAR_NONE or COMET_GRAMMAR_PUSH */
    int32_t reward;    /* COMET_MCTS_REWARD_* */
    int64_t max_evals; /* evaluation budget, 0 = none (the search ends when every order is evaluated) */
    uint64_t seed;     /* SplitMix64 seed */
    double c_uct;      /* exploration constant c (0.8) */
    double eps_feas;   /* feasibility threshold on v_hat (1e-5) */
    double merit_mu;   /* mu of Eq. search_merit (100) */
    double max_ms;     /* comet_plan_mcts only: no further pool is asked for once the search has run this
                          long (wall time, milliseconds; the pool in flight completes); 0 = no time cap */
} comet_mcts_opts;     /* 64 bytes */

typedef struct {
    int64_t evaluations; /* orders told so far */
    int64_t tree_nodes;  /* nodes of the tree, the root included */
    int64_t pending;     /* orders of the last pool not told yet */
    int32_t exhausted;   /* 1 once every order has been claimed */
    int32_t reserved;
    double best;         /* J_best or M_best so far (+inf if none) */
} comet_mcts_stats;      /* 40 bytes */

/* Defaults: n_modes 12, l_max 4, no grammar, feasibility reward, no budget,
 * seed 0, c = 0.8, eps_feas 1e-5, mu 100, no time cap. */
comet_status comet_mcts_default_opts(comet_mcts_opts* o);

/* A search over the orders of 1..l_max segments.  Host memory only; no GPU
 * call.  Errors: INVALID_ARG (n_modes outside 1..65535, l_max outside
 * 1..16, the code overflow above, grammar PUSH with n_modes != 13, an
 * unknown reward kind, c_uct < 0 or not finite, max_evals < 0, max_ms < 0
 * or not finite), OOM. */
comet_status comet_mcts_create(const comet_mcts_opts* o, comet_mcts** out);
comet_status comet_mcts_destroy(comet_mcts* t);

/* The next pool: up to `pool` orders written to the host array out (record
 * `instance` in each), their number to *n; *n = 0 when the budget is spent
 * or every order has been evaluated.  The pool must be told before the next
 * ask (INVALID_ARG otherwise; also for pool < 1 or null pointers). */
comet_status comet_mcts_ask(comet_mcts* t, int32_t instance, int64_t pool, comet_mode_seq* out, int64_t* n);

/* Results of the last pool, in its order: cost[i] = J_hat and viol[i] =
 * v_hat of order i (host arrays of n floats; non-finite values count as
 * infeasible).  INVALID_ARG when n differs from the pool's size. */
comet_status comet_mcts_tell(comet_mcts* t, const float* cost, const float* viol, int64_t n);

comet_status comet_mcts_get_stats(const comet_mcts* t, comet_mcts_stats* out);

/* The k evaluated orders of least (M_hat, mode code) -- the ranking of
 * Algorithm 1's refinement -- as mode codes (host array of k), optionally
 * with their merits; *n = min(k, evaluations). */
comet_status comet_mcts_best(const comet_mcts* t, int64_t k, uint64_t* codes, double* merits, int64_t* n);

/* MCTS plan for one instance of problem p: the search runs over that
 * instance's alphabet and segment cap (o->n_modes and o->l_max are taken
 * from the instance; o->grammar, reward, seed, c_uct, max_evals and max_ms from o;
 * eps_feas and merit_mu from the problem's solver options), each pool is
 * evaluated with comet_eval_modes (budget t_exp), and the po->k_ref best
 * orders by merit are then refined with comet_plan (those orders as seeds,
 * rounds = 0, po->ref_iters).  out as comet_plan; out->evaluations counts the
 * search's evaluations, out->rounds_run its pools, out->explore_ms is the
 * search's wall time (host search and GPU evaluation) plus the seeds'
 * re-evaluation inside comet_plan, out->refine_ms the refinement's device
 * time.  The search stops at the first of: the budget max_evals, every
 * order evaluated, the time cap max_ms (checked before each pool).  out_traj
 * as comet_plan.  Synchronises.  Errors: INVALID_ARG (pool < 1, bad options,
 * max_evals = 0 and max_ms = 0 with more than 2^22 orders in the space), and
 * those of comet_eval_modes and comet_plan. */
comet_status comet_plan_mcts(comet_problem* p, int32_t instance, const comet_mcts_opts* o, int64_t pool,
                             const comet_plan_opts* po, comet_plan_result* out, float* out_traj);

#ifdef __cplusplus
}
#endif

#endif
