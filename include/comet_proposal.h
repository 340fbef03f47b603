/* comet_proposal.h -- the learned proposal of the CoMET hot path (C ABI).
 *
 * The paper has no learned part.  This is a cost and warm-start predictor in
 * front of the greedy expansion of Algorithm 1 (Sec. III-B): a 4-layer MLP
 * (width 256, GELU, BF16 weights and activations, FP32 accumulation on the
 * tensor cores) maps an (instance, mode order) pair to
 *   y[0]                 = log M_hat, the log of the order's merit
 *                          (Eq. search_merit), and
 *   y[1 + c N_max + k]   = control component c (f_n, f_t, s_dot) of interval
 *                          k of the order's solved trajectory (Eq. mode_nlp).
 * It is trained on the GPU on (order, evaluator result) samples, orders and
 * prunes the neighbours an expansion round generates, and warm-starts their
 * TOs.  The evaluator (comet_eval_modes) still solves and certifies every
 * returned plan.
 *
 * Input features of an order of length L (in_dim = 12 + 13 L_max rounded
 * up to a multiple of 64, zero padded): start pose (x, y, theta), goal pose,
 * 10 side_x, 10 side_y, the goal in the start frame (3 R(-theta_s)(g - s)
 * for x and y, theta_g - theta_s), one zero, then for each slot i < L_max a
 * 13-way one-hot (entries 0..11 = mode m_i, entry 12 = blank when i >= L).
 * out_dim = 1 + 3 N_max rounded up to a multiple of 16.
 *
 * Bimanual problems (COMET_TASK_BIMANUAL): the mode m = 169 g + 13 h_L +
 * h_R enters as a factored one-hot of 30 entries per slot (ground g at
 * 0..2, left hand at 3..15, right hand at 16..28, blank at 29), so in_dim =
 * 12 + 30 L_max rounded up to 64; the instance part is the start pose
 * (x, z, theta), the goal pose, 10 side_x, 10 side_y, 3 (x_g - x_s),
 * 3 (z_g - z_s), theta_g - theta_s and the mass.  The outputs are log M_hat
 * and the 12 controls of every interval, y[1 + c N_max + k] for c = xd, zd,
 * thd, fn_L, ft_L, sd_L, fn_R, ft_R, sd_R, lam_n, lam_t, p_c, with the six
 * forces in units of the box's weight m g (g = 9.81 m/s^2); out_dim = 1 +
 * 12 N_max rounded up to 16.  Warm starts take the cold start's poses (hand
 * offsets 0) with the predicted controls (warm_mode 0 is read as 1).
 *
 * Parameters (flat FP32 vector, the optimiser's master copy):
 *   [W_1 (width x in_dim), b_1, W_2 (width x width), b_2, W_3, b_3,
 *    W_4 (out_dim x width), b_4], W row-major [out][in].
 * Forward: Z_l = H_{l-1} W_l^T + b_l, H_l = GELU(Z_l) (tanh form:
 * 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))) for
 * l = 1..3 with H_0 = X; Y = H_3 W_4^T + b_4.  X, W and H_l are BF16.
 * Inference runs the four layers in one persistent kernel (the activations
 * stay in shared memory and TMEM); training runs them as separate GEMMs.
 * Loss of a batch of B rows: L = (1/B) sum_{b,j} Omega_bj (Y_bj - T_bj)^2.
 * Optimiser: AdamW with bias-corrected moments and decoupled weight decay.
 *
 * Conventions as in comet.h: calls run on the problem's stream; pointers
 * marked "host or device" are detected, others must be device memory.
 */
#ifndef COMET_PROPOSAL_H
#define COMET_PROPOSAL_H

#include <stdint.h>

#include "comet.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct comet_proposal comet_proposal;

typedef struct {
    int32_t width;         /* hidden width (256) */
    int32_t rows_cap;      /* rows of one forward / training batch held at once (4096); grown by calls */
    int64_t dataset_cap;   /* samples the proposal's training set can hold (0 = none) */
    uint64_t seed;         /* weight initialisation: U(-1/sqrt(fan_in), 1/sqrt(fan_in)), zero biases */
    double lambda_w;       /* weight of the control loss (1.0): Omega = lambda_w / (n_u N) per control */
    int32_t warm_mode;     /* warm-start states: 0 = Euler rollout of the predicted controls from
                              the start pose (s reset to 0 at a face change), 1 = the cold start's
                              poses (1; fewer solver iterations in measurements) */
    int32_t reserved;
} comet_proposal_desc;

typedef struct {
    double lr, beta1, beta2, eps, weight_decay;  /* (1e-3, 0.9, 0.999, 1e-8, 0) */
} comet_adamw_opts;

void comet_default_proposal_desc(comet_proposal_desc* d);
void comet_default_adamw_opts(comet_adamw_opts* o);

/* Create a proposal for problem p's instances (pushing: n_modes 12 or 13;
 * bimanual: 507; L_max and N_max of the problem).  The problem must outlive
 * it.  Errors: INVALID_ARG for a bad descriptor, CUDA / OOM from the
 * runtime. */
comet_status comet_proposal_create(comet_problem* p, const comet_proposal_desc* d, comet_proposal** out);
comet_status comet_proposal_destroy(comet_proposal* q);

/* Sizes: in_dim, width, out_dim and the number of parameters (any may be NULL). */
comet_status comet_proposal_dims(const comet_proposal* q, int32_t* in_dim, int32_t* width, int32_t* out_dim,
                                 int64_t* n_params);

/* Replace the parameters with `flat` (n_params floats, host or device) and
 * reset the optimiser (moments and step count).  Synchronous. */
comet_status comet_proposal_set_params(comet_proposal* q, const float* flat);

/* Copy the parameters and (if not NULL) the gradient of the last training
 * step into host or device buffers of n_params floats.  Synchronous. */
comet_status comet_proposal_get_params(comet_proposal* q, float* flat, float* grad);

/* Checkpoint and resume (an addition of this library).  save writes the
 * parameters, both AdamW moments and the step count to the file at `path`
 * (a 48-byte header -- magic "COMETPR1", version 1, in_dim, width, out_dim,
 * the task layout, n_params, the step count -- then 3 x n_params floats,
 * little-endian); load reads such a file into a proposal of the same layout
 * (in_dim, width, out_dim, task), so that training continues exactly where
 * it stopped.  The training set is not part of the file.  Both synchronous;
 * COMET_ERR_INVALID_ARG if the file cannot be opened, written or read, is not
 * a checkpoint, or holds another layout (the proposal is then unchanged). */
comet_status comet_proposal_save(comet_proposal* q, const char* path);
comet_status comet_proposal_load(comet_proposal* q, const char* path);

/* Features of n orders (host or device seqs) into out_x [n][in_dim] BF16
 * bit patterns (device).  Orders of another instance index than the
 * problem's are an error (host) or zero rows (device). */
comet_status comet_proposal_features(comet_proposal* q, const comet_mode_seq* seqs, int64_t n, uint16_t* out_x);

/* Forward pass: x [n][in_dim] BF16 (host or device) -> out_y [n][out_dim]
 * FP32 (host or device). */
comet_status comet_proposal_forward(comet_proposal* q, const uint16_t* x, int64_t n, float* out_y);

/* Device time of the forward pass (the kernels only): x [n][in_dim] BF16
 * (host or device) is copied once, then `reps` forward passes run back to
 * back on the problem's stream between two CUDA events; *out_ms receives the
 * mean per pass.  Synchronous. */
comet_status comet_proposal_time_forward(comet_proposal* q, const uint16_t* x, int64_t n, int32_t reps,
                                         float* out_ms);

/* One training step on a given batch: forward, loss, backward, AdamW.
 * x [n][in_dim] BF16, target and weight [n][out_dim] FP32 (host or device);
 * out_loss (nullable, host) receives L before the update.  With lr = 0 the
 * parameters stay and the gradient is left for comet_proposal_get_params.
 * n <= rows_cap is required during stream capture. */
comet_status comet_proposal_train_batch(comet_proposal* q, const uint16_t* x, const float* target,
                                        const float* weight, int64_t n, const comet_adamw_opts* o,
                                        float* out_loss);

/* Append evaluator results to the training set (all device pointers, or all
 * host): orders, and comet_eval_modes' cost, status and trajectory with
 * comet_eval_stats' v_hat.  Targets: T_0 = log max(M_hat, 1e-12) with
 * M_hat = J_hat + merit_mu max(v_hat - eps_feas, 0), weight 1 unless the TO
 * is NONFINITE; controls of CONVERGED TOs with weight lambda_w / (n_u N)
 * (n_u = 3 pushing, 12 bimanual, forces in units of m g), all other weights
 * 0.  Errors: BUDGET when the set is full. */
comet_status comet_proposal_add_samples(comet_proposal* q, const comet_mode_seq* seqs, int64_t n,
                                        const float* cost, const float* viol, const int32_t* status,
                                        const float* traj);

/* Number of samples in the training set. */
comet_status comet_proposal_dataset_size(comet_proposal* q, int64_t* n);

/* Copy rows [first, first + n) of the training set: features out_x
 * [n][in_dim] BF16 bits, targets out_t and weights out_w [n][out_dim] FP32
 * (host or device; each nullable).  Synchronous. */
comet_status comet_proposal_dataset_rows(comet_proposal* q, int64_t first, int64_t n, uint16_t* out_x,
                                         float* out_t, float* out_w);

/* `steps` AdamW steps on mini-batches of `batch` samples drawn uniformly
 * with replacement from the training set (counter-based hash of seed, step
 * and row); one step is captured once as a CUDA graph and replayed.
 * out_loss (nullable, host) receives the loss of every step.  Synchronous. */
comet_status comet_proposal_train(comet_proposal* q, int64_t steps, int32_t batch, const comet_adamw_opts* o,
                                  uint64_t seed, float* out_loss);

/* Predictions for n orders (host or device): out_merit [n] = exp(y_0)
 * (nullable), out_warm [n][comet_traj_stride] (nullable) = a warm start in
 * comet_eval_modes' layout built from the predicted controls (warm_mode). */
comet_status comet_proposal_predict(comet_proposal* q, const comet_mode_seq* seqs, int64_t n, float* out_merit,
                                    float* out_warm);

/* Order and prune the next batch of a frontier (after comet_expand): the
 * candidates are ranked by predicted merit (ties by mode code), the best
 * `keep` are kept in that order and out_warm (device, [keep][stride],
 * nullable) receives their warm starts.  Stays on the device. */
comet_status comet_proposal_prune(comet_proposal* q, comet_frontier* f, int32_t keep, float* out_warm);

/* Algorithm 1 with the proposal (see comet_plan in comet.h for the options
 * and the result): the seed batch is warm-started by the proposal; each round
 * generates the whole one-edit neighbourhood of the k best orders of V, keeps
 * the opts->batch (<= 4096) best by predicted merit, warm-starts and
 * evaluates them, and adds them to V; the K_ref best of V are re-solved
 * from the cold start as in comet_plan, so the evaluator alone scores the
 * returned plan.  Synchronises the stream. */
comet_status comet_plan_learned(comet_problem* p, int32_t instance, const comet_mode_seq* seeds, int64_t n_seeds,
                                const comet_plan_opts* opts, comet_proposal* q, comet_plan_result* out,
                                float* out_traj);

/* comet_plan_batch (comet.h) with the proposal: Algorithm 1 over several
 * instances of p, each round's evaluations of all instances in one launch;
 * every instance's seeds are warm-started by the proposal, and in every
 * round each instance's whole one-edit neighbourhood of its k best orders
 * is ranked by predicted merit and the opts->batch (<= 4096) best are kept
 * and warm-started, as in comet_plan_learned.  The proposal must have been
 * created for p.  Outputs and synchronisation as comet_plan_batch. */
comet_status comet_plan_batch_learned(comet_problem* p, int32_t n_instances, const int32_t* instances,
                                      const comet_mode_seq* seeds, const int64_t* seed_offsets,
                                      const comet_plan_opts* opts, comet_proposal* q, comet_plan_result* out);

/* ---- raw BF16 tensor-core GEMM (device pointers) --------------------------
 * D[M][N] = A[M][K] B[N][K]^T with A, B row-major BF16 (leading dimensions
 * lda, ldb in elements, multiples of 8, 16-byte aligned bases), FP32
 * accumulation, and one fused epilogue. */
enum {
    COMET_GEMM_STORE = 0,      /* out_f32 = D + bias */
    COMET_GEMM_BIAS_GELU = 1,  /* out_f32 = Z = D + bias; out_bf16 = GELU(Z); out_bf16_t = its transpose */
    COMET_GEMM_GELU_GRAD = 2,  /* out_bf16 = D * GELU'(z_in); out_bf16_t = its transpose */
    COMET_GEMM_ATOMIC_ADD = 3  /* out_f32 += D, K split into k_splits chunks */
};

typedef struct {
    int32_t kind;
    int32_t k_splits;          /* >= 1; > 1 only with COMET_GEMM_ATOMIC_ADD */
    const float* bias;         /* [N] or NULL */
    float* out_f32;            /* [M][ld_f32] */
    int64_t ld_f32;
    uint16_t* out_bf16;        /* [M][ld_bf16] or NULL */
    int64_t ld_bf16;
    uint16_t* out_bf16_t;      /* [N][ld_bf16_t] or NULL */
    int64_t ld_bf16_t;
    const float* z_in;         /* [M][ld_z] (GELU_GRAD) */
    int64_t ld_z;
} comet_gemm_epilogue;

comet_status comet_gemm_bf16(const uint16_t* a, int64_t lda, const uint16_t* b, int64_t ldb, int64_t m, int32_t n,
                             int32_t k, const comet_gemm_epilogue* ep, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* COMET_PROPOSAL_H */
