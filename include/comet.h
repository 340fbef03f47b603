/*
 * comet.h -- C ABI of the GB300 CoMET hot path.
 *
 * CoMET (Li & Chalvatzaki, "Contact-Rich Motion Planning via GPU-Parallel
 * Mode Evaluation") scores contact-mode orders m by solving one
 * mode-conditioned trajectory optimisation (TO) per order, Eq. mode_nlp
 *     J*(m) = min_z J(z, m)  s.t.  g(z, m) = 0,  h(z, m) <= 0,
 * returns the inexact mode value of Eq. inexact_mode_value
 *     J_hat = J(z_hat, m),  v_hat = max(|g|_inf, |[h]+|_inf)
 * and ranks orders by the merit of Eq. search_merit
 *     M_hat = J_hat + mu * max(v_hat - eps_feas, 0),
 * expanding the best ones by one-edit neighbourhoods (Sec. III-B,
 * Algorithm 1).
 *
 * Conventions for every entry point
 *   - All functions return a comet_status; call-level failures return an
 *     error code and set a thread-local message (comet_last_error()).
 *     Per-TO numerical failures never fail a call: they are reported in the
 *     per-TO status array (COMET_TO_*).
 *   - Buffers are owned by the caller.  A pointer argument may point to
 *     host memory or to device memory of the device the problem was created
 *     on; the library detects which (cudaPointerGetAttributes).  Device
 *     buffers are used in place and the call is asynchronous on the
 *     problem's stream; host buffers are staged through device memory owned
 *     by the problem, and the call returns after the results are copied
 *     back.
 *   - Trajectory layout (warm starts and outputs), one record of
 *     comet_traj_stride(problem) floats per TO, component-major and padded
 *     to N_max intervals:  x[N_max+1], y[N_max+1], theta[N_max+1],
 *     s[N_max+1], f_n[N_max], f_t[N_max], sdot[N_max]; only the first N+1
 *     states and N controls of a TO with N intervals are meaningful.
 *   - Mode code of an order (m_0 .. m_{L-1}) over an alphabet of M modes:
 *     code = L + sum_i (m_i + 1) (M + 1)^(i + 1)   (unsigned 64-bit).
 */
#ifndef COMET_H
#define COMET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    COMET_OK = 0,
    COMET_ERR_INVALID_ARG = 1, /* a null, negative or out-of-range argument */
    COMET_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    COMET_ERR_OOM = 3,         /* device memory could not be allocated */
    COMET_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
    COMET_ERR_BUDGET = 5,      /* a capacity (frontier, batch) is exhausted */
    COMET_ERR_INTERNAL = 6
} comet_status;

/* per-TO status (Sec. III-C "Stopping and scoring") */
enum {
    COMET_TO_CONVERGED = 0,   /* scaled feasibility, stationarity and complementarity met,
                                 and the FP64-certified v_hat <= eps_feas */
    COMET_TO_MAX_ITER = 1,    /* iteration budget exhausted (feasibility not implied) */
    COMET_TO_INFEASIBLE = 2,  /* FP32 stop test met but the FP64 certificate v_hat > eps_feas */
    COMET_TO_FACTOR_FAIL = 3, /* reserved: every step of the budget was rejected */
    COMET_TO_NONFINITE = 4    /* a non-finite value appeared in the iterate */
};

enum { COMET_TASK_PUSHER_SLIDER = 0, COMET_TASK_BIMANUAL = 1 };

#define COMET_MAX_SEGMENTS 16

/* One planning instance (Sec. III-A).  Pushing: a rectangular slider of
 * sides side_x x side_y [m] with an ellipsoidal limit surface of radius
 * c_ls [m] and force-to-velocity gain kappa, pusher friction mu, state
 * (x, y, theta, s), control (f_n, f_t, sdot), K = knots_per_segment
 * intervals of dt [s] per mode segment, orders of at most max_segments
 * segments over n_modes = 12 modes (face 0..3 x stick, slide+, slide-:
 * mode 3 face + kind) or n_modes = 13, where mode 12 is free motion
 * (Sec. III-A: the pusher is off the slider, the contact force is zero, the
 * slider rests, and the contact offset may jump across it; max_segments
 * <= 15 so that mode codes fit in 64 bits), cost w_terminal
 * |pose_N - goal|^2 + w_control sum_k |u_k|^2.
 * Bimanual (task 1): a box of width side_x and height side_y [m] and mass
 * `mass` [kg] in the vertical plane, hand friction mu, ground friction
 * ground_mu, state (x, z, theta, s_L, s_R), control (xd, zd, thd, fn_L, ft_L,
 * sd_L, fn_R, ft_R, sd_R, lam_n, lam_t, p_c), n_modes = 507 (ground stick /
 * slide / pivot x 13 x 13 hand modes: none or face 0..3 x stick, slide+,
 * slide-), cost w_terminal |pose_N - goal|^2 + w_control (|twist|^2 +
 * |sliding rates|^2 + p_c^2 + |forces|^2 / (m g)^2); trajectories
 * x[5][N_max+1] then u[12][N_max] (stride 17 N_max + 5).  A problem holds
 * instances of one task. */
typedef struct {
    int32_t task;
    int32_t knots_per_segment;
    int32_t max_segments;
    int32_t n_modes;
    double side_x, side_y, c_ls, mu, dt, kappa;
    double start[3], goal[3];
    double w_terminal, w_control;
    double mass, ground_mu; /* bimanual only */
} comet_instance_desc;

/* Solver options (Sec. III-C).  Zero-initialised fields take the defaults
 * returned by comet_default_opts(). */
typedef struct {
    int32_t max_iters;       /* exploration budget t_exp (default 300) */
    int32_t ref_iters;       /* refinement budget t_ref (default 1500) */
    double eps_feas;         /* feasibility tolerance on v_hat (1e-5) */
    double eps_primal;       /* scaled primal tolerance of the stop test (1e-6); the stop test
                                also holds every row within eps_feas / 2 in physical units */
    double eps_dual;         /* stationarity tolerance (1e-4), taken relative to the objective:
                                eps_dual * max(1, beta / beta_ref) * max(1, |J|) */
    double eps_comp;         /* complementarity tolerance (1e-6) */
    double merit_mu;         /* mu of Eq. search_merit (100) */
    double beta0, beta_max, beta_ref; /* penalty 1/mu_AL: start, cap, reference (100, 1e4, 1e3) */
    double rho0, rho_min;    /* proximal damping: start and lower bound (1e-4, 1e-4) */
    int32_t precision_flags; /* bit 0: one step of FP64 iterative refinement of the Riccati
                                solve while the penalty exceeds refine_beta (default on) */
    int32_t reserved;
    double refine_beta;      /* penalty above which the refinement runs (1e4; with the
                                default cap beta_max = 1e4 it is not reached) */
} comet_solver_opts;

/* One mode order: instance index, length and modes (40 bytes; 16-bit modes
 * so that alphabets beyond 256 modes, such as the bimanual 507, fit). */
typedef struct {
    int32_t instance;
    uint8_t len;
    uint8_t pad[3];
    uint16_t modes[COMET_MAX_SEGMENTS];
} comet_mode_seq;

typedef struct comet_problem comet_problem;
typedef struct comet_frontier comet_frontier;

/* Fill *opts with the defaults listed above. */
comet_status comet_default_opts(comet_solver_opts* opts);

/* Create a problem holding n_instances instance descriptors (copied) and
 * the solver options (copied; NULL = defaults) on the current CUDA device.
 * cuda_stream is a cudaStream_t (NULL = the legacy default stream).  The
 * problem owns its device scratch (descriptors, per-warp workspaces, staging
 * buffers).  Errors: INVALID_ARG for bad descriptors (non-positive sizes,
 * K * max_segments > 4096, max_segments > 16, n_modes not 12 or 13 for
 * pushing, max_segments > 15 with 13 modes),
 * CUDA / OOM from the runtime. */
comet_status comet_problem_create(const comet_instance_desc* inst, int32_t n_instances,
                                  const comet_solver_opts* opts, void* cuda_stream,
                                  comet_problem** out);

/* Release the problem and its device memory (synchronises its stream). */
comet_status comet_problem_destroy(comet_problem* p);

/* Floats per trajectory record: 7 * N_max + 4 with N_max the largest
 * K * max_segments over the instances. */
int64_t comet_traj_stride(const comet_problem* p);

/* Solve one mode-conditioned TO (Eq. mode_nlp) per order.
 *   mode_seqs   [n] orders (instance index < n_instances, 1 <= len <=
 *               max_segments of that instance, modes < n_modes); a TO with
 *               order length L has N = K * L intervals split evenly among
 *               the segments
 *   warm_starts [n][stride] floats or NULL for the cold start (zero
 *               controls, pose interpolated from start to goal, s = 0)
 *   out_cost    [n]  J_hat in physical units (FP64-certified, rounded to float)
 *   out_traj    [n][stride] returned trajectories, or NULL
 *   out_status  [n]  COMET_TO_*
 * The budget is opts.max_iters per TO.  Errors: INVALID_ARG (n < 0, null
 * required pointers, a malformed order -- checked on the host for host
 * buffers and on the device for device buffers, where the TO's status
 * becomes COMET_TO_NONFINITE and the call returns INVALID_ARG after the
 * stream is synchronised), CUDA, OOM. */
comet_status comet_eval_modes(comet_problem* p, const comet_mode_seq* mode_seqs, int64_t n,
                              const float* warm_starts, float* out_cost, float* out_traj,
                              int32_t* out_status);

/* Same as comet_eval_modes with an explicit iteration budget (e.g. the
 * refinement budget t_ref of Algorithm 1). */
comet_status comet_eval_modes_budget(comet_problem* p, const comet_mode_seq* mode_seqs, int64_t n,
                                     const float* warm_starts, int32_t max_iters, float* out_cost,
                                     float* out_traj, int32_t* out_status);

/* Per-TO diagnostics of the last comet_eval_modes call on this problem, all
 * nullable, each [n]: v_hat (FP64-certified, physical units), M_hat, the
 * number of iterations used and the FP64 stationarity residual
 * |grad J + A^T lambda|_inf.  Same host/device rules as comet_eval_modes. */
comet_status comet_eval_stats(comet_problem* p, float* out_viol, float* out_merit,
                              int32_t* out_iters, float* out_stat);

/* Failure report of the last evaluator launch on this problem (an addition
 * of this library, for callers that pass device arrays, where
 * comet_eval_modes returns before the launch ends).  Synchronises the
 * problem's stream and reads the launch's device flag into *out_flag
 * (nullable): 0 = nothing to report; 1 = a malformed order was met (its TO
 * carries COMET_TO_NONFINITE); 2 = a bounded device wait gave up (the
 * warm-start staging copy did not complete within about a second; the TO
 * carries COMET_TO_NONFINITE and NaN cost), in which case the call returns
 * COMET_ERR_TIMEOUT.  Device waits never hang: each gives up after its
 * bound and leaves the context usable.  comet_eval_modes with host arrays
 * makes the same check itself and returns COMET_ERR_TIMEOUT. */
comet_status comet_eval_check(comet_problem* p, int32_t* out_flag);

/* Test hook: with on != 0, the evaluator's launches on this problem do not
 * issue the warm-start staging copy, so the bounded wait for it runs out
 * (failure detection is tested on a wait that nothing completes; no copy is
 * left in flight).  Off by default; no production path sets it. */
comet_status comet_debug_stall_staging(comet_problem* p, int32_t on);

/* Solve one mode-conditioned TO per order without allocating any memory.
 * (An addition of this library; the paper has no counterpart.)
 *
 * For callers that cannot allocate device memory: code running inside a
 * memory pool or arena that owns all device memory of the process, real-time
 * loops where an allocation (and the synchronisation cudaMalloc / cudaFree
 * can imply) is not allowed after start-up, or hosts that forbid the CUDA
 * allocator.  No problem object is needed and nothing is allocated or freed:
 * the evaluator's scratch lives in one fixed 32 MiB device array inside the
 * library, which every device that loads the library holds until the
 * process exits.
 *   inst, n_instances  host descriptors, 1 <= n_instances <= 64 (more is
 *                      rejected with COMET_ERR_INVALID_ARG)
 *   opts               host options or NULL (defaults)
 *   cuda_stream        cudaStream_t of the launch (NULL = legacy stream)
 *   mode_seqs, warm_starts, out_cost, out_traj, out_status: as in
 *                      comet_eval_modes, but every array must be DEVICE
 *                      memory (nothing is staged; host pointers are rejected
 *                      with COMET_ERR_INVALID_ARG); the trajectory stride is
 *                      7 * N_max + 4 with N_max = max K * max_segments.
 * Asynchronous on cuda_stream: the call reads no host memory on the GPU
 * (the instance table travels as a kernel launch parameter) and does not
 * wait for the stream.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) with the current device; the first call on a device
 * may load the library's device code there, so make that first call before
 * any stream capture.  Every call shares the
 * array and it keeps the last call's contents (the work counter and error
 * flag are cleared by each call); calls whose kernels overlap on the GPU --
 * two streams or two host threads at once -- race on it and must be
 * serialised by the caller.  Orders too long for the array (N_max such that
 * four warps' stage records exceed it) are rejected with INVALID_ARG.
 * Per-TO diagnostics (comet_eval_stats) are not produced. */
comet_status comet_eval_modes_noalloc(const comet_instance_desc* inst, int32_t n_instances,
                                      const comet_solver_opts* opts, void* cuda_stream,
                                      const comet_mode_seq* mode_seqs, int64_t n, const float* warm_starts,
                                      float* out_cost, float* out_traj, int32_t* out_status);

/* ---- greedy local mode expansion (Sec. III-B, Algorithm 1) ----------- */

/* Create a frontier for one instance: the evaluated set V (up to capacity
 * orders, with their merits M_hat of Eq. search_merit) and the next batch
 * F_{s+1} (up to `batch` orders).  k_max bounds the beam k of comet_expand
 * (1 <= k_max <= 4096).  Owns device memory; errors INVALID_ARG, OOM. */
comet_status comet_frontier_create(comet_problem* p, int32_t instance, int64_t capacity, int32_t batch,
                                   int32_t k_max, comet_frontier** out);

/* Neighbourhood rules of the expansion (Sec. III-A, III-B). */
enum {
    COMET_GRAMMAR_NONE = 0, /* every order over the instance's modes, lengths 1..max_segments */
    COMET_GRAMMAR_PUSH = 1  /* the pushing task grammar over the 13-mode alphabet: modes are
                             * stick on face f (3 f) or free motion (12); an order starts in free
                             * motion, no two consecutive segments share a mode, and a direct
                             * contact-to-contact switch joins adjacent faces (0-1-2-3-0) */
};

/* comet_frontier_create with a neighbourhood rule: the expansion walks
 * N_r(m), the orders within `radius` (1 or 2) edits (insert, delete or
 * substitute one segment) of m whose intermediate orders are all admissible
 * under `grammar`, in enumeration order: the one-edit orders (substitutions,
 * insertions, deletions, by position and then alphabet position), then with
 * radius 2 the one-edit orders of each of them in that order.  The pushing
 * grammar needs a pushing instance with n_modes = 13.  Errors: INVALID_ARG
 * (as comet_frontier_create, a bad radius or grammar, or k_max times the
 * slots of one neighbourhood above 2^26). */
comet_status comet_frontier_create_ex(comet_problem* p, int32_t instance, int64_t capacity, int32_t batch,
                                      int32_t k_max, int32_t radius, int32_t grammar, comet_frontier** out);

comet_status comet_frontier_destroy(comet_frontier* f);

/* Add n evaluated orders to V with their J_hat (cost) and v_hat (viol); the
 * merit M_hat = J_hat + mu max(v_hat - eps_feas, 0) uses the problem's
 * options.  An order already in V is not added twice.  Host or device
 * arrays.  Errors: INVALID_ARG (an order of another instance, from host
 * memory), BUDGET (more than the capacity); device-side overflow or
 * malformed orders set the flags read by comet_frontier_size. */
comet_status comet_frontier_add(comet_frontier* f, const comet_mode_seq* seqs, int64_t n, const float* cost,
                                const float* viol);

/* One expansion round (Algorithm 1, lines 5-10): rank V by (M_hat, mode
 * code), walk the k best orders in that order and admit their unseen one-edit
 * neighbours (substitutions, then insertions, then deletions; positions and
 * modes ascending; orders in V or already admitted are skipped) until the
 * batch holds `batch` orders.  Asynchronous on the problem's stream; the
 * batch stays on the device (comet_frontier_next). */
comet_status comet_expand(comet_problem* p, comet_frontier* frontier, int32_t k);

/* Device pointer to the next batch F_{s+1} (valid until the next
 * comet_expand) and its size; synchronises the problem's stream. */
comet_status comet_frontier_next(comet_frontier* f, const comet_mode_seq** seqs, int64_t* n);

/* Copy the next batch into out (host or device, room for cap orders) and
 * return its size in *n; BUDGET if cap is too small; synchronises. */
comet_status comet_frontier_copy_next(comet_frontier* f, comet_mode_seq* out, int64_t cap, int64_t* n);

/* Checkpoint and resume of a frontier (an addition of this library): save
 * writes V (its mode codes and M_hat merits) and the pending batch F_{s+1}
 * to the file at `path` (a 56-byte header -- magic "COMETFV1", version 1,
 * instance, alphabet size, L_max, edit radius, grammar, capacity, |V|,
 * |F_{s+1}| -- then |V| u64 codes, |V| f32 merits and |F_{s+1}|
 * comet_mode_seq records, little-endian); load reads such a file into a
 * frontier of the same instance, alphabet, L_max and neighbourhood rule
 * with room for it, replacing its contents and rebuilding the hash set, so
 * that expansion continues as if never interrupted.  Both synchronous;
 * COMET_ERR_INVALID_ARG if the file cannot be opened, written or read, is
 * not a frontier checkpoint, or does not fit this frontier. */
comet_status comet_frontier_save(comet_frontier* f, const char* path);
comet_status comet_frontier_load(comet_frontier* f, const char* path);

/* |V| and the device-side error flags (bit 0 malformed order, bit 1 value 2
 * capacity exceeded); synchronises. */
comet_status comet_frontier_size(comet_frontier* f, int64_t* n_evaluated, int32_t* error_flags);

/* The k best orders of V by (M_hat, code): host arrays of mode codes (0 past
 * |V|) and merits; synchronises. */
comet_status comet_frontier_best(comet_frontier* f, int32_t k, uint64_t* out_codes, float* out_merit);

/* ---- the planner: Algorithm 1 on the device ---------------------------- */

typedef struct {
    int32_t k;          /* beam: expand the k best orders of V each round (64) */
    int32_t batch;      /* batch width B (4096) */
    int32_t rounds;     /* expansion rounds s_max (3) */
    int32_t k_ref;      /* refinement count K_ref (256) */
    int64_t budget;     /* evaluation budget, 0 = none; the last batch is truncated to fit */
    int32_t ref_iters;  /* refinement budget t_ref, 0 = the problem's ref_iters */
    int32_t use_graph;  /* capture one round (expand, evaluate, add) as a CUDA graph and replay it (1) */
    int32_t radius;     /* edit radius r of the neighbourhoods N_r (1; 2 allowed, see comet_frontier_create_ex) */
    int32_t grammar;    /* COMET_GRAMMAR_NONE (0) or COMET_GRAMMAR_PUSH: expand admissible orders only */
} comet_plan_opts;

typedef struct {
    comet_mode_seq best;  /* best refined feasible order (len 0 if none) */
    float best_cost;      /* its J_hat after refinement */
    float best_viol;      /* its v_hat */
    int32_t best_status;
    int32_t rounds_run;
    int64_t evaluations;  /* |V| after exploration */
    float explore_ms;     /* seed batch + rounds, device time */
    float refine_ms;      /* top-K_ref re-solve, device time */
} comet_plan_result;

comet_status comet_default_plan_opts(comet_plan_opts* po);

/* CoMET (Algorithm 1) for one instance: evaluate the seed batch F_0 with
 * budget t_exp, add it to V, then run `rounds` rounds of {expand the k best
 * orders of V into F_{s+1} (<= batch orders, <= budget evaluations in total),
 * evaluate F_{s+1}, add it to V} entirely on the device -- batch sizes never
 * return to the host, and with use_graph the round is one CUDA graph replayed
 * `rounds` times (an empty round is a no-op).  Then re-solve the K_ref best
 * orders of V with budget t_ref and return the best refined feasible order
 * (status CONVERGED, v_hat <= eps_feas).  seeds: host or device orders of
 * this instance; out_traj (nullable, host or device, comet_traj_stride
 * floats) receives the winner's trajectory.  Synchronises the stream. */
comet_status comet_plan(comet_problem* p, int32_t instance, const comet_mode_seq* seeds, int64_t n_seeds,
                        const comet_plan_opts* opts, comet_plan_result* out, float* out_traj);

/* ---- launch shape of the persistent evaluator and its autotuner ------- */

typedef struct {
    int32_t warps_per_block;    /* TOs per CTA (one warp per TO): 1..4 (default 4) */
    int32_t blocks_per_sm;      /* resident CTAs per SM the grid is sized for */
    int32_t max_blocks_per_sm;  /* occupancy limit of warps_per_block (get only) */
    int32_t unroll;             /* stages per trip of the evaluator's stage-parallel loops:
                                   1 or 2 (0 reads as 1) */
} comet_launch_config;

/* The problem's current launch shape. */
comet_status comet_get_launch_config(comet_problem* p, comet_launch_config* out);

/* Set the launch shape (warps_per_block in 1..4, blocks_per_sm in 1..the
 * occupancy limit, unroll 0, 1 or 2; INVALID_ARG otherwise).  Results never
 * depend on warps_per_block and blocks_per_sm: every shape solves each TO in
 * one warp with the same arithmetic.  The unrolled build of the stage loops
 * is the same solver compiled with other multiply-add contractions, so its
 * FP32 rounding differs.  Synchronises. */
comet_status comet_set_launch_config(comet_problem* p, const comet_launch_config* cfg);

/* Autotuner (no paper counterpart; the paper sizes its worker pool by hand):
 * times the evaluator on the n orders of `sample` (host or device) with an
 * iteration budget max_iters (0 = the solver's) under every candidate shape
 * -- 1..4 TOs per CTA, each at its occupancy limit and at three quarters of
 * it, each with the stage loops unrolled 1 and 2 times -- keeps the fastest
 * for p and caches it per (device, N_max) for problems created later in the
 * process.  out (nullable) receives the pick, out_ms (nullable, >= 16
 * floats) the time of each candidate in order, and n_candidates (nullable)
 * their number.  Synchronises. */
comet_status comet_autotune(comet_problem* p, const comet_mode_seq* sample, int64_t n, int32_t max_iters,
                            comet_launch_config* out, float* out_ms, int32_t* n_candidates);

/* Algorithm 1 for many instances at once: one frontier per instance; the
 * seed batches of all instances are evaluated in one persistent launch, and
 * each round expands every frontier and evaluates all next batches (opts->batch
 * slots per instance) in ONE persistent launch before each frontier adds its
 * results; the round is captured once as a CUDA graph (use_graph) and
 * replayed.  Refinement re-solves the K_ref best of every instance in one
 * launch.  seeds: host or device orders, instance i's in
 * [seed_offsets[i], seed_offsets[i+1]) (seed_offsets[0] = 0, each slice
 * non-empty, orders of instance instances[i]); out[i] as comet_plan, with
 * explore_ms and refine_ms the times of the whole batch.  Synchronises. */
comet_status comet_plan_batch(comet_problem* p, int32_t n_instances, const int32_t* instances,
                              const comet_mode_seq* seeds, const int64_t* seed_offsets, const comet_plan_opts* opts,
                              comet_plan_result* out);

/* The uniform-sampling search policy (a comparison policy on the same
 * evaluator): orders first .. first + n - 1 of a uniform sample of the
 * instance's order space -- every order of 1..max_segments segments
 * (COMET_GRAMMAR_NONE) or the admissible pushing orders (COMET_GRAMMAR_PUSH,
 * n_modes = 13).  Order i is the order at index draw_i mod T of the
 * (length, lexicographic) enumeration, T the number of orders and draw_i the
 * i-th output of SplitMix64 (Steele, Lea and Flood 2014) from `seed`
 * (state seed + (i + 1) * 0x9E3779B97F4A7C15).  The draws are independent
 * (with replacement); the first k distinct orders of the stream are a
 * uniform sample of k orders without replacement.  Uniform sampling
 * followed by refinement is comet_plan with the sample as seeds and
 * rounds = 0.  out:
 * host or device array of n records (host: synchronises).  Errors:
 * INVALID_ARG. */
comet_status comet_sample_orders(comet_problem* p, int32_t instance, uint64_t seed, int64_t first, int64_t n,
                                 int32_t grammar, comet_mode_seq* out);

/* Mode code of an order (see the conventions above); 0 if invalid. */
uint64_t comet_mode_code(const comet_mode_seq* seq, int32_t n_modes);

/* ---- timing optimisation (Sec. III-C, Sec. IV-A) --------------------- */

/* Bounds of the interval durations when timing is optimised. */
typedef struct {
    double h_min, h_max; /* bounds of every interval's duration h_k [s], 0 < h_min <= h_max */
    double T_max;        /* duration bound: sum_k h_k <= T_max [s], T_max > 0 */
} comet_timing_opts;

/* Solve the mode-conditioned TO of each order of a pushing problem with the
 * interval durations among the controls (Sec. III-C: with timing optimised
 * the interval durations join the controls; Sec. IV-A: an optimised time
 * step under the benchmark's duration bound).  Readings: interval k lasts
 * h_k, a fourth control bounded by h_min <= h_k <= h_max; the elapsed time
 * tau, a fifth state, carries the duration bound (tau_{k+1} = tau_k + h_k,
 * tau_0 = 0, tau_N <= T_max), which keeps the problem stage-wise; the
 * dynamics rows are (x_{k+1} - x_k - h_k f(x_k, u_k)) / sigma_i with the
 * fixed-step row scales; the cost is the fixed-step one (no term in h).
 * The method (PHR augmented Lagrangian, Newton step with the dynamics
 * curvature including the h cross terms and the Gauss-Newton fallback,
 * backward sweep, trial merits, multiplier and penalty updates, stop test,
 * FP64 certificate) is that of comet_eval_modes.
 *   mode_seqs, n: orders as in comet_eval_modes; malformed orders get
 *       COMET_TO_NONFINITE and a NaN cost;
 *   warm_starts: NULL (cold start: the fixed-step cold start, h_k = dt
 *       clipped into the bounds, tau_k = k h_0) or n records of
 *       9 N_max + 5 floats: x, y, theta, s, tau [N_max + 1] each, then
 *       f_n, f_t, sdot, h [N_max] each;
 *   max_iters: iteration budget (0 = the problem's max_iters);
 *   out_cost, out_status: [n]; out_traj: NULL or n records in the
 *       warm-start layout.
 * Every array must be device memory of the problem's device (host pointers
 * are rejected with INVALID_ARG); the call is asynchronous on the problem's
 * stream.  Per-TO diagnostics are then read with comet_eval_stats.  The
 * per-warp state lives in shared memory (about 1.2 + 0.19 N_max KB);
 * problems whose N_max does not fit are rejected with INVALID_ARG.
 * Errors: INVALID_ARG (NULL problem or timing, a bimanual problem, bounds
 * out of order, n < 0, host arrays, N_max too large), OOM / CUDA. */
comet_status comet_eval_modes_timed(comet_problem* p, const comet_timing_opts* timing,
                                    const comet_mode_seq* mode_seqs, int64_t n, const float* warm_starts,
                                    int32_t max_iters, float* out_cost, float* out_traj, int32_t* out_status);

/* ---- measurement (no paper counterpart) ------------------------------ */

/* FP32 FMA throughput of the current device, the peak of the evaluator's
 * roofline: one launch of a kernel whose threads each run 8 independent
 * fmaf chains (a grid of whole waves of resident 256-thread blocks) is timed
 * with CUDA events on cuda_stream after one untimed launch.  iters >= 1 is
 * the number of 128-FMA rounds per thread (a few thousand give ~10 ms);
 * out_scratch is device memory of comet_fp32_fma_peak_threads() floats that
 * receives one folded value per thread.  *out_tflops = 2 x FMAs / time,
 * *out_ms (nullable) the kernel time.  Synchronises the stream.  Errors:
 * INVALID_ARG, CUDA. */
comet_status comet_fp32_fma_peak(void* cuda_stream, int32_t iters, float* out_scratch, double* out_tflops,
                                 double* out_ms);

/* Threads of one comet_fp32_fma_peak launch on the current device (the
 * scratch size in floats), or -1 on a CUDA error. */
int32_t comet_fp32_fma_peak_threads(void);

/* Message of the last error on the calling thread ("" if none). */
const char* comet_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
