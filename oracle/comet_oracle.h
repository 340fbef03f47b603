/*
 * comet_oracle.h -- FP64 CPU oracle for the mode-conditioned trajectory
 * optimisation (TO) of CoMET (Li & Chalvatzaki, "Contact-Rich Motion
 * Planning via GPU-Parallel Mode Evaluation").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include,
 * link or call this file: only tests/, __graft_entry__.smoke() and the
 * bench's cpu_baseline / reference legs use it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * What it computes (paper Sec. III-A and III-C):
 *   - the quasi-static pusher-slider transcription with the fixed masked
 *     row layout of Sec. III-C "Shared representation across contact modes";
 *   - one mode-conditioned TO J*(m) (Eq. mode_nlp) solved locally by an
 *     augmented-Lagrangian Gauss-Newton method whose step is obtained by a
 *     backward sweep over the local systems
 *         S_k = H_k + rho_k I + beta A_k^T A_k        (beta = 1/mu_AL)
 *     factored by Cholesky without pivoting, with damping retries, a forward
 *     pass and parallel trial-step merits (Sec. III-C "Fixed-workspace local
 *     solves"), multiplier/penalty updates and the stop test of Sec. III-C
 *     "Stopping and scoring";
 *   - the inexact mode value (J_hat, v_hat) of Eq. inexact_mode_value in
 *     physical units and the merit M_hat of Eq. search_merit.
 * All arithmetic is IEEE double.  Layouts are plain arrays.
 */
#ifndef COMET_ORACLE_H
#define COMET_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* per-interval constraint rows, fixed positions (Sec. III-C, shared masked
 * representation): 0..3 dynamics defect d_k, 4 mode equality,
 * 5..10 inequalities (cone+, cone-, slide direction, -f_n, s-ell, -s-ell). */
#define ORC_NX 4
#define ORC_NU 3
#define ORC_NROW 11
#define ORC_NEQ 5
#define ORC_MAX_SEG 16
/* Pushing modes 0..11: face (mode / 3) x {stick, slide+, slide-} (mode % 3).
 * Mode 12: free motion (Sec. III-A: a contact changes faces only through a
 * free-motion segment): the pusher is off the slider (f_n = 0), the slider
 * rests and the contact offset is unconstrained. */
#define ORC_MODE_FREE 12

typedef struct {
    double side_x, side_y;   /* slider full side lengths [m] */
    double c_ls;             /* ellipsoidal limit-surface radius c [m] */
    double mu;               /* pusher-slider friction coefficient */
    double dt;               /* interval duration [s] */
    double kappa;            /* force-to-velocity gain of the limit surface */
    int32_t knots_per_segment;
    int32_t pad0;
    double start[3], goal[3];
    double w_terminal, w_control;
} orc_instance;

typedef struct {
    int32_t max_iters;        /* iteration budget t */
    int32_t max_factor_retries;
    int32_t n_alpha;          /* trial steps alpha = 2^-i, i < n_alpha (default 7) */
    int32_t max_inner;        /* inner iterations before a forced dual update */
    double beta0, beta_max, beta_growth;
    double rho0, rho_min, rho_max;
    double armijo_c1, ls_slack;
    double eps_primal, eps_dual, eps_comp;
    double omega_ratio;       /* inner tolerance omega = max(eps_dual, omega_ratio * viol) */
    double eta_ratio;         /* penalty grows if viol > eta_ratio * previous outer viol */
    double eps_feas;          /* feasibility tolerance for v_hat */
    double merit_mu;          /* mu of Eq. search_merit */
    double beta_ref;          /* stationarity tolerance eps_dual * max(1, beta / beta_ref) * max(1, |J|) */
    int32_t curv_skip;        /* after an indefinite Newton model, iterations that use Gauss-Newton only (3) */
    int32_t pad1;
} orc_opts;

enum { ORC_CONVERGED = 0, ORC_MAX_ITER = 1, ORC_INFEASIBLE = 2,
       ORC_FACTOR_FAIL = 3, ORC_NONFINITE = 4 };

typedef struct {
    double cost;      /* J_hat, physical units */
    double viol;      /* v_hat = max(|g|_inf, |[h]+|_inf), physical units */
    double merit;     /* M_hat = J_hat + mu max(v_hat - eps_feas, 0) */
    double stat;      /* |grad J + A^T lambda|_inf at the returned point */
    double comp;      /* max |lambda_i c_i| over inequality rows */
    double beta, rho;
    int32_t status;
    int32_t iters;
    int32_t n_outer;
    int32_t n_rejected;
    int32_t n_curv_fail;      /* Newton models found indefinite */
    int32_t pad1;
} orc_result;

void orc_default_opts(orc_opts* o);

/* Floating-point operations of the method counted on the calling thread
 * since the last reset (the counting build, -DORC_COUNT_FLOPS, only; 0
 * otherwise).  See comet_oracle.c for what is counted. */
uint64_t orc_flop_count(void);
void orc_flop_reset(void);

/* Stationarity tolerance of the stop test at penalty beta and objective
 * value `cost`: eps_dual * max(1, beta / beta_ref) * max(1, |cost|).  The
 * paper stops on scaled feasibility, stationarity and dual-residual
 * tolerances (Sec. III-C "Stopping and scoring"); row scaling leaves the
 * Lagrangian gradient unchanged, so the scaling read here is the
 * objective's: the test is relative to max(1, |J|).  The beta factor keeps
 * the test reachable in FP32 at large penalties. */
double orc_stat_tol(const orc_opts* opt, double beta, double cost);

/* Continuous dynamics f(x,u) of the quasi-static pusher-slider on `face`
 * and its Jacobians (row-major Fx[4][4], Fu[4][3]); any output may be NULL. */
void orc_dynamics(const orc_instance* in, int32_t face, const double* x, const double* u,
                  double* f, double* Fx, double* Fu);

/* Number of intervals and segment of interval k: N intervals are split
 * among `len` segments by seg(k) = floor(k*len/N). */
int32_t orc_segment_of(int32_t k, int32_t len, int32_t N);

/* Cold start of Sec. "Cold start": zero controls, pose interpolated from
 * start to goal, s = 0.  traj layout: component-major
 * x[N+1], y[N+1], th[N+1], s[N+1], fn[N], ft[N], sd[N]. */
void orc_cold_start(const orc_instance* in, int32_t N, double* traj);

/* Residual rows of every interval at traj: c[N][11] scaled values,
 * mask[N][11] (1 = row present), c_init[3]; physical row value =
 * c / scale, with scale[N][11].  Any output may be NULL. */
void orc_rows(const orc_instance* in, int32_t len, const uint8_t* modes, int32_t N,
              const double* traj, double* c, uint8_t* mask, double* scale, double* c_init);

/* Dense Jacobian of all rows w.r.t. z in interleaved order
 * z = [x_0, u_0, x_1, u_1, ..., u_{N-1}, x_N] (nz = 7N+4):
 * jac[(3 + 11N) x nz], rows ordered as init(3), then interval k rows 0..10.
 * Masked rows are zero.  For pins on tiny N only. */
void orc_dense_jacobian(const orc_instance* in, int32_t len, const uint8_t* modes, int32_t N,
                        const double* traj, double* jac);

/* One step by the backward (Riccati) sweep at (traj, lam, beta, rho);
 * lam layout: lam_init[3] then lam[N][11].  curvature = 1 adds the
 * Lagrangian curvature of the dynamics rows to the Gauss-Newton model.
 * Outputs the step dz in interleaved order and the AL gradient grad
 * (interleaved).  Returns 0 on success, -1 if a local Cholesky fails. */
int32_t orc_gn_step(const orc_instance* in, int32_t len, const uint8_t* modes, int32_t N,
                    const double* traj, const double* lam, double beta, double rho,
                    int32_t curvature, double* dz, double* grad);

/* AL merit L_A(z; lam, beta) and cost J at traj. */
double orc_al_merit(const orc_instance* in, int32_t len, const uint8_t* modes, int32_t N,
                    const double* traj, const double* lam, double beta, double* cost_out);

/* Solve one mode-conditioned TO.  warm (nullable) and out_traj use the
 * component-major layout; out_lam (nullable) receives 3 + 11N multipliers. */
int32_t orc_solve(const orc_instance* in, int32_t len, const uint8_t* modes, int32_t N,
                  const double* warm, const orc_opts* opt,
                  double* out_traj, double* out_lam, orc_result* res);

/* Solve n TOs on nthreads host threads (one TO per thread at a time).
 * inst_idx[n], lens[n], modes[n][lmax], Ns[n]; out_traj (nullable) has
 * stride traj_stride doubles per TO. */
int32_t orc_solve_batch(const orc_instance* insts, const int32_t* inst_idx,
                        const int32_t* lens, const uint8_t* modes, int32_t lmax,
                        const int32_t* Ns, int64_t n, const orc_opts* opt, int32_t nthreads,
                        double* out_traj, int64_t traj_stride, orc_result* res);

/* orc_solve_batch with optional warm starts (TO i starts from the
 * component-major trajectory at warm + i * warm_stride, in its own N, and
 * from the multipliers at warm_lam + i * lam_stride) and optional
 * multipliers out (3 + 11 N at out_lam + i * lam_stride). */
int32_t orc_solve_batch_ex(const orc_instance* insts, const int32_t* inst_idx, const int32_t* lens,
                           const uint8_t* modes, int32_t lmax, const int32_t* Ns, int64_t n, const orc_opts* opt,
                           int32_t nthreads, const double* warm, int64_t warm_stride, const double* warm_lam,
                           double* out_traj, int64_t traj_stride, double* out_lam, int64_t lam_stride,
                           orc_result* res);

/* orc_solve starting from the multipliers warm_lam (3 + 11 N; NULL = 0). */
int32_t orc_solve_ex(const orc_instance* in, int32_t len, const uint8_t* modes, int32_t N, const double* warm,
                     const double* warm_lam, const orc_opts* opt, double* out_traj, double* out_lam,
                     orc_result* res);

#ifdef __cplusplus
}
#endif
#endif
