/*
 * bimanual.h -- FP64 CPU oracle of the bimanual variant of the CoMET hot
 * path: quasi-static flipping of a box in the vertical plane with two point
 * hands and a ground contact.  TEST INFRASTRUCTURE ONLY (see
 * comet_oracle.h); it shares no code with the CUDA library.
 *
 * The paper's bimanual task (Sec. IV-B, Experiment 2) uses an L-shaped block
 * whose geometry is not given; this is the simplified box model of the
 * hot-path scope, in the shared masked row layout of Sec. III-C:
 *
 * state x = (x, z, theta, s_L, s_R): box pose (centre, counter-clockwise
 *   angle) and the two hands' contact offsets along their faces;
 * control u = (xd, zd, thd, fn_L, ft_L, sd_L, fn_R, ft_R, sd_R, lam_n,
 *   lam_t, p_c): the box twist, each hand's normal / tangential force and
 *   sliding rate, the ground force and its centre-of-pressure offset
 *   (horizontal, from the box centre);
 * kinematics x_{k+1} = x_k + dt (xd, zd, thd, sd_L, sd_R) (explicit Euler);
 * physics as constraints: quasi-static wrench balance of gravity, the hand
 *   wrenches and the ground wrench, plus the rows of the contact modes.
 *
 * Mode of a segment (507 = 3 x 13 x 13): m = g * 169 + h_L * 13 + h_R,
 *   ground g: 0 stick (no motion), 1 slide (horizontal translation,
 *   friction on the cone edge opposing the motion), 2 pivot about the
 *   lower-left corner (body (-a_x, -a_z));
 *   hand h: 0 none (zero force), 1 + 3 f + kind for face f = 0..3 (inward
 *   normals (1,0), (0,1), (-1,0), (0,-1) in the body frame, as in pushing)
 *   and kind 0 stick, 1 slide+, 2 slide-.
 *
 * Rows per interval (32, fixed positions; masked rows are zero):
 *   0..4  kinematic defects (rows 3, 4 masked when that hand changes face)
 *   5..7  wrench balance: F_x / mg, (F_z - mg) / mg, torque / (mg l)
 *   8..10 ground equalities, 11..15 ground inequalities
 *   16..18 hand L equalities, 19..23 hand L inequalities
 *   24..26 hand R equalities, 27..31 hand R inequalities
 * plus 3 initial-pose rows.  Internally the force rows are divided by m g
 * and the torque row by m g l (l the larger half-side); the violation v_hat
 * (Eq. inexact_mode_value) is taken in physical units, separately from that
 * scaling (Sec. III-C "Stopping and scoring"): lengths in m, angles in rad,
 * velocities in m/s, forces in N, the torque in N m, the slide-direction row
 * as the friction force's power in W, and the slide friction row (internally
 * (lam_t^2 - mu^2 lam_n^2) / (m g)^2) as the friction force's distance from
 * the cone edge, |lam_t| - mu |lam_n| in N.  Cost: w_T |pose_N - goal|^2 + sum_k u_k^T R u_k
 * with R = diag(w_v (twist), w_f (forces), w_s (sliding rates), w_c (p_c)).
 */
#ifndef COMET_BIMANUAL_ORACLE_H
#define COMET_BIMANUAL_ORACLE_H
#include <stdint.h>

#include "comet_oracle.h"

#ifdef __cplusplus
extern "C" {
#endif

#define BIM_NX 5
#define BIM_NU 12
#define BIM_NROW 32
#define BIM_NLOC (2 * BIM_NX + BIM_NU) /* local variables (x_k, u_k, x_{k+1}) */
#define BIM_NMODES 507

typedef struct {
    double ax, az;       /* half-width and half-height of the box [m] */
    double mass;         /* [kg] */
    double mu_g, mu_h;   /* ground and hand friction coefficients */
    double dt;           /* interval duration [s] */
    double grav;         /* gravity [m/s^2] */
    int32_t knots_per_segment;
    int32_t pad0;
    double start[3], goal[3];
    double w_terminal;   /* on the pose error */
    double w_v, w_f, w_s, w_c;
} bim_instance;

/* Rows of interval k at local variables (x_k[5], u_k[12], x_{k+1}[5]):
 * scaled values c[32], presence mask, inequality flags, physical factors
 * (physical = c / scale) and the local Jacobian J[32][22] (row-major). */
void bim_interval_rows(const bim_instance* in, int32_t mode, int32_t mask_sL, int32_t mask_sR,
                       const double* xk, const double* uk, const double* xk1, double* c, uint8_t* mask,
                       uint8_t* ineq, double* scale, double* J);

/* Rows of a whole trajectory (component-major x[5][N+1], u[12][N]):
 * c [N][32], mask, scale (each nullable) and c_init[3]. */
void bim_rows(const bim_instance* in, int32_t len, const uint16_t* modes, int32_t N, const double* traj, double* c,
              uint8_t* mask, double* scale, double* c_init);

/* Dense Jacobian [(3 + 32 N) x (17 N + 5)] over the interleaved variables
 * (x_k, u_k per knot, x_N last); masked rows are zero. */
void bim_dense_jacobian(const bim_instance* in, int32_t len, const uint16_t* modes, int32_t N, const double* traj,
                        double* jac);

void bim_cold_start(const bim_instance* in, int32_t N, double* traj);

double bim_cost(const bim_instance* in, int32_t N, const double* traj);

/* Gauss-Newton step of the augmented Lagrangian by the backward sweep over
 * w_k = (u_k, x_{k+1}) (17 x 17 S_k, Cholesky without pivoting); dz and grad
 * are interleaved (17 N + 5).  Returns 0, or -1 on a non-positive pivot. */
int32_t bim_gn_step(const bim_instance* in, int32_t len, const uint16_t* modes, int32_t N, const double* traj,
                    const double* lam, double beta, double rho, double* dz, double* grad);

double bim_al_merit(const bim_instance* in, int32_t len, const uint16_t* modes, int32_t N, const double* traj,
                    const double* lam, double beta);

/* The TO of one mode order (same method and options as orc_solve; the step
 * model is Gauss-Newton). */
int32_t bim_solve(const bim_instance* in, int32_t len, const uint16_t* modes, int32_t N, const double* warm,
                  const orc_opts* opt, double* out_traj, double* out_lam, orc_result* res);

int32_t bim_solve_batch(const bim_instance* insts, const int32_t* inst_idx, const int32_t* lens,
                        const uint16_t* modes, int32_t lmax, const int32_t* Ns, int64_t n, const orc_opts* opt,
                        int32_t nthreads, double* out_traj, int64_t traj_stride, orc_result* res);

/* bim_solve_batch with optional warm starts (TO i from the trajectory at
 * warm + i * warm_stride, in its own N, and from the multipliers at
 * warm_lam + i * lam_stride) and optional multipliers out (3 + 32 N at
 * out_lam + i * lam_stride). */
int32_t bim_solve_batch_ex(const bim_instance* insts, const int32_t* inst_idx, const int32_t* lens,
                           const uint16_t* modes, int32_t lmax, const int32_t* Ns, int64_t n, const orc_opts* opt,
                           int32_t nthreads, const double* warm, int64_t warm_stride, const double* warm_lam,
                           double* out_traj, int64_t traj_stride, double* out_lam, int64_t lam_stride,
                           orc_result* res);

/* bim_solve starting from the multipliers warm_lam (3 + 32 N; NULL = 0). */
int32_t bim_solve_ex(const bim_instance* in, int32_t len, const uint16_t* modes, int32_t N, const double* warm,
                     const double* warm_lam, const orc_opts* opt, double* out_traj, double* out_lam,
                     orc_result* res);

#ifdef __cplusplus
}
#endif

#endif
