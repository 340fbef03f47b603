/*
 * comet_oracle.c -- FP64 CPU oracle of the CoMET mode-conditioned TO.
 *
 * TEST INFRASTRUCTURE ONLY (see comet_oracle.h).  Plain double-precision
 * loops over explicit small matrices; no blocking, fusion or structure
 * exploitation beyond what the method itself states.
 *
 * Paper passages followed:
 *   Eq. crmp / Eq. mode_nlp            -- problem min J s.t. g = 0, h <= 0
 *   Sec. III-C, shared representation  -- N intervals, d_k = x_{k+1} - F_k(x_k,u_k;m),
 *                                          fixed row positions with binary masks,
 *                                          masked rows have zero residual,
 *                                          derivative and multiplier
 *   Sec. III-C, fixed-workspace solves -- S_k = H_k + rho_k I + A_k^T A_k / mu_AL
 *                                          over (u_k, x_{k+1}), Cholesky without
 *                                          pivoting, damping retries, forward pass,
 *                                          parallel trial-step merits
 *   Sec. III-C, stopping and scoring   -- feasibility / stationarity / dual
 *                                          tolerances or iteration limit; score in
 *                                          physical units
 *   Eq. inexact_mode_value             -- J_hat and v_hat
 *   Eq. search_merit                   -- M_hat
 * Where the paper is silent (dynamics equations, hyper-parameters, row
 * scaling constants) the readings are stated beside the code that takes
 * them.
 */
#include "comet_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "flops.h"

#ifdef ORC_COUNT_FLOPS
__thread uint64_t orc_g_flops;
__thread int orc_g_rows_on = 1, orc_g_jac_on = 1;
#endif

uint64_t orc_flop_count(void) {
#ifdef ORC_COUNT_FLOPS
    return orc_g_flops;
#else
    return 0;
#endif
}

void orc_flop_reset(void) {
#ifdef ORC_COUNT_FLOPS
    orc_g_flops = 0;
#endif
}

/* ---------------------------------------------------------------- model */

/* Face f of the rectangular slider: inward push direction n_f in the body
 * frame, tangent t_f = n_f rotated by +90 degrees, half-depth a_f (distance
 * from the centre to the face) and half-length ell_f (half the face). */
static void face_frame(const orc_instance* in, int32_t face, double n[2], double t[2],
                       double* a, double* ell) {
    static const double NX_[4] = {1.0, 0.0, -1.0, 0.0};
    static const double NY_[4] = {0.0, 1.0, 0.0, -1.0};
    n[0] = NX_[face];
    n[1] = NY_[face];
    t[0] = -n[1];
    t[1] = n[0];
    if (face % 2 == 0) {
        *a = 0.5 * in->side_x;
        *ell = 0.5 * in->side_y;
    } else {
        *a = 0.5 * in->side_y;
        *ell = 0.5 * in->side_x;
    }
}

void orc_dynamics(const orc_instance* in, int32_t face, const double* x, const double* u,
                  double* f, double* Fx, double* Fu) {
    double n[2], t[2], a, ell;
    face_frame(in, face, n, t, &a, &ell);
    const double th = x[2], s = x[3];
    const double fn = u[0], ft = u[1], sd = u[2];
    const double k = in->kappa, c2 = in->c_ls * in->c_ls;
    /* body-frame wrench from the point contact at p = -a n + s t */
    const double Fbx = fn * n[0] + ft * t[0];
    const double Fby = fn * n[1] + ft * t[1];
    const double mz = -a * ft - s * fn;
    /* ellipsoidal limit surface H(w) = Fx^2 + Fy^2 + mz^2/c^2: twist ~ grad H */
    const double vx = k * Fbx, vy = k * Fby, w = k * mz / c2;
    const double ct = cos(th), st = sin(th);
    FLOPS_ROWS(3 + 3 + 3 + 4 + 2); /* body wrench, twist, sine and cosine */
    if (f) FLOPS_ROWS(6);
    if (Fx) FLOPS_JAC(6 + 2);
    if (Fu) FLOPS_JAC(16);
    if (f) {
        f[0] = ct * vx - st * vy;
        f[1] = st * vx + ct * vy;
        f[2] = w;
        f[3] = sd;
    }
    if (Fx) {
        for (int i = 0; i < 16; ++i) Fx[i] = 0.0;
        Fx[0 * 4 + 2] = -st * vx - ct * vy;
        Fx[1 * 4 + 2] = ct * vx - st * vy;
        Fx[2 * 4 + 3] = -k * fn / c2;
    }
    if (Fu) {
        for (int i = 0; i < 12; ++i) Fu[i] = 0.0;
        /* d/dfn of body twist: k (n_x, n_y, -s/c^2); d/dft: k (t_x, t_y, -a/c^2) */
        Fu[0 * 3 + 0] = k * (ct * n[0] - st * n[1]);
        Fu[1 * 3 + 0] = k * (st * n[0] + ct * n[1]);
        Fu[2 * 3 + 0] = -k * s / c2;
        Fu[0 * 3 + 1] = k * (ct * t[0] - st * t[1]);
        Fu[1 * 3 + 1] = k * (st * t[0] + ct * t[1]);
        Fu[2 * 3 + 1] = -k * a / c2;
        Fu[3 * 3 + 2] = 1.0;
    }
}

/* Curvature of the dynamics: Hf = sum_r y_r * d^2 f_r / d(x,u)^2 over the
 * seven variables (x, y, theta, s, f_n, f_t, sdot), row-major 7x7.  f is
 * bilinear in the forces and in (cos theta, sin theta), so only the
 * (theta, theta), (theta, f_n), (theta, f_t) and (s, f_n) entries are
 * non-zero. */
static void dynamics_curvature(const orc_instance* in, int32_t face, const double* x, const double* u,
                               const double* y, double* Hf) {
    double n[2], t[2], a, ell;
    face_frame(in, face, n, t, &a, &ell);
    const double th = x[2], fn = u[0], ft = u[1];
    const double k = in->kappa, c2 = in->c_ls * in->c_ls;
    const double ct = cos(th), st = sin(th);
    const double vx = k * (fn * n[0] + ft * t[0]);
    const double vy = k * (fn * n[1] + ft * t[1]);
    const double f0 = ct * vx - st * vy, f1 = st * vx + ct * vy;
    FLOPS(2 + 6 + 6 + 3 + 10 + 10 + 2);
    for (int i = 0; i < 49; ++i) Hf[i] = 0.0;
    Hf[2 * 7 + 2] = -y[0] * f0 - y[1] * f1;
    const double h_th_fn = y[0] * k * (-st * n[0] - ct * n[1]) + y[1] * k * (ct * n[0] - st * n[1]);
    const double h_th_ft = y[0] * k * (-st * t[0] - ct * t[1]) + y[1] * k * (ct * t[0] - st * t[1]);
    Hf[2 * 7 + 4] = Hf[4 * 7 + 2] = h_th_fn;
    Hf[2 * 7 + 5] = Hf[5 * 7 + 2] = h_th_ft;
    Hf[3 * 7 + 4] = Hf[4 * 7 + 3] = -y[2] * k / c2;
}

int32_t orc_segment_of(int32_t k, int32_t len, int32_t N) {
    return (int32_t)(((int64_t)k * len) / N);
}

/* trajectory accessors, component-major layout */
static double* TX(double* tr, int32_t N, int32_t k, int32_t i) { return &tr[i * (N + 1) + k]; }
static double* TU(double* tr, int32_t N, int32_t k, int32_t j) { return &tr[4 * (N + 1) + j * N + k]; }
static double CX(const double* tr, int32_t N, int32_t k, int32_t i) { return tr[i * (N + 1) + k]; }
static double CU(const double* tr, int32_t N, int32_t k, int32_t j) { return tr[4 * (N + 1) + j * N + k]; }

void orc_cold_start(const orc_instance* in, int32_t N, double* traj) {
    for (int32_t k = 0; k <= N; ++k) {
        const double a = (double)k / (double)N;
        for (int i = 0; i < 3; ++i) *TX(traj, N, k, i) = (1.0 - a) * in->start[i] + a * in->goal[i];
        *TX(traj, N, k, 3) = 0.0;
    }
    for (int32_t k = 0; k < N; ++k)
        for (int j = 0; j < 3; ++j) *TU(traj, N, k, j) = 0.0;
}

/* Internal scaling of the dynamics rows (Sec. IV-A: rows are scaled by their
 * median Jacobian-row norm over sample orders).  Row i of d_k is divided by
 * sigma_i = median over the four faces of |d d_k,i / d(x_k, u_k, x_{k+1})|
 * at the cold-start reference point (x_k = 0, u_k = 0). */
static double dyn_row_scale(const orc_instance* in, int32_t i) {
    double nrm[4];
    const double x0[4] = {0.0, 0.0, 0.0, 0.0}, u0[3] = {0.0, 0.0, 0.0};
#ifdef ORC_COUNT_FLOPS
    /* a constant of the instance that this plain implementation recomputes
     * at every row evaluation: not the method's work */
    const int rows_on = orc_g_rows_on, jac_on = orc_g_jac_on;
    COUNT_ROWS(0, 0);
#endif
    for (int32_t face = 0; face < 4; ++face) {
        double Fx[16], Fu[12], s2 = 1.0; /* the x_{k+1} entry */
        orc_dynamics(in, face, x0, u0, NULL, Fx, Fu);
        for (int j = 0; j < 4; ++j) {
            const double v = -((i == j) ? 1.0 : 0.0) - in->dt * Fx[i * 4 + j];
            s2 += v * v;
        }
        for (int j = 0; j < 3; ++j) s2 += in->dt * Fu[i * 3 + j] * in->dt * Fu[i * 3 + j];
        nrm[face] = sqrt(s2);
    }
    /* median of four values: mean of the middle two after sorting */
    for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b)
            if (nrm[b] < nrm[a]) {
                const double t = nrm[a];
                nrm[a] = nrm[b];
                nrm[b] = t;
            }
#ifdef ORC_COUNT_FLOPS
    COUNT_ROWS(rows_on, jac_on);
#endif
    return 0.5 * (nrm[1] + nrm[2]);
}

/* Rows of a free-motion interval (mode ORC_MODE_FREE) at the same fixed
 * positions: the slider rests, d_k = x_{k+1} - x_k - dt (0, 0, 0, sdot)
 * (same row scales), and the mode equality is f_n = 0 (no contact).  Every
 * other row is off: f_t then acts on nothing and the effort cost sets it
 * to zero, which keeps the active rows independent (an f_t = 0 written as
 * two opposite inequalities, or -f_n <= 0 beside f_n = 0, would not be). */
static void free_rows(const orc_instance* in, int32_t s_row_masked, const double* xk, const double* uk,
                      const double* xk1, double* c, uint8_t* mask, double* scale, double* J) {
    for (int i = 0; i < ORC_NROW * 11; ++i) J[i] = 0.0;
    for (int r = 0; r < ORC_NROW; ++r) {
        c[r] = 0.0;
        mask[r] = 1;
        scale[r] = 1.0;
    }
    for (int i = 0; i < 4; ++i) {
        const double sg = dyn_row_scale(in, i);
        const double rate = (i == 3) ? uk[2] : 0.0;
        c[i] = (xk1[i] - xk[i] - in->dt * rate) / sg;
        J[i * 11 + i] = -1.0 / sg;
        J[i * 11 + 7 + i] = 1.0 / sg;
        scale[i] = 1.0 / sg;
    }
    J[3 * 11 + 6] = -in->dt / dyn_row_scale(in, 3);
    FLOPS_ROWS(4 * 3);
    FLOPS_JAC(1);
    if (s_row_masked) mask[3] = 0;
    c[4] = uk[0];
    J[4 * 11 + 4] = 1.0;
    for (int r = 5; r < ORC_NROW; ++r) mask[r] = 0;
    for (int r = 0; r < ORC_NROW; ++r)
        if (!mask[r]) {
            c[r] = 0.0;
            for (int j = 0; j < 11; ++j) J[r * 11 + j] = 0.0;
        }
}

/* Rows of interval k at local variables v = (x_k[4], u_k[3], x_{k+1}[4]).
 * Outputs scaled values c[11], mask[11], scale[11] (physical = c/scale)
 * and the local Jacobian J[11][11] (row r, local variable j). */
static void interval_rows(const orc_instance* in, int32_t mode, int32_t s_row_masked,
                          const double* xk, const double* uk, const double* xk1,
                          double* c, uint8_t* mask, double* scale, double* J) {
    if (mode == ORC_MODE_FREE) {
        free_rows(in, s_row_masked, xk, uk, xk1, c, mask, scale, J);
        return;
    }
    const int32_t face = mode / 3, kind = mode % 3; /* 0 stick, 1 slide+, 2 slide- */
    double n[2], t[2], a, ell;
    face_frame(in, face, n, t, &a, &ell);
    const double mu = in->mu, sc = 1.0 / sqrt(1.0 + mu * mu);
    double f[4], Fx[16], Fu[12];
    orc_dynamics(in, face, xk, uk, f, Fx, Fu);
    for (int i = 0; i < ORC_NROW * 11; ++i) J[i] = 0.0;
    for (int r = 0; r < ORC_NROW; ++r) {
        c[r] = 0.0;
        mask[r] = 1;
        scale[r] = 1.0;
    }
    /* dynamics defect d_k = x_{k+1} - x_k - dt f(x_k, u_k) (Sec. III-C),
     * row i divided by its internal scale sigma_i */
    for (int i = 0; i < 4; ++i) {
        const double sg = dyn_row_scale(in, i);
        c[i] = (xk1[i] - xk[i] - in->dt * f[i]) / sg;
        for (int j = 0; j < 4; ++j) J[i * 11 + j] = (-((i == j) ? 1.0 : 0.0) - in->dt * Fx[i * 4 + j]) / sg;
        for (int j = 0; j < 3; ++j) J[i * 11 + 4 + j] = -in->dt * Fu[i * 3 + j] / sg;
        J[i * 11 + 7 + i] = 1.0 / sg;
        scale[i] = 1.0 / sg;
    }
    /* defects (3 each), the nonzero Jacobian entries (x_k: diagonal and the
     * three terms of d f / d x; u_k: seven entries of d f / d u), the mode
     * rows' values */
    FLOPS_ROWS(4 * 3 + 18);
    FLOPS_JAC(4 + 3 * 2 + 7 * 2);
    if (s_row_masked) mask[3] = 0;
    /* mode equality (row 4) */
    if (kind == 0) {
        c[4] = uk[2];
        J[4 * 11 + 6] = 1.0;
    } else {
        const double sg = (kind == 1) ? -1.0 : 1.0; /* slide+: ft - mu fn = 0; slide-: ft + mu fn = 0 */
        c[4] = sc * (uk[1] + sg * mu * uk[0]);
        J[4 * 11 + 4] = sc * sg * mu;
        J[4 * 11 + 5] = sc;
        scale[4] = sc;
    }
    /* friction cone (rows 5, 6): sticking only */
    c[5] = sc * (uk[1] - mu * uk[0]);
    J[5 * 11 + 4] = -sc * mu;
    J[5 * 11 + 5] = sc;
    scale[5] = sc;
    c[6] = sc * (-uk[1] - mu * uk[0]);
    J[6 * 11 + 4] = -sc * mu;
    J[6 * 11 + 5] = -sc;
    scale[6] = sc;
    if (kind != 0) mask[5] = mask[6] = 0;
    /* sliding direction (row 7): slide+ needs sd >= 0, slide- needs sd <= 0 */
    if (kind == 0) {
        mask[7] = 0;
    } else {
        const double sg = (kind == 1) ? -1.0 : 1.0;
        c[7] = sg * uk[2];
        J[7 * 11 + 6] = sg;
    }
    /* unilateral contact (row 8): -f_n <= 0 */
    c[8] = -uk[0];
    J[8 * 11 + 4] = -1.0;
    /* contact point stays on the face (rows 9, 10): |s_k| <= ell */
    c[9] = xk[3] - ell;
    J[9 * 11 + 3] = 1.0;
    c[10] = -xk[3] - ell;
    J[10 * 11 + 3] = -1.0;
    for (int r = 0; r < ORC_NROW; ++r)
        if (!mask[r]) {
            c[r] = 0.0;
            for (int j = 0; j < 11; ++j) J[r * 11 + j] = 0.0;
        }
}

static int32_t mode_of_interval(const uint8_t* modes, int32_t len, int32_t N, int32_t k) {
    return modes[orc_segment_of(k, len, N)];
}

/* s-row of d_k is masked when the pusher is not on the same face on both
 * sides of knot k+1 (another face next, or free motion on either side):
 * the pusher relocates and the contact offset may jump. */
static int32_t s_row_masked(const uint8_t* modes, int32_t len, int32_t N, int32_t k) {
    const int32_t m0 = mode_of_interval(modes, len, N, k);
    if (m0 == ORC_MODE_FREE) return 1;
    if (k + 1 >= N) return 0;
    const int32_t m1 = mode_of_interval(modes, len, N, k + 1);
    return m1 == ORC_MODE_FREE || (m0 / 3) != (m1 / 3);
}

static void load_local(const double* tr, int32_t N, int32_t k, double* xk, double* uk, double* xk1) {
    for (int i = 0; i < 4; ++i) {
        xk[i] = CX(tr, N, k, i);
        xk1[i] = CX(tr, N, k + 1, i);
    }
    for (int j = 0; j < 3; ++j) uk[j] = CU(tr, N, k, j);
}

void orc_rows(const orc_instance* in, int32_t len, const uint8_t* modes, int32_t N,
              const double* traj, double* c, uint8_t* mask, double* scale, double* c_init) {
    double xk[4], uk[3], xk1[4], cc[11], sc[11], J[121];
    uint8_t mk[11];
    for (int32_t k = 0; k < N; ++k) {
        load_local(traj, N, k, xk, uk, xk1);
        interval_rows(in, mode_of_interval(modes, len, N, k), s_row_masked(modes, len, N, k),
                      xk, uk, xk1, cc, mk, sc, J);
        for (int r = 0; r < 11; ++r) {
            if (c) c[k * 11 + r] = cc[r];
            if (mask) mask[k * 11 + r] = mk[r];
            if (scale) scale[k * 11 + r] = sc[r];
        }
    }
    if (c_init)
        for (int i = 0; i < 3; ++i) c_init[i] = CX(traj, N, 0, i) - in->start[i];
}

void orc_dense_jacobian(const orc_instance* in, int32_t len, const uint8_t* modes, int32_t N,
                        const double* traj, double* jac) {
    const int64_t nz = 7 * (int64_t)N + 4, nr = 3 + 11 * (int64_t)N;
    double xk[4], uk[3], xk1[4], cc[11], sc[11], J[121];
    uint8_t mk[11];
    memset(jac, 0, sizeof(double) * nz * nr);
    for (int i = 0; i < 3; ++i) jac[i * nz + i] = 1.0;
    for (int32_t k = 0; k < N; ++k) {
        load_local(traj, N, k, xk, uk, xk1);
        interval_rows(in, mode_of_interval(modes, len, N, k), s_row_masked(modes, len, N, k),
                      xk, uk, xk1, cc, mk, sc, J);
        for (int r = 0; r < 11; ++r) {
            double* row = &jac[(3 + 11 * (int64_t)k + r) * nz];
            for (int j = 0; j < 11; ++j) row[7 * (int64_t)k + j] = J[r * 11 + j];
        }
    }
}

/* ------------------------------------------------------ AL ingredients */

/* multiplier estimate of one row: equality rows (r < 5, and the initial
 * rows) lam + beta c; inequality rows max(0, lam + beta c) (PHR). */
static double row_y(int32_t is_ineq, double lam, double beta, double c) {
    const double y = lam + beta * c;
    if (is_ineq) return y > 0.0 ? y : 0.0;
    return y;
}

/* PHR augmented-Lagrangian term of one row. */
static double row_al(int32_t is_ineq, double lam, double beta, double c) {
    if (!is_ineq) return lam * c + 0.5 * beta * c * c;
    const double y = lam + beta * c;
    const double p = y > 0.0 ? y : 0.0;
    return (p * p - lam * lam) / (2.0 * beta);
}

static double cost_of(const orc_instance* in, int32_t N, const double* tr) {
    double J = 0.0;
    FLOPS(3 * 4 + 3 * (int64_t)N * 3);
    for (int i = 0; i < 3; ++i) {
        const double e = CX(tr, N, N, i) - in->goal[i];
        J += in->w_terminal * e * e;
    }
    for (int32_t k = 0; k < N; ++k)
        for (int j = 0; j < 3; ++j) {
            const double u = CU(tr, N, k, j);
            J += in->w_control * u * u;
        }
    return J;
}

double orc_al_merit(const orc_instance* in, int32_t len, const uint8_t* modes, int32_t N,
                    const double* traj, const double* lam, double beta, double* cost_out) {
    const double J = cost_of(in, N, traj);
    if (cost_out) *cost_out = J;
    double L = J;
    for (int i = 0; i < 3; ++i) L += row_al(0, lam[i], beta, CX(traj, N, 0, i) - in->start[i]);
    double xk[4], uk[3], xk1[4], cc[11], sc[11], Jl[121];
    uint8_t mk[11];
    COUNT_ROWS(1, 0);
    for (int32_t k = 0; k < N; ++k) {
        load_local(traj, N, k, xk, uk, xk1);
        interval_rows(in, mode_of_interval(modes, len, N, k), s_row_masked(modes, len, N, k),
                      xk, uk, xk1, cc, mk, sc, Jl);
        for (int r = 0; r < 11; ++r)
            if (mk[r]) {
                L += row_al(r >= ORC_NEQ, lam[3 + 11 * k + r], beta, cc[r]);
                FLOPS(6);
            }
    }
    COUNT_ROWS(1, 1);
    return L;
}

/* Cholesky without pivoting of the n x n SPD matrix A (row-major, lower
 * triangle used) into L; returns -1 on a non-positive pivot. */
static int chol(int n, const double* A, double* L) {
    for (int i = 0; i < n * n; ++i) L[i] = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int p = 0; p < j; ++p) d -= L[j * n + p] * L[j * n + p];
        FLOPS(2 * j + 1 + (n - 1 - j) * (2 * j + 1));
        if (!(d > 0.0)) return -1;
        const double ljj = sqrt(d);
        L[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int p = 0; p < j; ++p) s -= L[i * n + p] * L[j * n + p];
            L[i * n + j] = s / ljj;
        }
    }
    return 0;
}

/* x = A^{-1} b with A = L L^T (forward then backward substitution). */
static void chol_solve(int n, const double* L, const double* b, double* x) {
    double y[16];
    FLOPS(2 * n * n);
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int p = 0; p < i; ++p) s -= L[i * n + p] * y[p];
        y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int p = i + 1; p < n; ++p) s -= L[p * n + i] * x[p];
        x[i] = s / L[i * n + i];
    }
}

/* Gauss-Newton step by the backward sweep (Sec. III-C).  Local variables of
 * interval k: v = (x_k, u_k, x_{k+1}); w_k = (u_k, x_{k+1}). */
int32_t orc_gn_step(const orc_instance* in, int32_t len, const uint8_t* modes, int32_t N,
                    const double* traj, const double* lam, double beta, double rho,
                    int32_t curvature, double* dz, double* grad) {
    double* Kg = (double*)malloc(sizeof(double) * 28 * (size_t)N); /* K_k = -S^-1 C, 7x4 */
    double* kg = (double*)malloc(sizeof(double) * 7 * (size_t)N);  /* k_k = -S^-1 g_w */
    const int64_t nz = 7 * (int64_t)N + 4;
    for (int64_t i = 0; i < nz; ++i) grad[i] = 0.0;

    /* value function of x_N: terminal cost w_T |pose_N - goal|^2 */
    double V[16] = {0}, v[4] = {0};
    for (int i = 0; i < 3; ++i) {
        V[i * 4 + i] = 2.0 * in->w_terminal;
        v[i] = 2.0 * in->w_terminal * (CX(traj, N, N, i) - in->goal[i]);
        grad[7 * (int64_t)N + i] += v[i];
    }
    double xk[4], uk[3], xk1[4], cc[11], sc[11], Jl[121];
    uint8_t mk[11];
    int32_t ok = 0;
    COUNT_ROWS(0, 0);
    for (int32_t k = N - 1; k >= 0; --k) {
        load_local(traj, N, k, xk, uk, xk1);
        interval_rows(in, mode_of_interval(modes, len, N, k), s_row_masked(modes, len, N, k),
                      xk, uk, xk1, cc, mk, sc, Jl);
        /* local model of the AL: H = cost Hessian + beta sum_active a a^T
         * (+ the Lagrangian curvature of the dynamics rows when `curvature`),
         * g = cost gradient + sum y_r a_r.  Without the curvature term S_k
         * is positive definite for any rho > 0 (Gauss-Newton). */
        double H[121] = {0}, g[11] = {0};
        FLOPS(3 * 3);
        for (int j = 0; j < 3; ++j) {
            H[(4 + j) * 11 + 4 + j] += 2.0 * in->w_control;
            g[4 + j] += 2.0 * in->w_control * uk[j];
        }
        for (int r = 0; r < 11; ++r) {
            if (!mk[r]) continue;
            const int32_t ineq = r >= ORC_NEQ;
            const double l = lam[3 + 11 * k + r];
            if (ineq && !(l + beta * cc[r] > 0.0)) continue; /* inactive */
            const double y = row_y(ineq, l, beta, cc[r]);
#ifdef ORC_COUNT_FLOPS
            {
                /* y, then per nonzero entry: g (2), beta a_i (1) and the
                 * lower-triangle products of the model (2 each) */
                int nnz = 0;
                for (int i = 0; i < 11; ++i) nnz += Jl[r * 11 + i] != 0.0;
                FLOPS(2 + 3 * nnz + nnz * (nnz + 1));
            }
#endif
            for (int i = 0; i < 11; ++i) {
                g[i] += y * Jl[r * 11 + i];
                for (int j = 0; j < 11; ++j) H[i * 11 + j] += beta * Jl[r * 11 + i] * Jl[r * 11 + j];
            }
        }
        if (curvature) {
            /* Lagrangian curvature of the dynamics rows: d_k = x_{k+1} - x_k - dt f,
             * so sum_r y_r d^2 d_r = -dt sum_r y_r d^2 f_r over (x_k, u_k) */
            double yd[4], Hf[49];
            for (int r = 0; r < 4; ++r)
                yd[r] = mk[r] ? row_y(0, lam[3 + 11 * k + r], beta, cc[r]) / dyn_row_scale(in, r) : 0.0;
            const int32_t mk_k = mode_of_interval(modes, len, N, k);
            if (mk_k != ORC_MODE_FREE) {  /* free motion: f is linear, no curvature */
                dynamics_curvature(in, mk_k / 3, xk, uk, yd, Hf);
                FLOPS(4 * 3 + 4 * 2); /* yd, and the four curvature entries into H */
                for (int i = 0; i < 7; ++i)
                    for (int j = 0; j < 7; ++j) H[i * 11 + j] -= in->dt * Hf[i * 7 + j];
            }
        }
        for (int i = 0; i < 4; ++i) grad[7 * (int64_t)k + i] += g[i];
        for (int j = 0; j < 3; ++j) grad[7 * (int64_t)k + 4 + j] += g[4 + j];
        for (int i = 0; i < 4; ++i) grad[7 * (int64_t)(k + 1) + i] += g[7 + i];

        /* S_k = H_ww + rho I + [0 0; 0 V_{k+1}],  C_k = H_wx,  g_w */
        double S[49], C[28], gw[7], L[49];
        for (int i = 0; i < 7; ++i) {
            for (int j = 0; j < 7; ++j) S[i * 7 + j] = H[(4 + i) * 11 + 4 + j];
            S[i * 7 + i] += rho;
            for (int j = 0; j < 4; ++j) C[i * 4 + j] = H[(4 + i) * 11 + j];
            gw[i] = g[4 + i];
        }
        for (int i = 0; i < 4; ++i) {
            for (int j = 0; j < 4; ++j) S[(3 + i) * 7 + 3 + j] += V[i * 4 + j];
            gw[3 + i] += v[i];
        }
        FLOPS(7 + 10 + 4); /* rho, V_{k+1} (lower triangle), v_{k+1} */
        if (chol(7, S, L) != 0) {
            ok = -1;
            break;
        }
        /* gains G_k = -S^-1 [C | g_w] */
        double col[7], sol[7];
        for (int j = 0; j < 4; ++j) {
            for (int i = 0; i < 7; ++i) col[i] = C[i * 4 + j];
            chol_solve(7, L, col, sol);
            for (int i = 0; i < 7; ++i) Kg[28 * (int64_t)k + i * 4 + j] = -sol[i];
        }
        chol_solve(7, L, gw, sol);
        for (int i = 0; i < 7; ++i) kg[7 * (int64_t)k + i] = -sol[i];
        /* V_k = H_xx - C^T S^-1 C = H_xx + C^T K_k ;  v_k = g_x + C^T k_k */
        FLOPS(10 * 7 * 2 + 4 * 7 * 2); /* symmetric V (lower triangle) and v */
        double Vn[16], vn[4];
        for (int i = 0; i < 4; ++i) {
            for (int j = 0; j < 4; ++j) {
                double s = H[i * 11 + j];
                for (int p = 0; p < 7; ++p) s += C[p * 4 + i] * Kg[28 * (int64_t)k + p * 4 + j];
                Vn[i * 4 + j] = s;
            }
            double s = g[i];
            for (int p = 0; p < 7; ++p) s += C[p * 4 + i] * kg[7 * (int64_t)k + p];
            vn[i] = s;
        }
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) V[i * 4 + j] = 0.5 * (Vn[i * 4 + j] + Vn[j * 4 + i]);
        for (int i = 0; i < 4; ++i) v[i] = vn[i];
    }
    if (ok == 0) {
        /* initial-state block: V_0 + rho I + beta on the three pose rows */
        double H0[16], g0[4], L0[16], dx[4];
        for (int i = 0; i < 16; ++i) H0[i] = V[i];
        for (int i = 0; i < 4; ++i) {
            H0[i * 4 + i] += rho;
            g0[i] = v[i];
        }
        for (int i = 0; i < 3; ++i) {
            const double y = row_y(0, lam[i], beta, CX(traj, N, 0, i) - in->start[i]);
            H0[i * 4 + i] += beta;
            g0[i] += y;
            grad[i] += y;
        }
        if (chol(4, H0, L0) != 0) {
            ok = -1;
        } else {
            chol_solve(4, L0, g0, dx);
            for (int i = 0; i < 4; ++i) dx[i] = -dx[i];
            /* forward pass: dw_k = K_k dx_k + k_k */
            for (int i = 0; i < 4; ++i) dz[i] = dx[i];
            FLOPS((int64_t)N * 7 * 8);
            for (int32_t k = 0; k < N; ++k) {
                double dw[7];
                for (int i = 0; i < 7; ++i) {
                    double s = kg[7 * (int64_t)k + i];
                    for (int j = 0; j < 4; ++j) s += Kg[28 * (int64_t)k + i * 4 + j] * dx[j];
                    dw[i] = s;
                }
                for (int j = 0; j < 3; ++j) dz[7 * (int64_t)k + 4 + j] = dw[j];
                for (int i = 0; i < 4; ++i) {
                    dz[7 * (int64_t)(k + 1) + i] = dw[3 + i];
                    dx[i] = dw[3 + i];
                }
            }
        }
    }
    COUNT_ROWS(1, 1);
    free(Kg);
    free(kg);
    return ok;
}

/* ------------------------------------------------------------- solver */

void orc_default_opts(orc_opts* o) {
    o->max_iters = 300;
    o->max_factor_retries = 8;
    o->n_alpha = 7;
    o->max_inner = 40;
    o->beta0 = 100.0;
    o->beta_max = 1e4;
    o->beta_growth = 10.0;
    o->rho0 = 1e-4;
    o->rho_min = 1e-4;
    o->rho_max = 1e6;
    o->armijo_c1 = 1e-4;
    o->ls_slack = 1e-6;
    o->eps_primal = 1e-6;
    o->eps_dual = 1e-4;
    o->eps_comp = 1e-6;
    o->omega_ratio = 1.0;
    o->eta_ratio = 0.25;
    o->eps_feas = 1e-5;
    o->merit_mu = 100.0;
    o->beta_ref = 1e3;
    o->curv_skip = 3;
}

double orc_stat_tol(const orc_opts* opt, double beta, double cost) {
    return opt->eps_dual * fmax(1.0, beta / opt->beta_ref) * fmax(1.0, fabs(cost));
}

/* add alpha * dz (interleaved) to a component-major trajectory */
static void axpy_traj(int32_t N, const double* tr, double alpha, const double* dz, double* out) {
    FLOPS(2 * (7 * (int64_t)N + 4));
    for (int32_t k = 0; k <= N; ++k)
        for (int i = 0; i < 4; ++i) out[i * (N + 1) + k] = CX(tr, N, k, i) + alpha * dz[7 * (int64_t)k + i];
    for (int32_t k = 0; k < N; ++k)
        for (int j = 0; j < 3; ++j)
            out[4 * (N + 1) + j * N + k] = CU(tr, N, k, j) + alpha * dz[7 * (int64_t)k + 4 + j];
}

typedef struct {
    double viol;  /* max scaled |c_E|, [c_I]+ */
    double stat;  /* |grad L_A|_inf = |grad J + A^T y|_inf */
    double comp;  /* max_I |y_i c_i| */
    double vphys; /* physical-unit violation (Eq. inexact_mode_value) */
    int finite;
} kkt_measures;

/* residual measures at traj for multipliers lam and penalty beta; y (3+11N)
 * receives the AL multiplier estimates.  grad work array of size 7N+4. */
static void measures(const orc_instance* in, int32_t len, const uint8_t* modes, int32_t N,
                     const double* traj, const double* lam, double beta, double* y,
                     double* grad, kkt_measures* m) {
    const int64_t nz = 7 * (int64_t)N + 4;
    for (int64_t i = 0; i < nz; ++i) grad[i] = 0.0;
    m->viol = 0.0;
    m->comp = 0.0;
    m->vphys = 0.0;
    m->finite = 1;
    /* cost gradient */
    for (int i = 0; i < 3; ++i) grad[7 * (int64_t)N + i] += 2.0 * in->w_terminal * (CX(traj, N, N, i) - in->goal[i]);
    for (int32_t k = 0; k < N; ++k)
        for (int j = 0; j < 3; ++j) grad[7 * (int64_t)k + 4 + j] += 2.0 * in->w_control * CU(traj, N, k, j);
    for (int i = 0; i < 3; ++i) {
        const double c = CX(traj, N, 0, i) - in->start[i];
        y[i] = row_y(0, lam[i], beta, c);
        grad[i] += y[i];
        if (fabs(c) > m->viol) m->viol = fabs(c);
        if (fabs(c) > m->vphys) m->vphys = fabs(c);
        if (!isfinite(c)) m->finite = 0;
    }
    double xk[4], uk[3], xk1[4], cc[11], sc[11], Jl[121];
    uint8_t mk[11];
    for (int32_t k = 0; k < N; ++k) {
        load_local(traj, N, k, xk, uk, xk1);
        interval_rows(in, mode_of_interval(modes, len, N, k), s_row_masked(modes, len, N, k),
                      xk, uk, xk1, cc, mk, sc, Jl);
        for (int r = 0; r < 11; ++r) {
            const int64_t idx = 3 + 11 * (int64_t)k + r;
            if (!mk[r]) {
                y[idx] = 0.0;
                continue;
            }
            if (!isfinite(cc[r])) m->finite = 0;
            const int32_t ineq = r >= ORC_NEQ;
            const double yr = row_y(ineq, lam[idx], beta, cc[r]);
            y[idx] = yr;
            const double v = ineq ? (cc[r] > 0.0 ? cc[r] : 0.0) : fabs(cc[r]);
            if (v > m->viol) m->viol = v;
            if (v / sc[r] > m->vphys) m->vphys = v / sc[r];
            if (ineq && fabs(yr * cc[r]) > m->comp) m->comp = fabs(yr * cc[r]);
            FLOPS(2 + 2 + 2); /* y, the violation in both units, complementarity */
            if (yr != 0.0) {
#ifdef ORC_COUNT_FLOPS
                int nnz = 0;
                for (int i = 0; i < 11; ++i) nnz += Jl[r * 11 + i] != 0.0;
                FLOPS(2 * nnz);
#endif
                for (int i = 0; i < 11; ++i) grad[7 * (int64_t)k + i] += yr * Jl[r * 11 + i];
            }
        }
    }
    m->stat = 0.0;
    for (int64_t i = 0; i < nz; ++i) {
        if (!isfinite(grad[i])) m->finite = 0;
        if (fabs(grad[i]) > m->stat) m->stat = fabs(grad[i]);
    }
}

int32_t orc_solve(const orc_instance* in, int32_t len, const uint8_t* modes, int32_t N,
                  const double* warm, const orc_opts* opt,
                  double* out_traj, double* out_lam, orc_result* res) {
    return orc_solve_ex(in, len, modes, N, warm, NULL, opt, out_traj, out_lam, res);
}

int32_t orc_solve_ex(const orc_instance* in, int32_t len, const uint8_t* modes, int32_t N, const double* warm,
                     const double* warm_lam, const orc_opts* opt, double* out_traj, double* out_lam,
                     orc_result* res) {
    const int64_t nt = 7 * (int64_t)N + 4, nl = 3 + 11 * (int64_t)N;
    double* z = (double*)malloc(sizeof(double) * nt);
    double* zt = (double*)malloc(sizeof(double) * nt);
    double* dz = (double*)malloc(sizeof(double) * nt);
    double* grad = (double*)malloc(sizeof(double) * nt);
    double* lam = (double*)calloc((size_t)nl, sizeof(double));
    if (warm_lam) memcpy(lam, warm_lam, sizeof(double) * nl);
    double* y = (double*)malloc(sizeof(double) * nl);
    if (warm)
        memcpy(z, warm, sizeof(double) * nt);
    else
        orc_cold_start(in, N, z);

    double beta = opt->beta0, rho = opt->rho0, eta = INFINITY;
    int32_t inner = 0, it = 0, status = ORC_MAX_ITER, n_outer = 0, n_rej = 0, curv_hold = 0, n_curv_fail = 0;
    kkt_measures m;
    for (it = 0; it < opt->max_iters; ++it) {
        measures(in, len, modes, N, z, lam, beta, y, grad, &m);
        if (!m.finite) {
            status = ORC_NONFINITE;
            break;
        }
        /* stop test (Sec. III-C "Stopping and scoring"): KKT of (z, y) on
         * the scaled problem.  Row scaling leaves grad L unchanged, so the
         * stationarity tolerance is taken relative to the objective's size,
         * max(1, |J|); the primal part asks for the scaled rows within
         * eps_primal and the rows in physical units within half eps_feas,
         * so that a converged TO is feasible by the score (Eq.
         * inexact_mode_value) */
        const double eps_d = orc_stat_tol(opt, beta, cost_of(in, N, z));
        if (m.viol <= opt->eps_primal && m.vphys <= 0.5 * opt->eps_feas && m.stat <= eps_d &&
            m.comp <= opt->eps_comp) {
            memcpy(lam, y, sizeof(double) * nl);
            status = ORC_CONVERGED;
            break;
        }
        /* multiplier and penalty update once the inner AL problem is solved
         * to omega, or after max_inner inner iterations */
        const double omega = fmax(eps_d, opt->omega_ratio * m.viol);
        const int32_t solved = m.stat <= omega;
        if (solved || inner >= opt->max_inner) {
            memcpy(lam, y, sizeof(double) * nl);
            /* the penalty grows only when a solved subproblem left the
             * violation above tolerance and did not reduce it enough; a
             * forced update leaves it unchanged */
            if (solved && m.viol > opt->eps_primal && m.viol > opt->eta_ratio * eta)
                beta = fmin(opt->beta_max, beta * opt->beta_growth);
            eta = m.viol;
            inner = 0;
            ++n_outer;
        }
        /* step: backward sweep with damping retries */
        /* Newton step on the AL with the Lagrangian curvature of the dynamics;
         * if a local Cholesky finds S_k indefinite, fall back to the
         * Gauss-Newton model, then raise the damping rho (Sec. III-C) */
        int32_t fac = -1;
        if (curv_hold == 0) {
            fac = orc_gn_step(in, len, modes, N, z, lam, beta, rho, 1, dz, grad);
            if (fac != 0) {
                ++n_curv_fail;
                curv_hold = opt->curv_skip;
            }
        } else {
            --curv_hold;
        }
        for (int32_t r = 0; fac != 0 && r <= opt->max_factor_retries; ++r) {
            if (r > 0) rho = fmin(opt->rho_max, rho * 10.0);
            fac = orc_gn_step(in, len, modes, N, z, lam, beta, rho, 0, dz, grad);
        }
        ++inner;
        if (fac != 0) {
            ++n_rej;
            continue;
        }
        /* parallel trial-step merits alpha = 2^-i; take the largest alpha
         * satisfying the Armijo condition */
        double D = 0.0;
        for (int64_t i = 0; i < nt; ++i) D += grad[i] * dz[i];
        FLOPS(2 * nt);
        const double phi0 = orc_al_merit(in, len, modes, N, z, lam, beta, NULL);
        /* when the predicted decrease is below the merit's resolution
         * (|D| <= ls_slack |phi0|) the merit cannot rank the trials: the full
         * step is taken if it does not raise the merit beyond that level */
        const double slack = opt->ls_slack * fabs(phi0);
        const int32_t flat = fabs(D) <= slack;
        double alpha = 0.0;
        for (int32_t i = 0; i < opt->n_alpha; ++i) {
            const double a = ldexp(1.0, -i);
            axpy_traj(N, z, a, dz, zt);
            const double phi = orc_al_merit(in, len, modes, N, zt, lam, beta, NULL);
            if (phi <= phi0 + opt->armijo_c1 * a * D || (flat && i == 0 && phi <= phi0 + slack)) {
                alpha = a;
                break;
            }
        }
        if (alpha > 0.0) {
            axpy_traj(N, z, alpha, dz, zt);
            memcpy(z, zt, sizeof(double) * nt);
            rho = fmax(opt->rho_min, rho / 10.0);
        } else {
            rho = fmin(opt->rho_max, rho * 10.0);
            ++n_rej;
        }
    }
    /* scoring in physical units (Eq. inexact_mode_value, Eq. search_merit) */
    if (status != ORC_CONVERGED) measures(in, len, modes, N, z, lam, beta, y, grad, &m);
    res->cost = cost_of(in, N, z);
    res->viol = m.vphys;
    res->stat = m.stat;
    res->comp = m.comp;
    res->merit = res->cost + opt->merit_mu * fmax(res->viol - opt->eps_feas, 0.0);
    if (!isfinite(res->cost) || !m.finite) status = ORC_NONFINITE;
    if (status == ORC_CONVERGED && !(res->viol <= opt->eps_feas)) status = ORC_INFEASIBLE;
    res->status = status;
    res->iters = it;
    res->n_outer = n_outer;
    res->n_rejected = n_rej;
    res->n_curv_fail = n_curv_fail;
    res->beta = beta;
    res->rho = rho;
    if (out_traj) memcpy(out_traj, z, sizeof(double) * nt);
    if (out_lam) memcpy(out_lam, status == ORC_CONVERGED ? lam : y, sizeof(double) * nl);
    free(z);
    free(zt);
    free(dz);
    free(grad);
    free(lam);
    free(y);
    return status;
}

/* ------------------------------------------------------ threaded batch */

typedef struct {
    const orc_instance* insts;
    const int32_t *inst_idx, *lens, *Ns;
    const uint8_t* modes;
    int32_t lmax;
    int64_t n;
    const orc_opts* opt;
    double* out_traj;
    int64_t traj_stride;
    const double* warm;
    int64_t warm_stride;
    double* out_lam;
    int64_t lam_stride;
    const double* warm_lam;
    orc_result* res;
    int64_t next;
    pthread_mutex_t lock;
} batch_ctx;

static void* batch_worker(void* arg) {
    batch_ctx* b = (batch_ctx*)arg;
    for (;;) {
        pthread_mutex_lock(&b->lock);
        const int64_t i = b->next++;
        pthread_mutex_unlock(&b->lock);
        if (i >= b->n) break;
        const int32_t N = b->Ns[i];
        double* tr = b->out_traj ? b->out_traj + i * b->traj_stride : NULL;
        const double* w = b->warm ? b->warm + i * b->warm_stride : NULL;
        double* lam = b->out_lam ? b->out_lam + i * b->lam_stride : NULL;
        const double* wl = b->warm_lam ? b->warm_lam + i * b->lam_stride : NULL;
        orc_solve_ex(&b->insts[b->inst_idx[i]], b->lens[i], b->modes + i * b->lmax, N, w, wl, b->opt,
                     tr, lam, &b->res[i]);
    }
    return NULL;
}

int32_t orc_solve_batch(const orc_instance* insts, const int32_t* inst_idx,
                        const int32_t* lens, const uint8_t* modes, int32_t lmax,
                        const int32_t* Ns, int64_t n, const orc_opts* opt, int32_t nthreads,
                        double* out_traj, int64_t traj_stride, orc_result* res) {
    return orc_solve_batch_ex(insts, inst_idx, lens, modes, lmax, Ns, n, opt, nthreads, NULL, 0, NULL, out_traj,
                              traj_stride, NULL, 0, res);
}

int32_t orc_solve_batch_ex(const orc_instance* insts, const int32_t* inst_idx, const int32_t* lens,
                           const uint8_t* modes, int32_t lmax, const int32_t* Ns, int64_t n, const orc_opts* opt,
                           int32_t nthreads, const double* warm, int64_t warm_stride, const double* warm_lam,
                           double* out_traj, int64_t traj_stride, double* out_lam, int64_t lam_stride,
                           orc_result* res) {
    batch_ctx b;
    b.warm_lam = warm_lam;
    b.warm = warm;
    b.warm_stride = warm_stride;
    b.out_lam = out_lam;
    b.lam_stride = lam_stride;
    b.insts = insts;
    b.inst_idx = inst_idx;
    b.lens = lens;
    b.Ns = Ns;
    b.modes = modes;
    b.lmax = lmax;
    b.n = n;
    b.opt = opt;
    b.out_traj = out_traj;
    b.traj_stride = traj_stride;
    b.res = res;
    b.next = 0;
    pthread_mutex_init(&b.lock, NULL);
    if (nthreads < 1) nthreads = 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int32_t t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, batch_worker, &b);
    for (int32_t t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&b.lock);
    return 0;
}
