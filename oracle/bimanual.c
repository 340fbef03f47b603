/*
 * bimanual.c -- FP64 CPU oracle of the bimanual box-flipping TO.
 * TEST INFRASTRUCTURE ONLY; see bimanual.h for the model.  The solver
 * follows the same steps as orc_solve (Sec. III-C): PHR augmented
 * Lagrangian, a Gauss-Newton step from the backward sweep over
 * w_k = (u_k, x_{k+1}) with Cholesky without pivoting and damping retries,
 * trial steps alpha = 2^-i with the Armijo test, multiplier / penalty updates
 * and the KKT stop test; scoring by Eq. inexact_mode_value and Eq.
 * search_merit.  All arithmetic is IEEE double.
 */
#include "bimanual.h"
#include "flops.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define NX BIM_NX
#define NU BIM_NU
#define NW (BIM_NU + BIM_NX)
#define NR BIM_NROW
#define NL BIM_NLOC

/* local variable indices */
enum { VX = 0, VZ, VTH, VSL, VSR, UXD = 5, UZD, UTHD, UFNL, UFTL, USDL, UFNR, UFTR, USDR, ULN, ULT, UPC, X1 = 17 };

static double* TXb(double* tr, int32_t N, int32_t k, int32_t i) { return &tr[i * (N + 1) + k]; }
static double CXb(const double* tr, int32_t N, int32_t k, int32_t i) { return tr[i * (N + 1) + k]; }
static double CUb(const double* tr, int32_t N, int32_t k, int32_t j) { return tr[NX * (N + 1) + j * N + k]; }

/* face frame of a hand: inward normal n, tangent t = rot90(n), depth a
 * (distance of the face from the centre) and half-length ell */
static void face_geom(const bim_instance* in, int32_t f, double n[2], double t[2], double* a, double* ell) {
    static const double nx[4] = {1, 0, -1, 0}, nz[4] = {0, 1, 0, -1};
    n[0] = nx[f];
    n[1] = nz[f];
    t[0] = -n[1];
    t[1] = n[0];
    *a = (f % 2 == 0) ? in->ax : in->az;
    *ell = (f % 2 == 0) ? in->az : in->ax;
}

static int32_t hand_face(int32_t h) { return h == 0 ? -1 : (h - 1) / 3; }

static void control_weights(const bim_instance* in, double R[NU]) {
    const double w[NU] = {in->w_v, in->w_v, in->w_v, in->w_f, in->w_f, in->w_s,
                          in->w_f, in->w_f, in->w_s, in->w_f, in->w_f, in->w_c};
    for (int j = 0; j < NU; ++j) R[j] = w[j];
}

void bim_interval_rows(const bim_instance* in, int32_t mode, int32_t mask_sL, int32_t mask_sR,
                       const double* xk, const double* uk, const double* xk1, double* c, uint8_t* mask,
                       uint8_t* ineq, double* scale, double* J) {
    const int32_t g = mode / 169, hL = (mode / 13) % 13, hR = mode % 13;
    const double mg = in->mass * in->grav, lbar = in->ax > in->az ? in->ax : in->az;
    const double th = xk[2], cth = cos(th), sth = sin(th);
    /* values: kinematic defects 15, wrench sums 6 + 2 x 14 + scaling 3,
     * sine and cosine 2, ground rows 10, hand rows 2 x 8; Jacobians: wrench
     * entries 2 x 12 + 4 + scaling 24, ground 10, hands 2 x 6 */
    FLOPS_ROWS(15 + 6 + 28 + 3 + 2 + 10 + 16);
    FLOPS_JAC(24 + 4 + 24 + 10 + 12);
    for (int r = 0; r < NR; ++r) {
        c[r] = 0.0;
        mask[r] = 1;
        ineq[r] = (r >= 11 && r <= 15) || (r >= 19 && r <= 23) || (r >= 27);
        scale[r] = 1.0; /* physical = c / scale; set below for rows scaled by m g */
        for (int j = 0; j < NL; ++j) J[r * NL + j] = 0.0;
    }
#define JJ(r, v) J[(r) * NL + (v)]
    /* kinematic defects x_{k+1} - x_k - dt (twist, sliding rates) */
    const int32_t vel[NX] = {UXD, UZD, UTHD, USDL, USDR};
    for (int i = 0; i < NX; ++i) {
        c[i] = xk1[i] - xk[i] - in->dt * uk[vel[i] - 5];
        JJ(i, i) = -1.0;
        JJ(i, X1 + i) = 1.0;
        JJ(i, vel[i]) = -in->dt;
    }
    if (mask_sL) mask[3] = 0;
    if (mask_sR) mask[4] = 0;
    /* wrench balance: gravity, hands, ground force at (x + p_c, 0) */
    double Fx = uk[ULT - 5], Fz = uk[ULN - 5] - mg;
    double tau = uk[UPC - 5] * uk[ULN - 5] + xk[1] * uk[ULT - 5];
    JJ(5, ULT) = 1.0;
    JJ(6, ULN) = 1.0;
    JJ(7, UPC) = uk[ULN - 5];
    JJ(7, ULN) = uk[UPC - 5];
    JJ(7, VZ) = uk[ULT - 5];
    JJ(7, ULT) = xk[1];
    for (int side = 0; side < 2; ++side) {
        const int32_t h = side ? hR : hL;
        if (h == 0) continue;
        const int32_t ufn = side ? UFNR : UFNL, uft = side ? UFTR : UFTL, vs = side ? VSR : VSL;
        double n[2], t[2], a, ell;
        face_geom(in, hand_face(h), n, t, &a, &ell);
        const double fn = uk[ufn - 5], ft = uk[uft - 5], s = xk[vs];
        const double Fb[2] = {fn * n[0] + ft * t[0], fn * n[1] + ft * t[1]};
        const double Fwx = cth * Fb[0] - sth * Fb[1], Fwz = sth * Fb[0] + cth * Fb[1];
        Fx += Fwx;
        Fz += Fwz;
        tau += -a * ft - s * fn;
        JJ(5, VTH) += -Fwz;
        JJ(6, VTH) += Fwx;
        JJ(5, ufn) = cth * n[0] - sth * n[1];
        JJ(6, ufn) = sth * n[0] + cth * n[1];
        JJ(5, uft) = cth * t[0] - sth * t[1];
        JJ(6, uft) = sth * t[0] + cth * t[1];
        JJ(7, uft) = -a;
        JJ(7, ufn) = -s;
        JJ(7, vs) = -fn;
    }
    c[5] = Fx / mg;
    c[6] = Fz / mg;
    c[7] = tau / (mg * lbar);
    for (int j = 0; j < NL; ++j) {
        JJ(5, j) /= mg;
        JJ(6, j) /= mg;
        JJ(7, j) /= mg * lbar;
    }
    scale[5] = scale[6] = 1.0 / mg; /* N */
    scale[7] = 1.0 / (mg * lbar);   /* N m */
    /* ground */
    const double mu = in->mu_g, cg = sqrt(1.0 + mu * mu);
    const double xd = uk[0], zd = uk[1], thd = uk[2], ln = uk[ULN - 5], lt = uk[ULT - 5], pc = uk[UPC - 5];
    const double rcx = -in->ax * cth + in->az * sth, rcz = -in->ax * sth - in->az * cth;
    const double w = in->ax * cth * cth + in->az * sth * sth, dw = 2.0 * sth * cth * (in->az - in->ax);
    if (g == 0) { /* stick: no motion, force inside the cone, CoP on the support face */
        c[8] = xd;
        JJ(8, UXD) = 1.0;
        c[9] = zd;
        JJ(9, UZD) = 1.0;
        c[10] = thd;
        JJ(10, UTHD) = 1.0;
    } else if (g == 1) { /* slide: no lift or rotation, friction on the cone edge opposing xd */
        c[8] = zd;
        JJ(8, UZD) = 1.0;
        c[9] = thd;
        JJ(9, UTHD) = 1.0;
        c[10] = (lt * lt - mu * mu * ln * ln) / (mg * mg);
        JJ(10, ULT) = 2.0 * lt / (mg * mg);
        JJ(10, ULN) = -2.0 * mu * mu * ln / (mg * mg);
        /* in physical units the row is the friction force's distance from
         * the cone edge, |lam_t| - mu |lam_n| [N] = c (m g)^2 / (|lam_t| +
         * mu |lam_n|); both forces zero is on the edge */
        const double den = fabs(lt) + mu * fabs(ln);
        scale[10] = den > 0.0 ? den / (mg * mg) : 1.0;
    } else { /* pivot about the lower-left corner: its velocity is zero, the CoP is the corner */
        c[8] = xd - thd * rcz;
        JJ(8, UXD) = 1.0;
        JJ(8, UTHD) = -rcz;
        JJ(8, VTH) = -thd * rcx;
        c[9] = zd + thd * rcx;
        JJ(9, UZD) = 1.0;
        JJ(9, UTHD) = rcx;
        JJ(9, VTH) = -thd * rcz;
        c[10] = pc - rcx;
        JJ(10, UPC) = 1.0;
        JJ(10, VTH) = rcz;
    }
    if (g != 1) { /* cone (stick, pivot) */
        c[11] = (lt - mu * ln) / (mg * cg);
        JJ(11, ULT) = 1.0 / (mg * cg);
        JJ(11, ULN) = -mu / (mg * cg);
        c[12] = (-lt - mu * ln) / (mg * cg);
        JJ(12, ULT) = -1.0 / (mg * cg);
        JJ(12, ULN) = -mu / (mg * cg);
        scale[11] = scale[12] = 1.0 / (mg * cg); /* N */
    } else { /* slide: friction opposes the motion, lam_t xd <= 0 */
        c[11] = lt * xd / mg;
        JJ(11, ULT) = xd / mg;
        JJ(11, UXD) = lt / mg;
        scale[11] = 1.0 / mg; /* W (the friction force's power) */
        mask[12] = 0;
    }
    c[13] = -ln / mg;
    JJ(13, ULN) = -1.0 / mg;
    scale[13] = 1.0 / mg; /* N */
    if (g != 2) { /* CoP within the support half-width w(theta) */
        c[14] = pc - w;
        JJ(14, UPC) = 1.0;
        JJ(14, VTH) = -dw;
        c[15] = -pc - w;
        JJ(15, UPC) = -1.0;
        JJ(15, VTH) = -dw;
    } else {
        mask[14] = mask[15] = 0;
    }
    /* hands */
    const double muh = in->mu_h, ch = sqrt(1.0 + muh * muh);
    for (int side = 0; side < 2; ++side) {
        const int32_t h = side ? hR : hL, b = side ? 24 : 16;
        const int32_t ufn = side ? UFNR : UFNL, uft = side ? UFTR : UFTL, usd = side ? USDR : USDL;
        const int32_t vs = side ? VSR : VSL;
        const double fn = uk[ufn - 5], ft = uk[uft - 5], sd = uk[usd - 5], s = xk[vs];
        if (h == 0) { /* none: no force, the offset stays */
            c[b] = fn / mg;
            JJ(b, ufn) = 1.0 / mg;
            c[b + 1] = ft / mg;
            JJ(b + 1, uft) = 1.0 / mg;
            c[b + 2] = sd;
            JJ(b + 2, usd) = 1.0;
            scale[b] = scale[b + 1] = 1.0 / mg; /* N */
            for (int r = b + 3; r < b + 8; ++r) mask[r] = 0;
            continue;
        }
        double n[2], t[2], a, ell;
        face_geom(in, hand_face(h), n, t, &a, &ell);
        const int32_t kind = (h - 1) % 3;
        mask[b + 1] = mask[b + 2] = 0;
        if (kind == 0) {
            c[b] = sd;
            JJ(b, usd) = 1.0;
            c[b + 3] = (ft - muh * fn) / (mg * ch);
            JJ(b + 3, uft) = 1.0 / (mg * ch);
            JJ(b + 3, ufn) = -muh / (mg * ch);
            c[b + 4] = (-ft - muh * fn) / (mg * ch);
            JJ(b + 4, uft) = -1.0 / (mg * ch);
            JJ(b + 4, ufn) = -muh / (mg * ch);
            scale[b + 3] = scale[b + 4] = 1.0 / (mg * ch); /* N */
        } else {
            const double sg = (kind == 1) ? -1.0 : 1.0; /* slide+: ft - mu fn = 0, sd >= 0 */
            c[b] = (ft + sg * muh * fn) / (mg * ch);
            JJ(b, uft) = 1.0 / (mg * ch);
            JJ(b, ufn) = sg * muh / (mg * ch);
            scale[b] = 1.0 / (mg * ch); /* N */
            c[b + 3] = sg * sd;
            JJ(b + 3, usd) = sg;
            mask[b + 4] = 0;
        }
        c[b + 5] = -fn / mg;
        JJ(b + 5, ufn) = -1.0 / mg;
        scale[b + 5] = 1.0 / mg; /* N */
        c[b + 6] = s - ell;
        JJ(b + 6, vs) = 1.0;
        c[b + 7] = -s - ell;
        JJ(b + 7, vs) = -1.0;
    }
#undef JJ
    for (int r = 0; r < NR; ++r)
        if (!mask[r]) {
            c[r] = 0.0;
            for (int j = 0; j < NL; ++j) J[r * NL + j] = 0.0;
        }
}

static int32_t seg_of(int32_t k, int32_t len, int32_t N) { return (int32_t)(((int64_t)k * len) / N); }

static void interval_masks(const uint16_t* modes, int32_t len, int32_t N, int32_t k, int32_t* mode, int32_t* mL,
                           int32_t* mR) {
    *mode = modes[seg_of(k, len, N)];
    *mL = *mR = 0;
    if (k + 1 < N) {
        const int32_t m1 = modes[seg_of(k + 1, len, N)];
        *mL = hand_face((*mode / 13) % 13) != hand_face((m1 / 13) % 13);
        *mR = hand_face(*mode % 13) != hand_face(m1 % 13);
    }
}

static void load_local(const double* tr, int32_t N, int32_t k, double* xk, double* uk, double* xk1) {
    for (int i = 0; i < NX; ++i) {
        xk[i] = CXb(tr, N, k, i);
        xk1[i] = CXb(tr, N, k + 1, i);
    }
    for (int j = 0; j < NU; ++j) uk[j] = CUb(tr, N, k, j);
}

static void rows_at(const bim_instance* in, const uint16_t* modes, int32_t len, int32_t N, const double* tr, int32_t k,
                    double* c, uint8_t* mask, uint8_t* ineq, double* scale, double* J) {
    double xk[NX], uk[NU], xk1[NX];
    int32_t mode, mL, mR;
    load_local(tr, N, k, xk, uk, xk1);
    interval_masks(modes, len, N, k, &mode, &mL, &mR);
    bim_interval_rows(in, mode, mL, mR, xk, uk, xk1, c, mask, ineq, scale, J);
}

void bim_rows(const bim_instance* in, int32_t len, const uint16_t* modes, int32_t N, const double* traj, double* c,
              uint8_t* mask, double* scale, double* c_init) {
    double cc[NR], sc[NR], J[NR * NL];
    uint8_t mk[NR], iq[NR];
    for (int32_t k = 0; k < N; ++k) {
        rows_at(in, modes, len, N, traj, k, cc, mk, iq, sc, J);
        for (int r = 0; r < NR; ++r) {
            if (c) c[k * NR + r] = cc[r];
            if (mask) mask[k * NR + r] = mk[r];
            if (scale) scale[k * NR + r] = sc[r];
        }
    }
    if (c_init)
        for (int i = 0; i < 3; ++i) c_init[i] = CXb(traj, N, 0, i) - in->start[i];
}

void bim_dense_jacobian(const bim_instance* in, int32_t len, const uint16_t* modes, int32_t N, const double* traj,
                        double* jac) {
    const int64_t nz = (int64_t)(NX + NU) * N + NX, nr = 3 + (int64_t)NR * N;
    double cc[NR], sc[NR], J[NR * NL];
    uint8_t mk[NR], iq[NR];
    memset(jac, 0, sizeof(double) * nz * nr);
    for (int i = 0; i < 3; ++i) jac[i * nz + i] = 1.0;
    for (int32_t k = 0; k < N; ++k) {
        rows_at(in, modes, len, N, traj, k, cc, mk, iq, sc, J);
        for (int r = 0; r < NR; ++r) {
            double* row = &jac[(3 + (int64_t)NR * k + r) * nz];
            for (int j = 0; j < NL; ++j) row[(int64_t)(NX + NU) * k + j] = J[r * NL + j];
        }
    }
}

void bim_cold_start(const bim_instance* in, int32_t N, double* traj) {
    for (int32_t k = 0; k <= N; ++k) {
        const double al = (double)k / (double)N;
        for (int i = 0; i < 3; ++i) *TXb(traj, N, k, i) = (1.0 - al) * in->start[i] + al * in->goal[i];
        *TXb(traj, N, k, 3) = 0.0;
        *TXb(traj, N, k, 4) = 0.0;
    }
    for (int32_t k = 0; k < N; ++k)
        for (int j = 0; j < NU; ++j) traj[NX * (N + 1) + j * N + k] = (j == ULN - 5) ? in->mass * in->grav : 0.0;
}

double bim_cost(const bim_instance* in, int32_t N, const double* tr) {
    double R[NU], J = 0.0;
    FLOPS(3 * 4 + (int64_t)NU * N * 3);
    control_weights(in, R);
    for (int i = 0; i < 3; ++i) {
        const double e = CXb(tr, N, N, i) - in->goal[i];
        J += in->w_terminal * e * e;
    }
    for (int32_t k = 0; k < N; ++k)
        for (int j = 0; j < NU; ++j) {
            const double u = CUb(tr, N, k, j);
            J += R[j] * u * u;
        }
    return J;
}

static double row_y(int32_t is_ineq, double lam, double beta, double c) {
    const double y = lam + beta * c;
    if (is_ineq) return y > 0.0 ? y : 0.0;
    return y;
}

static double row_al(int32_t is_ineq, double lam, double beta, double c) {
    if (!is_ineq) return lam * c + 0.5 * beta * c * c;
    const double y = lam + beta * c;
    const double p = y > 0.0 ? y : 0.0;
    return (p * p - lam * lam) / (2.0 * beta);
}

double bim_al_merit(const bim_instance* in, int32_t len, const uint16_t* modes, int32_t N, const double* traj,
                    const double* lam, double beta) {
    double L = bim_cost(in, N, traj);
    for (int i = 0; i < 3; ++i) L += row_al(0, lam[i], beta, CXb(traj, N, 0, i) - in->start[i]);
    double cc[NR], sc[NR], J[NR * NL];
    uint8_t mk[NR], iq[NR];
    COUNT_ROWS(1, 0);
    for (int32_t k = 0; k < N; ++k) {
        rows_at(in, modes, len, N, traj, k, cc, mk, iq, sc, J);
        for (int r = 0; r < NR; ++r)
            if (mk[r]) {
                L += row_al(iq[r], lam[3 + NR * k + r], beta, cc[r]);
                FLOPS(6);
            }
    }
    COUNT_ROWS(1, 1);
    return L;
}

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

static void chol_solve(int n, const double* L, const double* b, double* x) {
    double y[NW];
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

int32_t bim_gn_step(const bim_instance* in, int32_t len, const uint16_t* modes, int32_t N, const double* traj,
                    const double* lam, double beta, double rho, double* dz, double* grad) {
    const int32_t NZ = NX + NU;
    double* Kg = (double*)malloc(sizeof(double) * NW * NX * (size_t)N); /* K_k = -S^-1 C (17 x 5) */
    double* kg = (double*)malloc(sizeof(double) * NW * (size_t)N);      /* k_k = -S^-1 g_w */
    const int64_t nz = (int64_t)NZ * N + NX;
    for (int64_t i = 0; i < nz; ++i) grad[i] = 0.0;
    double R[NU];
    control_weights(in, R);
    double V[NX * NX] = {0}, v[NX] = {0};
    for (int i = 0; i < 3; ++i) {
        V[i * NX + i] = 2.0 * in->w_terminal;
        v[i] = 2.0 * in->w_terminal * (CXb(traj, N, N, i) - in->goal[i]);
        grad[(int64_t)NZ * N + i] += v[i];
    }
    double cc[NR], sc[NR], Jl[NR * NL];
    uint8_t mk[NR], iq[NR];
    int32_t ok = 0;
    COUNT_ROWS(0, 0);
    for (int32_t k = N - 1; k >= 0; --k) {
        rows_at(in, modes, len, N, traj, k, cc, mk, iq, sc, Jl);
        /* local Gauss-Newton model of the AL over (x_k, u_k, x_{k+1}) */
        double H[NL * NL], g[NL];
        memset(H, 0, sizeof(H));
        memset(g, 0, sizeof(g));
        FLOPS(NU * 3);
        for (int j = 0; j < NU; ++j) {
            H[(NX + j) * NL + NX + j] += 2.0 * R[j];
            g[NX + j] += 2.0 * R[j] * CUb(traj, N, k, j);
        }
        for (int r = 0; r < NR; ++r) {
            if (!mk[r]) continue;
            const double l = lam[3 + NR * (int64_t)k + r];
            if (iq[r] && !(l + beta * cc[r] > 0.0)) continue;
            const double y = row_y(iq[r], l, beta, cc[r]);
#ifdef ORC_COUNT_FLOPS
            {
                int nnz = 0;
                for (int i = 0; i < NL; ++i) nnz += Jl[r * NL + i] != 0.0;
                FLOPS(2 + 3 * nnz + nnz * (nnz + 1));
            }
#endif
            for (int i = 0; i < NL; ++i) {
                if (Jl[r * NL + i] == 0.0) continue;
                g[i] += y * Jl[r * NL + i];
                for (int j = 0; j < NL; ++j) H[i * NL + j] += beta * Jl[r * NL + i] * Jl[r * NL + j];
            }
        }
        for (int i = 0; i < NX; ++i) grad[(int64_t)NZ * k + i] += g[i];
        for (int j = 0; j < NU; ++j) grad[(int64_t)NZ * k + NX + j] += g[NX + j];
        for (int i = 0; i < NX; ++i) grad[(int64_t)NZ * (k + 1) + i] += g[NX + NU + i];
        /* S_k = H_ww + rho I + [0 0; 0 V_{k+1}], C_k = H_wx, g_w */
        double S[NW * NW], C[NW * NX], gw[NW], L[NW * NW];
        for (int i = 0; i < NW; ++i) {
            for (int j = 0; j < NW; ++j) S[i * NW + j] = H[(NX + i) * NL + NX + j];
            S[i * NW + i] += rho;
            for (int j = 0; j < NX; ++j) C[i * NX + j] = H[(NX + i) * NL + j];
            gw[i] = g[NX + i];
        }
        for (int i = 0; i < NX; ++i) {
            for (int j = 0; j < NX; ++j) S[(NU + i) * NW + NU + j] += V[i * NX + j];
            gw[NU + i] += v[i];
        }
        FLOPS(NW + 15 + NX); /* rho, V_{k+1} (lower triangle), v_{k+1} */
        if (chol(NW, S, L) != 0) {
            ok = -1;
            break;
        }
        double col[NW], sol[NW];
        for (int j = 0; j < NX; ++j) {
            for (int i = 0; i < NW; ++i) col[i] = C[i * NX + j];
            chol_solve(NW, L, col, sol);
            for (int i = 0; i < NW; ++i) Kg[(int64_t)NW * NX * k + i * NX + j] = -sol[i];
        }
        chol_solve(NW, L, gw, sol);
        for (int i = 0; i < NW; ++i) kg[(int64_t)NW * k + i] = -sol[i];
        double Vn[NX * NX], vn[NX];
        FLOPS(15 * NW * 2 + NX * NW * 2); /* symmetric V (lower triangle) and v */
        for (int i = 0; i < NX; ++i) {
            for (int j = 0; j < NX; ++j) {
                double s = H[i * NL + j];
                for (int p = 0; p < NW; ++p) s += C[p * NX + i] * Kg[(int64_t)NW * NX * k + p * NX + j];
                Vn[i * NX + j] = s;
            }
            double s = g[i];
            for (int p = 0; p < NW; ++p) s += C[p * NX + i] * kg[(int64_t)NW * k + p];
            vn[i] = s;
        }
        for (int i = 0; i < NX; ++i)
            for (int j = 0; j < NX; ++j) V[i * NX + j] = 0.5 * (Vn[i * NX + j] + Vn[j * NX + i]);
        for (int i = 0; i < NX; ++i) v[i] = vn[i];
    }
    if (ok == 0) {
        /* initial block: V_0 + rho I + beta on the three pose rows */
        double H0[NX * NX], g0[NX], L0[NX * NX], dx[NX];
        for (int i = 0; i < NX * NX; ++i) H0[i] = V[i];
        for (int i = 0; i < NX; ++i) {
            H0[i * NX + i] += rho;
            g0[i] = v[i];
        }
        for (int i = 0; i < 3; ++i) {
            const double y = row_y(0, lam[i], beta, CXb(traj, N, 0, i) - in->start[i]);
            H0[i * NX + i] += beta;
            g0[i] += y;
            grad[i] += y;
        }
        if (chol(NX, H0, L0) != 0) {
            ok = -1;
        } else {
            double yv[NX];
            for (int i = 0; i < NX; ++i) {
                double s = g0[i];
                for (int p = 0; p < i; ++p) s -= L0[i * NX + p] * yv[p];
                yv[i] = s / L0[i * NX + i];
            }
            for (int i = NX - 1; i >= 0; --i) {
                double s = yv[i];
                for (int p = i + 1; p < NX; ++p) s -= L0[p * NX + i] * dx[p];
                dx[i] = s / L0[i * NX + i];
            }
            for (int i = 0; i < NX; ++i) dx[i] = -dx[i];
            for (int i = 0; i < NX; ++i) dz[i] = dx[i];
            FLOPS((int64_t)N * NW * 2 * NX);
            for (int32_t k = 0; k < N; ++k) {
                double dw[NW];
                for (int i = 0; i < NW; ++i) {
                    double s = kg[(int64_t)NW * k + i];
                    for (int j = 0; j < NX; ++j) s += Kg[(int64_t)NW * NX * k + i * NX + j] * dx[j];
                    dw[i] = s;
                }
                for (int j = 0; j < NU; ++j) dz[(int64_t)NZ * k + NX + j] = dw[j];
                for (int i = 0; i < NX; ++i) {
                    dz[(int64_t)NZ * (k + 1) + i] = dw[NU + i];
                    dx[i] = dw[NU + i];
                }
            }
        }
    }
    COUNT_ROWS(1, 1);
    free(Kg);
    free(kg);
    return ok;
}

static void axpy_traj(int32_t N, const double* tr, double alpha, const double* dz, double* out) {
    const int32_t NZ = NX + NU;
    FLOPS(2 * ((int64_t)NZ * N + NX));
    for (int32_t k = 0; k <= N; ++k)
        for (int i = 0; i < NX; ++i) out[i * (N + 1) + k] = CXb(tr, N, k, i) + alpha * dz[(int64_t)NZ * k + i];
    for (int32_t k = 0; k < N; ++k)
        for (int j = 0; j < NU; ++j)
            out[NX * (N + 1) + j * N + k] = CUb(tr, N, k, j) + alpha * dz[(int64_t)NZ * k + NX + j];
}

typedef struct {
    double viol, stat, comp, vphys;
    int finite;
} meas;

static void measures(const bim_instance* in, int32_t len, const uint16_t* modes, int32_t N, const double* traj,
                     const double* lam, double beta, double* y, double* grad, meas* m) {
    const int32_t NZ = NX + NU;
    const int64_t nz = (int64_t)NZ * N + NX;
    double R[NU];
    control_weights(in, R);
    for (int64_t i = 0; i < nz; ++i) grad[i] = 0.0;
    m->viol = m->comp = m->vphys = 0.0;
    m->finite = 1;
    for (int i = 0; i < 3; ++i)
        grad[(int64_t)NZ * N + i] += 2.0 * in->w_terminal * (CXb(traj, N, N, i) - in->goal[i]);
    for (int32_t k = 0; k < N; ++k)
        for (int j = 0; j < NU; ++j) grad[(int64_t)NZ * k + NX + j] += 2.0 * R[j] * CUb(traj, N, k, j);
    for (int i = 0; i < 3; ++i) {
        const double c = CXb(traj, N, 0, i) - in->start[i];
        y[i] = row_y(0, lam[i], beta, c);
        grad[i] += y[i];
        if (fabs(c) > m->viol) m->viol = fabs(c);
        if (fabs(c) > m->vphys) m->vphys = fabs(c);
        if (!isfinite(c)) m->finite = 0;
    }
    double cc[NR], sc[NR], Jl[NR * NL];
    uint8_t mk[NR], iq[NR];
    for (int32_t k = 0; k < N; ++k) {
        rows_at(in, modes, len, N, traj, k, cc, mk, iq, sc, Jl);
        for (int r = 0; r < NR; ++r) {
            const int64_t idx = 3 + (int64_t)NR * k + r;
            if (!mk[r]) {
                y[idx] = 0.0;
                continue;
            }
            if (!isfinite(cc[r])) m->finite = 0;
            const double yr = row_y(iq[r], lam[idx], beta, cc[r]);
            y[idx] = yr;
            FLOPS(6);
#ifdef ORC_COUNT_FLOPS
            if (yr != 0.0) {
                int nnz = 0;
                for (int i = 0; i < NL; ++i) nnz += Jl[r * NL + i] != 0.0;
                FLOPS(2 * nnz);
            }
#endif
            const double vv = iq[r] ? (cc[r] > 0.0 ? cc[r] : 0.0) : fabs(cc[r]);
            if (vv > m->viol) m->viol = vv;
            if (vv / sc[r] > m->vphys) m->vphys = vv / sc[r];
            if (iq[r] && fabs(yr * cc[r]) > m->comp) m->comp = fabs(yr * cc[r]);
            if (yr != 0.0)
                for (int i = 0; i < NL; ++i) grad[(int64_t)NZ * k + i] += yr * Jl[r * NL + i];
        }
    }
    m->stat = 0.0;
    for (int64_t i = 0; i < nz; ++i) {
        if (!isfinite(grad[i])) m->finite = 0;
        if (fabs(grad[i]) > m->stat) m->stat = fabs(grad[i]);
    }
}

int32_t bim_solve(const bim_instance* in, int32_t len, const uint16_t* modes, int32_t N, const double* warm,
                  const orc_opts* opt, double* out_traj, double* out_lam, orc_result* res) {
    return bim_solve_ex(in, len, modes, N, warm, NULL, opt, out_traj, out_lam, res);
}

int32_t bim_solve_ex(const bim_instance* in, int32_t len, const uint16_t* modes, int32_t N, const double* warm,
                     const double* warm_lam, const orc_opts* opt, double* out_traj, double* out_lam,
                     orc_result* res) {
    const int64_t nt = (int64_t)(NX + NU) * N + NX, nl = 3 + (int64_t)NR * N;
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
        bim_cold_start(in, N, z);
    double beta = opt->beta0, rho = opt->rho0, eta = INFINITY;
    int32_t inner = 0, it = 0, status = ORC_MAX_ITER, n_outer = 0, n_rej = 0;
    meas m;
    for (it = 0; it < opt->max_iters; ++it) {
        measures(in, len, modes, N, z, lam, beta, y, grad, &m);
        if (!m.finite) {
            status = ORC_NONFINITE;
            break;
        }
        /* stop test as in orc_solve: scaled rows within eps_primal, rows in
         * physical units within half eps_feas, stationarity relative to
         * max(1, |J|) (Sec. III-C "Stopping and scoring") */
        const double eps_d = orc_stat_tol(opt, beta, bim_cost(in, N, z));
        if (m.viol <= opt->eps_primal && m.vphys <= 0.5 * opt->eps_feas && m.stat <= eps_d &&
            m.comp <= opt->eps_comp) {
            memcpy(lam, y, sizeof(double) * nl);
            status = ORC_CONVERGED;
            break;
        }
        const double omega = fmax(eps_d, opt->omega_ratio * m.viol);
        const int32_t solved = m.stat <= omega;
        if (solved || inner >= opt->max_inner) {
            memcpy(lam, y, sizeof(double) * nl);
            if (solved && m.viol > opt->eps_primal && m.viol > opt->eta_ratio * eta)
                beta = fmin(opt->beta_max, beta * opt->beta_growth);
            eta = m.viol;
            inner = 0;
            ++n_outer;
        }
        int32_t fac = -1;
        for (int32_t r = 0; fac != 0 && r <= opt->max_factor_retries; ++r) {
            if (r > 0) rho = fmin(opt->rho_max, rho * 10.0);
            fac = bim_gn_step(in, len, modes, N, z, lam, beta, rho, dz, grad);
        }
        ++inner;
        if (fac != 0) {
            ++n_rej;
            continue;
        }
        double D = 0.0;
        for (int64_t i = 0; i < nt; ++i) D += grad[i] * dz[i];
        FLOPS(2 * nt);
        const double phi0 = bim_al_merit(in, len, modes, N, z, lam, beta);
        const double slack = opt->ls_slack * fabs(phi0);
        const int32_t flat = fabs(D) <= slack;
        double alpha = 0.0;
        for (int32_t i = 0; i < opt->n_alpha; ++i) {
            const double a = ldexp(1.0, -i);
            axpy_traj(N, z, a, dz, zt);
            const double phi = bim_al_merit(in, len, modes, N, zt, lam, beta);
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
    if (status != ORC_CONVERGED) measures(in, len, modes, N, z, lam, beta, y, grad, &m);
    res->cost = bim_cost(in, N, z);
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
    res->n_curv_fail = 0;
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

typedef struct {
    const bim_instance* insts;
    const int32_t *inst_idx, *lens, *Ns;
    const uint16_t* modes;
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
} bctx;

static void* bworker(void* arg) {
    bctx* b = (bctx*)arg;
    for (;;) {
        pthread_mutex_lock(&b->lock);
        const int64_t i = b->next++;
        pthread_mutex_unlock(&b->lock);
        if (i >= b->n) break;
        double* tr = b->out_traj ? b->out_traj + i * b->traj_stride : NULL;
        const double* w = b->warm ? b->warm + i * b->warm_stride : NULL;
        double* lam = b->out_lam ? b->out_lam + i * b->lam_stride : NULL;
        const double* wl = b->warm_lam ? b->warm_lam + i * b->lam_stride : NULL;
        bim_solve_ex(&b->insts[b->inst_idx[i]], b->lens[i], b->modes + i * b->lmax, b->Ns[i], w, wl, b->opt, tr,
                     lam, &b->res[i]);
    }
    return NULL;
}

int32_t bim_solve_batch(const bim_instance* insts, const int32_t* inst_idx, const int32_t* lens,
                        const uint16_t* modes, int32_t lmax, const int32_t* Ns, int64_t n, const orc_opts* opt,
                        int32_t nthreads, double* out_traj, int64_t traj_stride, orc_result* res) {
    return bim_solve_batch_ex(insts, inst_idx, lens, modes, lmax, Ns, n, opt, nthreads, NULL, 0, NULL, out_traj,
                              traj_stride, NULL, 0, res);
}

int32_t bim_solve_batch_ex(const bim_instance* insts, const int32_t* inst_idx, const int32_t* lens,
                           const uint16_t* modes, int32_t lmax, const int32_t* Ns, int64_t n, const orc_opts* opt,
                           int32_t nthreads, const double* warm, int64_t warm_stride, const double* warm_lam,
                           double* out_traj, int64_t traj_stride, double* out_lam, int64_t lam_stride,
                           orc_result* res) {
    bctx b;
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
    for (int32_t t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, bworker, &b);
    for (int32_t t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&b.lock);
    return 0;
}
