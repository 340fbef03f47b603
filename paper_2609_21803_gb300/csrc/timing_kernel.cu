// timing_kernel.cu -- the pushing TO with the interval durations among the
// controls (timing optimisation: Sec. III-C, "When timing is optimized,
// interval durations are included in the controls"; the optimised time step
// under the benchmark's duration bound of Sec. IV-A).  One warp per TO,
// persistent, FP32 with compensated state storage and an FP64 certificate,
// like the fixed-step evaluator (eval_kernel.cu).
//
// Variables of interval k: state x_k = (x, y, theta, s, tau), control
// u_k = (f_n, f_t, sdot, h).  h_k is the interval's duration and tau the
// elapsed time, which carries the duration bound and keeps the problem
// stage-wise.  Rows (14 per interval, fixed positions):
//   0..3   dynamics (x_{k+1} - x_k - h_k f(x_k, u_k)) / sigma_i
//   4      mode equality;  5..10 the fixed-step inequalities
//   11     elapsed time (tau_{k+1} - tau_k - h_k) / sqrt(3)
//   12, 13 h_min - h_k <= 0 and h_k - h_max <= 0
// plus four initial rows (x, y, theta at the start pose, tau_0 = 0) and the
// terminal row tau_N - T <= 0.  The dynamics rows are bilinear in h and f,
// so the Newton model's curvature gains the cross terms between h_k and
// the stage's other variables.
//
// One iteration (the method of Sec. III-C, as in eval_kernel.cu):
//   A  stage-parallel: rows, PHR multiplier estimates, measures, the local
//      AL model over (u_k, x_{k+1}, x_k) and the elimination of its u block;
//   B  the state steps by the lane-parallel elimination of the
//      block-tridiagonal system (lanes fold their stages, a shuffle tree
//      over the lanes, a 10 x 10 root solve, back-substitution);
//   C  the control steps, stage-parallel;
//   D  trial merits of alpha in {1, 1/2, ..., 1/64};
//   E  compensated update.

#include <cuda_runtime.h>
#include <cuda/annotated_ptr>
#include <math.h>
#include <stdint.h>

#include "comet_internal.h"

namespace comet {
namespace {

constexpr unsigned kFullT = 0xffffffffu;
constexpr int TX = 5, TU = 4, TW = TX + TU;   // state, control, stage variables
constexpr int TR = 14;                        // rows per interval
constexpr int TLOC = 2 * TX + TU;             // local variables (u_k, x_{k+1}, x_k)
constexpr int TM = TLOC + 1;                  // local model with the rhs row
constexpr int TMTRI = TM * (TM + 1) / 2;      // 120
constexpr int kModeFreeT = 12;
constexpr float kInvSqrt3 = 0.57735026918962576f;
constexpr float kSqrt3 = 1.7320508075688772f;

// the four initial rows pin x, y, theta (to the start pose) and tau_0 = 0;
// row i acts on state component tinit_comp(i)
__host__ __device__ constexpr int tinit_comp(int i) { return i < 3 ? i : 4; }

// local model order: u 0..3, y = x_{k+1} 4..8, x = x_k 9..13, rhs 14
constexpr int LU = 0, LY = 4, LX = 9, LR = 14;

// Stage record (kTRec floats, chunk-major float4 chunks as in eval_kernel):
//   R_UF  0..9    u-block Cholesky factor (lower triangle, 1/l_jj on the diagonal)
//   R_CP  10..53  coupling columns: local row 4 + c (c = 0..10) x u column j at 10 + 4c + j
//   R_PD  54      +1 / -1: the u block was positive definite
//   R_RED 56..120 reduced lower triangle over local rows 4..14 (no (rhs, rhs) entry):
//                 the stage's element in (dx_{k+1}, dx_k); once the elimination of
//                 phase B has taken a stage's node, floats 56..125 hold that node's
//                 factor and solved columns
constexpr int kTRec = 128;
constexpr int R_UF = 0, R_CP = 10, R_PD = 54, R_RED = 56;

__device__ __forceinline__ float twarp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullT, v, o);
    return v;
}
__device__ __forceinline__ float twarp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFullT, v, o));
    return v;
}
__device__ __forceinline__ double twarp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullT, v, o);
    return v;
}
__device__ __forceinline__ double twarp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFullT, v, o));
    return v;
}

// error-free sum a + b = s + e (Knuth two-sum)
__device__ __forceinline__ void two_sum_t(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__host__ __device__ constexpr int ttri(int i, int j) { return i * (i + 1) / 2 + j; }

__device__ __forceinline__ void tface_nt(int face, float& nx, float& ny) {
    nx = (face == 0) ? 1.f : ((face == 2) ? -1.f : 0.f);
    ny = (face == 1) ? 1.f : ((face == 3) ? -1.f : 0.f);
}

struct TModeInfo {
    int face, kind;  // kind 0 stick, 1 slide+, 2 slide-, 3 free motion
    bool smask;      // s-row of the dynamics masked
};

__device__ __forceinline__ TModeInfo tmode_of(unsigned char b) {
    TModeInfo mi;
    mi.face = b & 3;
    mi.kind = (b >> 2) & 3;
    mi.smask = (b >> 4) & 1;
    return mi;
}

// ---------------------------------------------------------------- the rows

// Rows of interval k (scaled values, physical factors, presence) and the
// pieces of their Jacobians.  xk: x_k rounded to FP32; dx: x_{k+1} - x_k,
// with dx[2] + ex[0] the exact theta difference and xk[3] + ex[1] = s_k.
struct TRows {
    float c[TR];
    float phys[TR];
    bool on[TR];
    float ax[4][4];   // d c_r / d (x, y, theta, s)_k, dynamics rows
    float au[4][4];   // d c_r / d (f_n, f_t, sdot, h)
    float ay[4];      // d c_r / d x_{k+1, r}
    float lu[5][3];   // rows 4..8 over (f_n, f_t, sdot)
    // unscaled pieces of f for the curvature
    float f0, f1, ct, st, kf;
    float fx02, fx12, fx23;
    float fu00, fu01, fu10, fu11, fu20, fu21;
};

__device__ __forceinline__ void trows(const DevInstance& P, const TModeInfo& mi, float h_min, float h_max,
                                      const float xk[TX], const float dx[TX], const float ex[2], const float u[TU],
                                      TRows& R) {
    float nx, ny;
    tface_nt(mi.face, nx, ny);
    const float tx = -ny, ty = nx;
    const float a = P.a[mi.face], ell = P.ell[mi.face];
    const bool free = mi.kind == 3;
    const float k = free ? 0.f : P.kappa, ic2 = P.inv_c2;
    const float th = xk[2], s = xk[3];
    const float fn = u[0], ft = u[1], sd = u[2], h = u[3];
    float st, ct;
    sincosf(th, &st, &ct);
    const float vx = k * (fn * nx + ft * tx);
    const float vy = k * (fn * ny + ft * ty);
    const float w = k * (-a * ft - s * fn) * ic2;
    const float f[4] = {ct * vx - st * vy, st * vx + ct * vy, w, sd};
    R.f0 = f[0];
    R.f1 = f[1];
    R.ct = ct;
    R.st = st;
    R.kf = k;
    R.fx02 = -st * vx - ct * vy;
    R.fx12 = ct * vx - st * vy;
    R.fx23 = -k * fn * ic2;
    R.fu00 = k * (ct * nx - st * ny);
    R.fu01 = k * (ct * tx - st * ty);
    R.fu10 = k * (st * nx + ct * ny);
    R.fu11 = k * (st * tx + ct * ty);
    R.fu20 = -k * s * ic2;
    R.fu21 = -k * a * ic2;
    const float Fu[4][3] = {{R.fu00, R.fu01, 0.f}, {R.fu10, R.fu11, 0.f}, {R.fu20, R.fu21, 0.f}, {0.f, 0.f, 1.f}};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float is = P.inv_sigma[r];
        R.c[r] = (dx[r] - h * f[r]) * is;
        R.phys[r] = 1.f / is;
        R.on[r] = true;
#pragma unroll
        for (int j = 0; j < 4; ++j) R.ax[r][j] = (r == j) ? -is : 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) R.au[r][j] = -h * Fu[r][j] * is;
        R.au[r][3] = -f[r] * is;
        R.ay[r] = is;
    }
    {
        // c_2 sigma_2 = dtheta + h (kappa / c^2) (a f_t + s f_n) in
        // double-float: the product pairs by fma, the sums by two_sum
        const float kh = free ? 0.f : P.kc_hi, kl = free ? 0.f : P.kc_lo;
        const float hk = h * kh, hke = fmaf(h, kh, -hk) + h * kl;
        const float p = a * ft, pe = fmaf(a, ft, -p) + P.a_lo[mi.face] * ft;
        const float q = s * fn, qe = fmaf(s, fn, -q) + ex[1] * fn;
        float m, me;
        two_sum_t(p, q, m, me);
        me += pe + qe;
        const float km = hk * m, kme = fmaf(hk, m, -km) + (hk * me + hke * m);
        float t, te;
        two_sum_t(dx[2], km, t, te);
        R.c[2] = (t + (te + ex[0] + kme)) * P.inv_sigma[2];
    }
    R.ax[0][2] += -h * R.fx02 * P.inv_sigma[0];
    R.ax[1][2] += -h * R.fx12 * P.inv_sigma[1];
    R.ax[2][3] += -h * R.fx23 * P.inv_sigma[2];
    if (mi.smask) R.on[3] = false;

    const float mu = P.mu, sc = P.sc_cone;
    const bool stick = mi.kind == 0;
    const float sg = (mi.kind == 1) ? -1.f : 1.f;
    if (free) {
        R.c[4] = fn;
        R.phys[4] = 1.f;
        R.lu[0][0] = 1.f; R.lu[0][1] = 0.f; R.lu[0][2] = 0.f;
    } else if (stick) {
        R.c[4] = sd;
        R.phys[4] = 1.f;
        R.lu[0][0] = 0.f; R.lu[0][1] = 0.f; R.lu[0][2] = 1.f;
    } else {
        R.c[4] = sc * (ft + sg * mu * fn);
        R.phys[4] = 1.f / sc;
        R.lu[0][0] = sc * sg * mu; R.lu[0][1] = sc; R.lu[0][2] = 0.f;
    }
    R.on[4] = true;
    R.c[5] = sc * (ft - mu * fn);
    R.lu[1][0] = -sc * mu; R.lu[1][1] = sc; R.lu[1][2] = 0.f;
    R.c[6] = sc * (-ft - mu * fn);
    R.lu[2][0] = -sc * mu; R.lu[2][1] = -sc; R.lu[2][2] = 0.f;
    R.phys[5] = R.phys[6] = 1.f / sc;
    R.on[5] = R.on[6] = stick;
    R.c[7] = sg * sd;
    R.lu[3][0] = 0.f; R.lu[3][1] = 0.f; R.lu[3][2] = sg;
    R.phys[7] = 1.f;
    R.on[7] = !stick && !free;
    R.c[8] = -fn;
    R.lu[4][0] = -1.f; R.lu[4][1] = 0.f; R.lu[4][2] = 0.f;
    R.phys[8] = 1.f;
    R.on[8] = !free;
    R.c[9] = s - ell;
    R.c[10] = -s - ell;
    R.phys[9] = R.phys[10] = 1.f;
    R.on[9] = R.on[10] = !free;
    // elapsed time and the duration bounds
    R.c[11] = (dx[4] - h) * kInvSqrt3;
    R.phys[11] = kSqrt3;
    R.on[11] = true;
    R.c[12] = h_min - h;
    R.c[13] = h - h_max;
    R.phys[12] = R.phys[13] = 1.f;
    R.on[12] = R.on[13] = true;
#pragma unroll
    for (int r = 0; r < TR; ++r)
        if (!R.on[r]) R.c[r] = 0.f;
}

__device__ __forceinline__ bool tineq(int r) { return (r >= 5 && r <= 10) || r >= 12; }

// Nonzero pattern of dynamics row r over the local model (u 0..3, y 4..8,
// x 9..13), ascending; -1 pads.
__host__ __device__ constexpr int tdyn_nz(int r, int a) {
    return r == 0 ? (a == 0 ? 0 : a == 1 ? 1 : a == 2 ? 3 : a == 3 ? 4 : a == 4 ? 9 : 11)
         : r == 1 ? (a == 0 ? 0 : a == 1 ? 1 : a == 2 ? 3 : a == 3 ? 5 : a == 4 ? 10 : 11)
         : r == 2 ? (a == 0 ? 0 : a == 1 ? 1 : a == 2 ? 3 : a == 3 ? 6 : a == 4 ? 11 : 12)
                  : (a == 0 ? 2 : a == 1 ? 3 : a == 2 ? 7 : a == 3 ? 12 : -1);
}

__device__ __forceinline__ float trow_al(bool ineq, float lam, float beta, float inv2b, float c) {
    if (!ineq) return lam * c + 0.5f * beta * c * c;
    const float t = fmaxf(lam + beta * c, 0.f);
    return (t * t - lam * lam) * inv2b;
}

// ------------------------------------------------------------ shared memory

struct TSmem {
    unsigned char* mb;  // [Nmax] mode byte: face | kind << 2 | smask << 4
    float* xh;          // [5][N+1] state, high part
    float* xl;          // [5][N+1] state, low part
    float* us;          // [4][N]
    float* lam;         // [4 + 14 N + 1]: initial rows, interval rows, terminal row
    float* dz;          // [9 N + 5] interleaved step
    float* gr;          // [9 N + 5] interleaved AL gradient
};

__host__ __device__ inline size_t tsmem_floats(int Nmax) {
    const size_t f = (size_t)(Nmax + 3) / 4 + (size_t)2 * TX * (Nmax + 1) +
                     (size_t)TU * Nmax + 5 + (size_t)TR * Nmax + 2 * ((size_t)TW * Nmax + TX);
    return (f + 3) / 4 * 4;
}

__device__ __forceinline__ TSmem tcarve(float* base, int Nmax) {
    TSmem s;
    float* p = base;
    s.mb = reinterpret_cast<unsigned char*>(p); p += (Nmax + 3) / 4;
    s.xh = p; p += TX * (Nmax + 1);
    s.xl = p; p += TX * (Nmax + 1);
    s.us = p; p += TU * Nmax;
    s.lam = p; p += 5 + TR * Nmax;
    s.dz = p; p += TW * Nmax + TX;
    s.gr = p;
    return s;
}

struct TCtx {
    const DevInstance* P;
    int N, Nmax, lane;
    float h_min, h_max, T;
    TSmem sm;
    float* rec;
};

__device__ __forceinline__ float4* trec(const TCtx& C, int q, int k) {
    return reinterpret_cast<float4*>(C.rec + 4 * ((size_t)q * C.Nmax + k));
}

// record stores with the persisting (evict-last) L2 priority: the resident
// warps' records fit in L2 and are rewritten every iteration (as in
// eval_kernel.cu)
__device__ __forceinline__ void trec_st(const TCtx& C, int q, int k, float4 v) {
    cuda::annotated_ptr<float4, cuda::access_property::persisting> p(trec(C, q, k));
    *p = v;
}

// states of interval k from the compensated storage, the low parts moved by
// alpha dz (alpha = 0: the iterate; dz is not read then, since it may hold
// the gradient's parked pieces or nothing yet)
__device__ __forceinline__ void tstage(const TCtx& C, int k, float alpha, float xk[TX], float dx[TX], float ex[2],
                                       float u[TU]) {
    const int Np1 = C.N + 1;
    const TSmem& S = C.sm;
    float h0[TX], h1[TX], l0[TX], l1[TX];
#pragma unroll
    for (int i = 0; i < TX; ++i) {
        h0[i] = S.xh[i * Np1 + k];
        h1[i] = S.xh[i * Np1 + k + 1];
        l0[i] = S.xl[i * Np1 + k] + (alpha != 0.f ? alpha * S.dz[TW * k + i] : 0.f);
        l1[i] = S.xl[i * Np1 + k + 1] + (alpha != 0.f ? alpha * S.dz[TW * (k + 1) + i] : 0.f);
    }
#pragma unroll
    for (int i = 0; i < TX; ++i) {
        xk[i] = h0[i] + l0[i];
        dx[i] = (h1[i] - h0[i]) + (l1[i] - l0[i]);
    }
    float e;
    two_sum_t(h1[2], -h0[2], dx[2], e);
    ex[0] = e + (l1[2] - l0[2]);
    two_sum_t(h0[3], l0[3], xk[3], ex[1]);
#pragma unroll
    for (int j = 0; j < TU; ++j) u[j] = S.us[j * C.N + k] + (alpha != 0.f ? alpha * S.dz[TW * k + TX + j] : 0.f);
}

__device__ __forceinline__ float tinit_row(const TCtx& C, int i, float alpha) {
    const TSmem& S = C.sm;
    const int q = tinit_comp(i), Np1 = C.N + 1;
    return (S.xh[q * Np1] - (i < 3 ? C.P->start[i] : 0.f)) + (S.xl[q * Np1] + (alpha != 0.f ? alpha * S.dz[q] : 0.f));
}
__device__ __forceinline__ float tterm_row(const TCtx& C, float alpha) {
    const TSmem& S = C.sm;
    const int N = C.N, Np1 = N + 1;
    return (S.xh[4 * Np1 + N] - C.T) + (S.xl[4 * Np1 + N] + (alpha != 0.f ? alpha * S.dz[TW * N + 4] : 0.f));
}

struct TMeasures {
    float viol, stat, comp, vphys, cost;
    bool finite;
};

// Phase A: measures, AL gradient (sm.gr) and the stage records.  With
// `update` the multipliers first take their PHR estimates at beta_old.
__device__ TMeasures tphase_a(TCtx& C, float beta, float rho, bool curvature, bool update, float beta_old) {
    const DevInstance& P = *C.P;
    const int N = C.N, Np1 = N + 1, lane = C.lane;
    TSmem& S = C.sm;
    float viol = 0.f, comp = 0.f, vph = 0.f, jc = 0.f;
    bool finite = true;
#pragma unroll 1
    for (int k = lane; k < N; k += 32) {
        const TModeInfo mi = tmode_of(S.mb[k]);
        float xk[TX], dx[TX], ex[2], u[TU];
        tstage(C, k, 0.f, xk, dx, ex, u);
        TRows R;
        trows(P, mi, C.h_min, C.h_max, xk, dx, ex, u, R);
        float* lam = S.lam + 4 + TR * k;
        float y[TR];
        bool act[TR];
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            const bool iq = tineq(r);
            float l = lam[r];
            if (update && R.on[r]) {
                const float t = l + beta_old * R.c[r];
                l = iq ? fmaxf(t, 0.f) : t;
                lam[r] = l;
            }
            const float t = l + beta * R.c[r];
            act[r] = R.on[r] && (!iq || t > 0.f);
            y[r] = act[r] ? (iq ? fmaxf(t, 0.f) : t) : 0.f;
            if (R.on[r]) {
                const float vr = iq ? fmaxf(R.c[r], 0.f) : fabsf(R.c[r]);
                viol = fmaxf(viol, vr);
                vph = fmaxf(vph, vr * R.phys[r]);
                if (iq) comp = fmaxf(comp, fabsf(y[r] * R.c[r]));
                if (!isfinite(R.c[r])) finite = false;
            }
        }
        jc += P.w_control * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        // local AL gradient over (x_k, u_k, x_{k+1})
        const float R2 = 2.f * P.w_control;
        float gx[TX] = {0.f, 0.f, 0.f, 0.f, 0.f}, gu[TU], gy[TX];
#pragma unroll
        for (int j = 0; j < 3; ++j) gu[j] = R2 * u[j];
        gu[3] = 0.f;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int j = 0; j < 4; ++j) gx[j] += y[r] * R.ax[r][j];
#pragma unroll
            for (int j = 0; j < TU; ++j) gu[j] += y[r] * R.au[r][j];
            gy[r] = y[r] * R.ay[r];
        }
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
            for (int j = 0; j < 3; ++j) gu[j] += y[4 + q] * R.lu[q][j];
        gx[3] += y[9] - y[10];
        {
            const float w11 = y[11] * kInvSqrt3;
            gu[3] += -w11 - y[12] + y[13];
            gx[4] -= w11;
            gy[4] = w11;
        }
#pragma unroll
        for (int i = 0; i < TX; ++i) {
            S.gr[TW * k + i] = gx[i];
            S.dz[TW * (k + 1) + i] = gy[i];
        }
#pragma unroll
        for (int j = 0; j < TU; ++j) S.gr[TW * k + TX + j] = gu[j];

        // augmented local matrix over (u 0..3, y 4..8, x 9..13, rhs 14)
        float A[TMTRI];
#pragma unroll
        for (int t = 0; t < TMTRI; ++t) A[t] = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) A[ttri(LU + j, LU + j)] += R2 + rho;
        A[ttri(LU + 3, LU + 3)] += rho;
#pragma unroll
        for (int i = 0; i < TX; ++i) A[ttri(LY + i, LY + i)] += rho;
        // beta a a^T of the dynamics rows on their nonzero pattern
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float vv[TLOC];
#pragma unroll
            for (int j = 0; j < TU; ++j) vv[LU + j] = R.au[r][j];
#pragma unroll
            for (int i = 0; i < TX; ++i) vv[LY + i] = (i == r) ? R.ay[r] : 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) vv[LX + i] = R.ax[r][i];
            vv[LX + 4] = 0.f;
            const float bw = act[r] ? beta : 0.f;
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                const int i = tdyn_nz(r, a);
                if (i < 0) continue;
                const float t = bw * vv[i];
#pragma unroll
                for (int b = 0; b <= a; ++b) A[ttri(i, tdyn_nz(r, b))] += t * vv[tdyn_nz(r, b)];
            }
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const float bw = act[4 + q] ? beta : 0.f;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j <= i; ++j) A[ttri(i, j)] += bw * R.lu[q][i] * R.lu[q][j];
        }
        A[ttri(LX + 3, LX + 3)] += (act[9] ? beta : 0.f) + (act[10] ? beta : 0.f);
        {
            // elapsed-time row over (h, tau_{k+1}, tau_k) = (-1, 1, -1) / sqrt(3)
            const float b3 = act[11] ? beta * (1.f / 3.f) : 0.f;
            A[ttri(LU + 3, LU + 3)] += b3;
            A[ttri(LY + 4, LU + 3)] -= b3;
            A[ttri(LY + 4, LY + 4)] += b3;
            A[ttri(LX + 4, LU + 3)] += b3;
            A[ttri(LX + 4, LY + 4)] -= b3;
            A[ttri(LX + 4, LX + 4)] += b3;
            A[ttri(LU + 3, LU + 3)] += (act[12] ? beta : 0.f) + (act[13] ? beta : 0.f);
        }
        if (curvature) {
            // Lagrangian curvature of the dynamics rows: -h sum_i yd_i d^2 f_i
            // over (x_k, u_k) and the cross terms -sum_i yd_i df_i/dv between
            // h and v (f is bilinear in h); yd_i = y_i / sigma_i
            float nx, ny;
            tface_nt(mi.face, nx, ny);
            const float tx = -ny, ty = nx, kk = R.kf, h = u[3];
            const float yd0 = y[0] * P.inv_sigma[0], yd1 = y[1] * P.inv_sigma[1];
            const float yd2 = y[2] * P.inv_sigma[2], yd3 = y[3] * P.inv_sigma[3];
            const float h_thth = -yd0 * R.f0 - yd1 * R.f1;
            const float h_thfn = yd0 * kk * (-R.st * nx - R.ct * ny) + yd1 * kk * (R.ct * nx - R.st * ny);
            const float h_thft = yd0 * kk * (-R.st * tx - R.ct * ty) + yd1 * kk * (R.ct * tx - R.st * ty);
            const float h_sfn = -yd2 * kk * P.inv_c2;
            A[ttri(LX + 2, LX + 2)] -= h * h_thth;
            A[ttri(LX + 2, LU + 0)] -= h * h_thfn;
            A[ttri(LX + 2, LU + 1)] -= h * h_thft;
            A[ttri(LX + 3, LU + 0)] -= h * h_sfn;
            A[ttri(LX + 2, LU + 3)] -= yd0 * R.fx02 + yd1 * R.fx12;
            A[ttri(LX + 3, LU + 3)] -= yd2 * R.fx23;
            A[ttri(LU + 3, LU + 0)] -= yd0 * R.fu00 + yd1 * R.fu10 + yd2 * R.fu20;
            A[ttri(LU + 3, LU + 1)] -= yd0 * R.fu01 + yd1 * R.fu11 + yd2 * R.fu21;
            A[ttri(LU + 3, LU + 2)] -= yd3;
        }
        // right-hand side row: the gradient
#pragma unroll
        for (int j = 0; j < TU; ++j) A[ttri(LR, LU + j)] = gu[j];
#pragma unroll
        for (int i = 0; i < TX; ++i) A[ttri(LR, LY + i)] = gy[i];
#pragma unroll
        for (int i = 0; i < TX; ++i) A[ttri(LR, LX + i)] = gx[i];
        // eliminate the u block (4 Cholesky steps, 1 / l_jj kept on the diagonal)
        bool pd = true;
#pragma unroll
        for (int j = 0; j < TU; ++j) {
            const float d = A[ttri(j, j)];
            pd = pd && (d > 0.f);
            const float il = rsqrtf(fmaxf(d, 1e-30f));
            A[ttri(j, j)] = il;
#pragma unroll
            for (int i = j + 1; i < TM; ++i) A[ttri(i, j)] *= il;
#pragma unroll
            for (int c = j + 1; c < TM; ++c)
#pragma unroll
                for (int i = c; i < TM; ++i) A[ttri(i, c)] -= A[ttri(i, j)] * A[ttri(c, j)];
        }
        float rec[kTRec];
#pragma unroll
        for (int t = 0; t < kTRec; ++t) rec[t] = 0.f;
#pragma unroll
        for (int i = 0; i < TU; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) rec[R_UF + ttri(i, j)] = A[ttri(i, j)];
#pragma unroll
        for (int c = 0; c < TM - TU; ++c)
#pragma unroll
            for (int j = 0; j < TU; ++j) rec[R_CP + 4 * c + j] = A[ttri(TU + c, j)];
        rec[R_PD] = pd ? 1.f : -1.f;
#pragma unroll
        for (int i = 0; i < TM - TU; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j)
                if (!(i == TM - TU - 1 && j == i)) rec[R_RED + ttri(i, j)] = A[ttri(TU + i, TU + j)];
#pragma unroll
        for (int q = 0; q < kTRec / 4; ++q)
            trec_st(C, q, k, make_float4(rec[4 * q], rec[4 * q + 1], rec[4 * q + 2], rec[4 * q + 3]));
    }
    __syncwarp();
    // initial rows (pose and tau_0 = 0) and the terminal row tau_N <= T
    if (lane < 4) {
        float l = S.lam[lane];
        const float c = tinit_row(C, lane, 0.f);
        if (update) {
            l = l + beta_old * c;
            S.lam[lane] = l;
        }
        viol = fmaxf(viol, fabsf(c));
        vph = fmaxf(vph, fabsf(c));
        if (!isfinite(c)) finite = false;
    }
    const int it = 4 + TR * N;
    if (lane == 4) {
        float l = S.lam[it];
        const float c = tterm_row(C, 0.f);
        if (update) {
            l = fmaxf(l + beta_old * c, 0.f);
            S.lam[it] = l;
        }
        const float y = fmaxf(l + beta * c, 0.f);
        viol = fmaxf(viol, fmaxf(c, 0.f));
        vph = fmaxf(vph, fmaxf(c, 0.f));
        comp = fmaxf(comp, fabsf(y * c));
        if (!isfinite(c)) finite = false;
    }
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float e = (S.xh[i * Np1 + N] - P.goal[i]) + S.xl[i * Np1 + N];
            jc += P.w_terminal * e * e;
        }
    __syncwarp();
    float stat = 0.f;
    for (int k = lane; k <= N; k += 32) {
#pragma unroll
        for (int i = 0; i < TX; ++i) {
            float g = (k < N) ? S.gr[TW * k + i] : 0.f;
            if (k > 0) g += S.dz[TW * k + i];
            if (k == N && i < 3) g += 2.f * P.w_terminal * ((S.xh[i * Np1 + N] - P.goal[i]) + S.xl[i * Np1 + N]);
            if (k == N && i == 4) g += fmaxf(S.lam[it] + beta * tterm_row(C, 0.f), 0.f);
            if (k == 0 && i != 3) {
                const int r = i < 3 ? i : 3;
                g += S.lam[r] + beta * tinit_row(C, r, 0.f);
            }
            S.gr[TW * k + i] = g;
            stat = fmaxf(stat, fabsf(g));
            if (!isfinite(g)) finite = false;
        }
        if (k < N)
#pragma unroll
            for (int j = 0; j < TU; ++j) {
                const float g = S.gr[TW * k + TX + j];
                stat = fmaxf(stat, fabsf(g));
                if (!isfinite(g)) finite = false;
            }
    }
    __syncwarp();
    TMeasures m;
    m.viol = twarp_max(viol);
    m.stat = twarp_max(stat);
    m.comp = twarp_max(comp);
    m.vphys = twarp_max(vph);
    m.cost = twarp_sum(jc);
    m.finite = __all_sync(kFullT, finite);
    return m;
}

// Phase B: the step's state part by a lane-parallel elimination of the
// block-tridiagonal system over dx_0 .. dx_N (Sec. III-C "Fixed-workspace
// local solves"), the order the fixed-step evaluator uses, here with 5 x 5
// blocks.  After phase A each stage record holds a quadratic element in
// (dx_{k+1}, dx_k): the reduced lower triangle over (y = x_{k+1}, x = x_k,
// rhs).  Lane l folds the elements of its stages [k0, k1) into one over
// (x_{k1}, x_{k0}); a tree over the lanes (the partner's element by
// shuffles) eliminates the nodes between the spans until lane 0 holds an
// element over (x_N, x_0) and solves that 10 x 10 system; the node steps
// follow by back-substitution down the tree and through each lane's span.
// Eliminating node m between E over (m, a) and F over (b, m):
// S = E_mm + F_mm = L L^T, Y = L^{-1} [F_mb | E_ma | r_m], the element over
// (b, a) is blockdiag(F_bb, E_aa) - Y^T Y, and later
// dx_m = -L^{-T} (Y_b dx_b + Y_a dx_a + y_r).  The same block Cholesky as
// the backward sweep, in another order: the matrix is positive definite
// exactly when every pivot is positive, in any order, so a non-positive
// pivot (or a u-block pivot flagged by phase A) reports failure.  Writes
// dx_k to dz[9k .. 9k+4], k = 0..N.

constexpr int kTElem = 65;  // 11 x 11 lower triangle without the (rhs, rhs) entry
constexpr int kTElemChunk0 = R_RED / 4;  // 14: element and node floats start here

// record floats 56..120 of stage k as an element, with the boundary terms:
// the terminal cost and the active terminal row on the last stage's y
// block, damping and the four initial rows on the first stage's x block
__device__ __forceinline__ void tload_elem(const TCtx& C, int k, float e[kTElem], float beta, float rho) {
    float v[68];
#pragma unroll
    for (int q = 0; q < 17; ++q) {
        const float4 t = *trec(C, kTElemChunk0 + q, k);
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
#pragma unroll
    for (int t = 0; t < kTElem; ++t) e[t] = v[t];
    const DevInstance& P = *C.P;
    const int N = C.N, Np1 = N + 1;
    const TSmem& S = C.sm;
    if (k == N - 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            e[ttri(i, i)] += 2.f * P.w_terminal;
            e[ttri(10, i)] += 2.f * P.w_terminal * ((S.xh[i * Np1 + N] - P.goal[i]) + S.xl[i * Np1 + N]);
        }
        const float t = S.lam[4 + TR * N] + beta * tterm_row(C, 0.f);  // tau_N - T <= 0 while active
        if (t > 0.f) {
            e[ttri(4, 4)] += beta;
            e[ttri(10, 4)] += t;
        }
    }
    if (k == 0) {
#pragma unroll
        for (int i = 0; i < TX; ++i) e[ttri(5 + i, 5 + i)] += rho;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int q = tinit_comp(i);
            e[ttri(5 + q, 5 + q)] += beta;
            e[ttri(10, 5 + q)] += S.lam[i] + beta * tinit_row(C, i, 0.f);
        }
    }
}

// Eliminate the node shared by e (over (y = m, x = a)) and f (over (y = b,
// x = m)); e becomes the element over (y = b, x = a).  Stores node m's
// (L, Y) in record `km` when `store`; false on a non-positive pivot.
__device__ __forceinline__ bool tcombine(const TCtx& C, float e[kTElem], const float f[kTElem], int km, bool store) {
    float L[15];
#pragma unroll
    for (int i = 0; i < TX; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) L[ttri(i, j)] = e[ttri(i, j)] + f[ttri(TX + i, TX + j)];
    bool pd = true;
#pragma unroll
    for (int j = 0; j < TX; ++j) {
        float d = L[ttri(j, j)];
#pragma unroll
        for (int q = 0; q < j; ++q) d -= L[ttri(j, q)] * L[ttri(j, q)];
        pd = pd && d > 0.f;
        const float il = rsqrtf(fmaxf(d, 1e-30f));
        L[ttri(j, j)] = il;
#pragma unroll
        for (int i = j + 1; i < TX; ++i) {
            float s = L[ttri(i, j)];
#pragma unroll
            for (int q = 0; q < j; ++q) s -= L[ttri(i, q)] * L[ttri(j, q)];
            L[ttri(i, j)] = s * il;
        }
    }
    // Y = L^{-1} [F_mb | E_ma | r_m]: columns b 0..4, a 0..4, rhs
    float Y[TX][11];
#pragma unroll
    for (int c = 0; c < 11; ++c)
#pragma unroll
        for (int i = 0; i < TX; ++i) {
            float s = (c < TX) ? f[ttri(TX + i, c)]
                               : (c < 2 * TX) ? e[ttri(TX + (c - TX), i)] : e[ttri(10, i)] + f[ttri(10, TX + i)];
#pragma unroll
            for (int q = 0; q < i; ++q) s -= L[ttri(i, q)] * Y[q][c];
            Y[i][c] = s * L[ttri(i, i)];
        }
    // the element over (y = b, x = a, rhs): blockdiag(F_bb, E_aa) - Y^T Y
    float g[kTElem];
#pragma unroll
    for (int i = 0; i < 11; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            if (i == 10 && j == 10) continue;
            float s;
            if (i < TX)
                s = f[ttri(i, j)];                                   // (b, b)
            else if (i < 2 * TX)
                s = (j < TX) ? 0.f : e[ttri(i, j)];                  // (a, b) fill-in, (a, a)
            else
                s = (j < TX) ? f[ttri(10, j)] : e[ttri(10, j)];      // (rhs, b), (rhs, a)
#pragma unroll
            for (int p = 0; p < TX; ++p) s -= Y[p][i] * Y[p][j];
            g[ttri(i, j)] = s;
        }
#pragma unroll
    for (int t = 0; t < kTElem; ++t) e[t] = g[t];
    if (store) {
        float o[72];
#pragma unroll
        for (int t = 0; t < 15; ++t) o[t] = L[t];
#pragma unroll
        for (int i = 0; i < TX; ++i)
#pragma unroll
            for (int c = 0; c < 11; ++c) o[15 + 11 * i + c] = Y[i][c];
        o[70] = o[71] = 0.f;
#pragma unroll
        for (int q = 0; q < 18; ++q)
            trec_st(C, kTElemChunk0 + q, km, make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]));
    }
    return pd;
}

// dx_m = -L^{-T} (Y_b dx_b + Y_a dx_a + y_r) from node m's stored (L, Y)
__device__ __forceinline__ void tback_node(const TCtx& C, int km, const float xa[TX], const float xb[TX],
                                           float xm[TX]) {
    float v[72];
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        const float4 t = *trec(C, kTElemChunk0 + q, km);
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
    const float* L = v;
    const float* Y = v + 15;  // [5][11]
    float t[TX];
#pragma unroll
    for (int i = 0; i < TX; ++i) {
        float s = Y[11 * i + 10];
#pragma unroll
        for (int j = 0; j < TX; ++j) s += Y[11 * i + j] * xb[j] + Y[11 * i + TX + j] * xa[j];
        t[i] = s;
    }
#pragma unroll
    for (int i = TX - 1; i >= 0; --i) {
        float s = -t[i];
#pragma unroll
        for (int q = i + 1; q < TX; ++q) s -= L[ttri(q, i)] * xm[q];
        xm[i] = s * L[ttri(i, i)];
    }
}

__device__ bool tphase_b(TCtx& C, float beta, float rho) {
    const int N = C.N, lane = C.lane;
    TSmem& S = C.sm;
    const int per = (N + 31) >> 5;
    const int nl = (N + per - 1) / per;  // lanes that own stages
    const int k0 = min(N, lane * per), k1 = min(N, k0 + per);
    const bool own = lane < nl;
    const int nlev = nl > 1 ? 32 - __clz(nl - 1) : 0;  // tree levels, ceil(log2 nl)
    const int nsteps = (per - 1) + nlev;
    bool pd = true;
    float e[kTElem];
#pragma unroll
    for (int t = 0; t < kTElem; ++t) e[t] = 0.f;
    if (own) {
        pd = reinterpret_cast<const float*>(trec(C, R_PD / 4, k0))[R_PD % 4] > 0.f;
        tload_elem(C, k0, e, beta, rho);
    }
    // folds of the lane's next stages, then the tree levels d = 1, 2, 4, ...:
    // lane l (a multiple of 2d) eliminates the first node of lane l + d's span
#pragma unroll 1
    for (int st = 0; st < nsteps; ++st) {
        float f[kTElem];
        bool act;
        int km;
        if (st < per - 1) {  // warp-uniform
            km = k0 + 1 + st;
            act = own && km < k1;
            if (act) {
                pd = pd && reinterpret_cast<const float*>(trec(C, R_PD / 4, km))[R_PD % 4] > 0.f;
                tload_elem(C, km, f, beta, rho);
            }
        } else {
            const int d = 1 << (st - (per - 1));
#pragma unroll
            for (int t = 0; t < kTElem; ++t) f[t] = __shfl_down_sync(kFullT, e[t], d);
            act = (lane & (2 * d - 1)) == 0 && lane + d < nl;
            km = (lane + d) * per;
        }
        if (act) pd = tcombine(C, e, f, km, true) && pd;
    }
    // lane 0 solves the root element over (x_N, x_0): a 10 x 10 Cholesky
    float xl[TX], xr[TX];
#pragma unroll
    for (int i = 0; i < TX; ++i) xl[i] = xr[i] = 0.f;
    if (lane == 0) {
        float A[55];
#pragma unroll
        for (int t = 0; t < 55; ++t) A[t] = e[t];
#pragma unroll
        for (int j = 0; j < 2 * TX; ++j) {
            float dd = A[ttri(j, j)];
#pragma unroll
            for (int q = 0; q < j; ++q) dd -= A[ttri(j, q)] * A[ttri(j, q)];
            pd = pd && dd > 0.f;
            const float il = rsqrtf(fmaxf(dd, 1e-30f));
            A[ttri(j, j)] = il;
#pragma unroll
            for (int i = j + 1; i < 2 * TX; ++i) {
                float s = A[ttri(i, j)];
#pragma unroll
                for (int q = 0; q < j; ++q) s -= A[ttri(i, q)] * A[ttri(j, q)];
                A[ttri(i, j)] = s * il;
            }
        }
        float yv[2 * TX], x[2 * TX];
#pragma unroll
        for (int i = 0; i < 2 * TX; ++i) {
            float s = e[ttri(10, i)];
#pragma unroll
            for (int q = 0; q < i; ++q) s -= A[ttri(i, q)] * yv[q];
            yv[i] = s * A[ttri(i, i)];
        }
#pragma unroll
        for (int i = 2 * TX - 1; i >= 0; --i) {
            float s = yv[i];
#pragma unroll
            for (int q = i + 1; q < 2 * TX; ++q) s -= A[ttri(q, i)] * x[q];
            x[i] = s * A[ttri(i, i)];
        }
#pragma unroll
        for (int i = 0; i < TX; ++i) {
            xr[i] = -x[i];       // dx_N
            xl[i] = -x[TX + i];  // dx_0
        }
    }
    // back-substitution: the tree levels top-down (lane l hands lane l + d
    // the node it eliminated and its own right end), then each lane's span
    // right to left
    float xc[TX];  // dx of the node right of the current interior node
#pragma unroll 1
    for (int st = nsteps - 1; st >= 0; --st) {
        const bool tree = st >= per - 1;  // warp-uniform
        const int d = tree ? 1 << (st - (per - 1)) : 0;
        if (st == per - 2)
#pragma unroll
            for (int i = 0; i < TX; ++i) xc[i] = xr[i];
        const bool act = tree ? ((lane & (2 * d - 1)) == 0 && lane + d < nl) : (own && k0 + 1 + st < k1);
        const int km = tree ? (lane + d) * per : k0 + 1 + st;
        float xm[TX];
#pragma unroll
        for (int i = 0; i < TX; ++i) xm[i] = 0.f;
        if (act) tback_node(C, km, xl, tree ? xr : xc, xm);
        if (tree) {
#pragma unroll
            for (int i = 0; i < TX; ++i) {
                const float pm = __shfl_up_sync(kFullT, xm[i], d), pr = __shfl_up_sync(kFullT, xr[i], d);
                if ((lane & (2 * d - 1)) == d && lane < nl) {
                    xl[i] = pm;
                    xr[i] = pr;
                }
                if (act) xr[i] = xm[i];
            }
        } else if (act) {
#pragma unroll
            for (int i = 0; i < TX; ++i) {
                S.dz[TW * km + i] = xm[i];
                xc[i] = xm[i];
            }
        }
    }
    if (own) {
#pragma unroll
        for (int i = 0; i < TX; ++i) S.dz[TW * k0 + i] = xl[i];
        if (lane == nl - 1)
#pragma unroll
            for (int i = 0; i < TX; ++i) S.dz[TW * N + i] = xr[i];
    }
    __syncwarp();
    return __all_sync(kFullT, pd);
}

// Phase C: the control steps, stage-parallel from the u-block factors of
// phase A and the state steps of phase B,
//   du_k = -L_u^{-T} (coupling^T [dx_{k+1}; dx_k; 1]).
// Returns D = grad . dz.
__device__ float tphase_c(TCtx& C) {
    const int N = C.N, lane = C.lane;
    TSmem& S = C.sm;
#pragma unroll 1
    for (int k = lane; k < N; k += 32) {
        float f[56];
#pragma unroll
        for (int qq = 0; qq < 14; ++qq) {
            const float4 t = *trec(C, qq, k);
            f[4 * qq] = t.x;
            f[4 * qq + 1] = t.y;
            f[4 * qq + 2] = t.z;
            f[4 * qq + 3] = t.w;
        }
        float xa[TX], xb[TX];
#pragma unroll
        for (int i = 0; i < TX; ++i) {
            xa[i] = S.dz[TW * k + i];
            xb[i] = S.dz[TW * (k + 1) + i];
        }
        float R[TU];
#pragma unroll
        for (int j = 0; j < TU; ++j) {
            float s = f[R_CP + 4 * 10 + j];
#pragma unroll
            for (int i = 0; i < TX; ++i) s += f[R_CP + 4 * i + j] * xb[i] + f[R_CP + 4 * (TX + i) + j] * xa[i];
            R[j] = s;
        }
        float du[TU];
#pragma unroll
        for (int i = TU - 1; i >= 0; --i) {
            float s = -R[i];
#pragma unroll
            for (int qq = i + 1; qq < TU; ++qq) s -= f[R_UF + ttri(qq, i)] * du[qq];
            du[i] = s * f[R_UF + ttri(i, i)];
        }
#pragma unroll
        for (int j = 0; j < TU; ++j) S.dz[TW * k + TX + j] = du[j];
    }
    __syncwarp();
    float D = 0.f;
    for (int t = lane; t < TW * N + TX; t += 32) D += S.gr[t] * S.dz[t];
    return twarp_sum(D);
}

// merit contribution of interval k at the trial step alpha
__device__ __forceinline__ float tstage_merit(const TCtx& C, int k, float alpha, float beta, float inv2b) {
    const DevInstance& P = *C.P;
    const int N = C.N, Np1 = N + 1;
    const TSmem& S = C.sm;
    const TModeInfo mi = tmode_of(S.mb[k]);
    float xk[TX], dx[TX], ex[2], u[TU];
    tstage(C, k, alpha, xk, dx, ex, u);
    TRows R;
    trows(P, mi, C.h_min, C.h_max, xk, dx, ex, u, R);
    const float* lam = S.lam + 4 + TR * k;
    float phi = P.w_control * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
    for (int r = 0; r < TR; ++r)
        if (R.on[r]) phi += trow_al(tineq(r), lam[r], beta, inv2b, R.c[r]);
    if (k == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i) phi += trow_al(false, S.lam[i], beta, inv2b, tinit_row(C, i, alpha));
    if (k == N - 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float e =
                (S.xh[i * Np1 + N] - P.goal[i]) + (S.xl[i * Np1 + N] + (alpha != 0.f ? alpha * S.dz[TW * N + i] : 0.f));
            phi += P.w_terminal * e * e;
        }
        phi += trow_al(true, S.lam[4 + TR * N], beta, inv2b, tterm_row(C, alpha));
    }
    return phi;
}

// Phase D: trial merits for alpha in {0, 1, 1/2, ..., 2^-(n_alpha-1)}, four
// at a time (lane = trial + 4 x stage group), stage merits summed as FP32
// pairs; the accepted alpha is the largest passing the Armijo test.
__device__ float tphase_d(const TCtx& C, float beta, float D, const SolverParams& sp) {
    const int lane = C.lane;
    const int sub = lane & 3, grp = lane >> 2;
    const float inv2b = 0.5f / beta;
    float phi0 = 0.f, phi0l = 0.f, slack = 0.f;
#pragma unroll 1
    for (int batch = 0; batch < 2; ++batch) {
        const int a = 4 * batch + sub;
        if (batch == 1 && sp.n_alpha < 4) break;
        const float alpha = (a == 0) ? 0.f : ldexpf(1.f, -(a - 1));
        float phi = 0.f, phil = 0.f;
        if (a <= sp.n_alpha)
#pragma unroll 1
            for (int k = grp; k < C.N; k += 8) {
                float e;
                two_sum_t(phi, tstage_merit(C, k, alpha, beta, inv2b), phi, e);
                phil += e;
            }
#pragma unroll
        for (int off = 4; off <= 16; off <<= 1) {
            const float oh = __shfl_xor_sync(kFullT, phi, off), ol = __shfl_xor_sync(kFullT, phil, off);
            float e;
            two_sum_t(phi, oh, phi, e);
            phil += ol + e;
        }
        if (batch == 0) {
            phi0 = __shfl_sync(kFullT, phi, 0);
            phi0l = __shfl_sync(kFullT, phil, 0);
            slack = sp.ls_slack * fabsf(phi0);
        }
        const float dphi = (phi - phi0) + (phil - phi0l);
        bool pass = (a >= 1) && (a <= sp.n_alpha) && (dphi <= sp.armijo_c1 * alpha * D);
        if (a == 1 && fabsf(D) <= slack && dphi <= slack) pass = true;
        const unsigned bal = __ballot_sync(kFullT, pass) & 0xfu;
        if (bal) return ldexpf(1.f, -(4 * batch + __ffs(bal) - 2));
    }
    return 0.f;
}

// Phase E: compensated update z += alpha dz
__device__ void tphase_e(TCtx& C, float alpha) {
    const int N = C.N, Np1 = N + 1, lane = C.lane;
    TSmem& S = C.sm;
#pragma unroll
    for (int i = 0; i < TX; ++i)
        for (int k = lane; k < Np1; k += 32) {
            const int t = i * Np1 + k;
            float s, e;
            two_sum_t(S.xh[t], S.xl[t] + alpha * S.dz[TW * k + i], s, e);
            S.xh[t] = s;
            S.xl[t] = e;
        }
#pragma unroll
    for (int j = 0; j < TU; ++j)
        for (int k = lane; k < N; k += 32) S.us[j * N + k] += alpha * S.dz[TW * k + TX + j];
    __syncwarp();
}

// FP64 rows of interval kk at the stored iterate: values, physical factors,
// presence and the Jacobian over (x_k 0..4, u_k 5..8, x_{k+1} 9..13).
struct TRows64 {
    double c[TR], ph[TR];
    bool on[TR];
    double J[TR][TLOC];
    double u[TU];
};

__device__ void trows64(const TCtx& C, int kk, TRows64& R) {
    const DevInstance& P = *C.P;
    const int N = C.N, Np1 = N + 1;
    const TSmem& S = C.sm;
    const TModeInfo mi = tmode_of(S.mb[kk]);
    double x0[TX], x1[TX];
    for (int i = 0; i < TX; ++i) {
        x0[i] = (double)S.xh[i * Np1 + kk] + (double)S.xl[i * Np1 + kk];
        x1[i] = (double)S.xh[i * Np1 + kk + 1] + (double)S.xl[i * Np1 + kk + 1];
    }
    for (int j = 0; j < TU; ++j) R.u[j] = (double)S.us[j * N + kk];
    const double nx = (mi.face == 0) ? 1.0 : ((mi.face == 2) ? -1.0 : 0.0);
    const double ny = (mi.face == 1) ? 1.0 : ((mi.face == 3) ? -1.0 : 0.0);
    const double tx = -ny, ty = nx;
    const double a = P.a_d[mi.face], ell = P.ell_d[mi.face];
    const double kp = (mi.kind == 3) ? 0.0 : P.kappa_d, ic2 = P.inv_c2_d;
    const double fn = R.u[0], ft = R.u[1], sd = R.u[2], h = R.u[3];
    double st, ct;
    sincos(x0[2], &st, &ct);
    const double vx = kp * (fn * nx + ft * tx), vy = kp * (fn * ny + ft * ty);
    const double f[4] = {ct * vx - st * vy, st * vx + ct * vy, kp * (-a * ft - x0[3] * fn) * ic2, sd};
    const double Fx02 = -st * vx - ct * vy, Fx12 = ct * vx - st * vy, Fx23 = -kp * fn * ic2;
    const double Fu[4][3] = {{kp * (ct * nx - st * ny), kp * (ct * tx - st * ty), 0.0},
                             {kp * (st * nx + ct * ny), kp * (st * tx + ct * ty), 0.0},
                             {-kp * x0[3] * ic2, -kp * a * ic2, 0.0},
                             {0.0, 0.0, 1.0}};
    const double mu = P.mu_d, sc = P.sc_cone_d;
    const bool stick = mi.kind == 0, free = mi.kind == 3;
    const double sg = (mi.kind == 1) ? -1.0 : 1.0;
    for (int r = 0; r < TR; ++r) {
        R.on[r] = true;
        R.ph[r] = 1.0;
        R.c[r] = 0.0;
        for (int j = 0; j < TLOC; ++j) R.J[r][j] = 0.0;
    }
    for (int r = 0; r < 4; ++r) {
        const double is = 1.0 / P.sigma_d[r];
        R.c[r] = (x1[r] - x0[r] - h * f[r]) * is;
        R.ph[r] = P.sigma_d[r];
        R.J[r][r] = -is;
        R.J[r][TW + r] = is;
        for (int j = 0; j < 3; ++j) R.J[r][TX + j] = -h * Fu[r][j] * is;
        R.J[r][TX + 3] = -f[r] * is;
    }
    R.J[0][2] += -h * Fx02 / P.sigma_d[0];
    R.J[1][2] += -h * Fx12 / P.sigma_d[1];
    R.J[2][3] += -h * Fx23 / P.sigma_d[2];
    if (mi.smask) R.on[3] = false;
    if (free) {
        R.c[4] = fn;
        R.J[4][TX + 0] = 1.0;
        for (int r = 5; r <= 10; ++r) R.on[r] = false;
    } else {
        if (stick) {
            R.c[4] = sd;
            R.J[4][TX + 2] = 1.0;
        } else {
            R.c[4] = sc * (ft + sg * mu * fn);
            R.J[4][TX + 0] = sc * sg * mu;
            R.J[4][TX + 1] = sc;
            R.ph[4] = 1.0 / sc;
        }
        R.c[5] = sc * (ft - mu * fn);
        R.J[5][TX + 0] = -sc * mu;
        R.J[5][TX + 1] = sc;
        R.c[6] = sc * (-ft - mu * fn);
        R.J[6][TX + 0] = -sc * mu;
        R.J[6][TX + 1] = -sc;
        R.ph[5] = R.ph[6] = 1.0 / sc;
        R.on[5] = R.on[6] = stick;
        R.c[7] = sg * sd;
        R.J[7][TX + 2] = sg;
        R.on[7] = !stick;
        R.c[8] = -fn;
        R.J[8][TX + 0] = -1.0;
        R.c[9] = x0[3] - ell;
        R.J[9][3] = 1.0;
        R.c[10] = -x0[3] - ell;
        R.J[10][3] = -1.0;
    }
    const double r3 = 1.0 / sqrt(3.0);
    R.c[11] = (x1[4] - x0[4] - h) * r3;
    R.J[11][4] = -r3;
    R.J[11][TX + 3] = -r3;
    R.J[11][TW + 4] = r3;
    R.ph[11] = sqrt(3.0);
    R.c[12] = (double)C.h_min - h;
    R.J[12][TX + 3] = -1.0;
    R.c[13] = h - (double)C.h_max;
    R.J[13][TX + 3] = 1.0;
    for (int r = 0; r < TR; ++r)
        if (!R.on[r]) {
            R.c[r] = 0.0;
            for (int j = 0; j < TLOC; ++j) R.J[r][j] = 0.0;
        }
}

struct TCert {
    double cost, viol, stat;
    bool finite;
};

// FP64 certificate: cost, physical violation and the KKT residual with the
// multiplier estimates at beta.
__device__ TCert tcertify(const TCtx& C, float beta_f) {
    const DevInstance& P = *C.P;
    const int N = C.N, Np1 = N + 1, lane = C.lane;
    const TSmem& S = C.sm;
    const double beta = beta_f;
    double cost = 0.0, viol = 0.0, stat = 0.0;
    bool finite = true;
    for (int k = lane; k <= N; k += 32) {
        double g[TW];
        for (int i = 0; i < TW; ++i) g[i] = 0.0;
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
            const int kk = (side == 0) ? k - 1 : k;
            if (kk < 0 || kk >= N) continue;
            TRows64 R;
            trows64(C, kk, R);
            const float* lam = S.lam + 4 + TR * kk;
            for (int r = 0; r < TR; ++r) {
                if (!R.on[r]) continue;
                const bool iq = tineq(r);
                const double t = (double)lam[r] + beta * R.c[r];
                const double y = iq ? fmax(t, 0.0) : t;
                if (side == 1) {
                    const double vr = iq ? fmax(R.c[r], 0.0) : fabs(R.c[r]);
                    viol = fmax(viol, vr * R.ph[r]);
                    if (!isfinite(R.c[r])) finite = false;
                }
                if (side == 0)
                    for (int i = 0; i < TX; ++i) g[i] += y * R.J[r][TW + i];
                else
                    for (int i = 0; i < TW; ++i) g[i] += y * R.J[r][i];
            }
            if (side == 1)
                for (int j = 0; j < 3; ++j) {
                    g[TX + j] += 2.0 * P.w_control_d * R.u[j];
                    cost += P.w_control_d * R.u[j] * R.u[j];
                }
        }
        if (k == N) {
            for (int i = 0; i < 3; ++i) {
                const double e = (double)S.xh[i * Np1 + N] + (double)S.xl[i * Np1 + N] - P.goal_d[i];
                g[i] += 2.0 * P.w_terminal_d * e;
                cost += P.w_terminal_d * e * e;
            }
            const double c = (double)S.xh[4 * Np1 + N] + (double)S.xl[4 * Np1 + N] - (double)C.T;
            g[4] += fmax((double)S.lam[4 + TR * N] + beta * c, 0.0);
            viol = fmax(viol, fmax(c, 0.0));
        }
        if (k == 0)
            for (int i = 0; i < 4; ++i) {
                const int q = tinit_comp(i);
                const double c = (double)S.xh[q * Np1] + (double)S.xl[q * Np1] - (i < 3 ? P.start_d[i] : 0.0);
                g[q] += (double)S.lam[i] + beta * c;
                viol = fmax(viol, fabs(c));
            }
        const int nv = (k < N) ? TW : TX;
        for (int i = 0; i < nv; ++i) {
            stat = fmax(stat, fabs(g[i]));
            if (!isfinite(g[i])) finite = false;
        }
    }
    TCert ct;
    ct.cost = twarp_sum_d(cost);
    ct.viol = twarp_max_d(viol);
    ct.stat = twarp_max_d(stat);
    ct.finite = __all_sync(kFullT, finite) && isfinite(ct.cost);
    return ct;
}

__global__ void __launch_bounds__(128, 3) timing_kernel(const TimingArgs A) {
    extern __shared__ float tsmem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int warp_global = blockIdx.x * (blockDim.x >> 5) + wib;
    const EvalArgs& E = A.e;
    const size_t per_warp = tsmem_floats(E.Nmax);
    TCtx C;
    C.lane = lane;
    C.Nmax = E.Nmax;
    C.h_min = A.h_min;
    C.h_max = A.h_max;
    C.T = A.T;
    C.sm = tcarve(tsmem_raw + per_warp * wib, E.Nmax);
    C.rec = E.ws + (size_t)warp_global * E.ws_per_warp;
    const SolverParams& sp = E.sp;
    const int64_t n_tos = E.d_n ? min(*E.d_n, E.n) : E.n;
    for (;;) {
        unsigned int t = 0;
        if (lane == 0) t = atomicAdd(E.queue, 1u);
        t = __shfl_sync(kFullT, t, 0);
        if ((int64_t)t >= n_tos) break;
        const int64_t ti = (int64_t)t;
        const comet_mode_seq sq = E.seqs[ti];
        bool bad = sq.instance < 0 || sq.instance >= E.n_inst;
        const DevInstance* P = bad ? E.inst : E.inst + sq.instance;
        const int len = sq.len;
        bad = bad || len < 1 || len > P->Lmax || len > COMET_MAX_SEGMENTS || P->K * len > E.Nmax;
        if (!bad)
            for (int i = 0; i < len; ++i) bad = bad || sq.modes[i] >= P->n_modes;
        if (bad) {
            if (lane == 0) {
                atomicExch(E.bad_input, 1);
                E.out_status[ti] = COMET_TO_NONFINITE;
                E.out_cost[ti] = __int_as_float(0x7fc00000);
                if (E.out_iters) E.out_iters[ti] = 0;
                if (E.out_viol) E.out_viol[ti] = __int_as_float(0x7fc00000);
                if (E.out_merit) E.out_merit[ti] = __int_as_float(0x7fc00000);
                if (E.out_stat) E.out_stat[ti] = __int_as_float(0x7fc00000);
            }
            continue;
        }
        C.P = P;
        C.N = P->K * len;
        const int N = C.N, Np1 = N + 1;
        TSmem& S = C.sm;
        // initial iterate: warm start, or the fixed-step cold start with
        // h_k = dt clipped into the bounds and tau_k = k h_0
        const float* warm = E.warm ? E.warm + ti * E.stride : nullptr;
        const int Nm1 = E.Nmax + 1;
        const float h0 = fminf(fmaxf(P->dt, C.h_min), C.h_max);
        for (int qq = lane; qq < TX * Np1; qq += 32) {
            const int i = qq / Np1, k = qq - i * Np1;
            float x;
            if (warm) {
                x = warm[i * Nm1 + k];
            } else if (i < 3) {
                const float al = (float)k / (float)N;
                x = (1.f - al) * P->start[i] + al * P->goal[i];
            } else {
                x = (i == 4) ? (float)k * h0 : 0.f;
            }
            S.xh[qq] = x;
            S.xl[qq] = 0.f;
        }
        for (int qq = lane; qq < TU * N; qq += 32) {
            const int j = qq / N, k = qq - j * N;
            S.us[qq] = warm ? warm[TX * Nm1 + j * E.Nmax + k] : ((j == 3) ? h0 : 0.f);
        }
        for (int qq = lane; qq < 5 + TR * N; qq += 32) S.lam[qq] = 0.f;
        for (int k = lane; k < N; k += 32) {
            const int seg = (int)(((long long)k * len) / N);
            const int m = sq.modes[seg];
            const bool free = m == kModeFreeT;
            const int face = free ? 0 : m / 3, kind = free ? 3 : m - 3 * (m / 3);
            bool smask = free;
            if (!free && k + 1 < N) {
                const int m1 = sq.modes[(int)(((long long)(k + 1) * len) / N)];
                smask = m1 == kModeFreeT || (m1 / 3) != face;
            }
            S.mb[k] = (unsigned char)(face | (kind << 2) | ((smask ? 1 : 0) << 4));
        }
        __syncwarp();
        float beta = sp.beta0, rho = sp.rho0, eta = INFINITY;
        int inner = 0, it = 0, status = COMET_TO_MAX_ITER, curv_hold = 0;
        bool nonfinite = false;
        for (it = 0; it < sp.max_iters; ++it) {
            const bool curv = curv_hold == 0;
            if (!curv) --curv_hold;
            // one call site per phase: MEASURE, UPDATE (dual update, then the
            // model at the new multipliers), RETRY (Gauss-Newton or more damping)
            enum { kMeasure, kUpdate, kRetry };
            int trip = kMeasure, retries = 0;
            bool model_curv = curv, fac = false, done = false;
            float beta_old = beta;
            for (;;) {
                const TMeasures m = tphase_a(C, beta, rho, model_curv, trip == kUpdate, beta_old);
                if (trip == kMeasure) {
                    if (!m.finite) {
                        status = COMET_TO_NONFINITE;
                        nonfinite = true;
                        done = true;
                        break;
                    }
                    // stop test of Sec. III-C, as in the fixed-step evaluator
                    const float eps_d = sp.eps_dual * fmaxf(1.f, beta / sp.beta_ref) * fmaxf(1.f, fabsf(m.cost));
                    if (m.viol <= sp.eps_primal && m.vphys <= 0.5f * (float)sp.eps_feas && m.stat <= eps_d &&
                        m.comp <= sp.eps_comp) {
                        status = COMET_TO_CONVERGED;
                        done = true;
                        break;
                    }
                    const float omega = fmaxf(eps_d, sp.omega_ratio * m.viol);
                    const bool solved = m.stat <= omega;
                    if (solved || inner >= sp.max_inner) {
                        beta_old = beta;
                        if (solved && m.viol > sp.eps_primal && m.viol > sp.eta_ratio * eta)
                            beta = fminf(sp.beta_max, beta * sp.beta_growth);
                        eta = m.viol;
                        inner = 0;
                        trip = kUpdate;
                        continue;
                    }
                }
                fac = tphase_b(C, beta, rho);
                if (fac) break;
                if (model_curv) {
                    curv_hold = sp.curv_skip;
                    model_curv = false;
                } else {
                    if (retries >= sp.max_retries) break;
                    ++retries;
                    rho = fminf(sp.rho_max, rho * 10.f);
                }
                trip = kRetry;
            }
            if (done) break;
            ++inner;
            if (!fac) continue;
            const float D = tphase_c(C);
            const float alpha = tphase_d(C, beta, D, sp);
            if (alpha > 0.f) {
                tphase_e(C, alpha);
                rho = fmaxf(sp.rho_min, rho / 10.f);
            } else {
                rho = fminf(sp.rho_max, rho * 10.f);
            }
        }
        const TCert ct = tcertify(C, beta);
        if (!ct.finite) nonfinite = true;
        if (nonfinite) status = COMET_TO_NONFINITE;
        if (status == COMET_TO_CONVERGED && !(ct.viol <= sp.eps_feas)) status = COMET_TO_INFEASIBLE;
        if (lane == 0) {
            E.out_status[ti] = status;
            E.out_cost[ti] = (float)ct.cost;
            if (E.out_viol) E.out_viol[ti] = (float)ct.viol;
            if (E.out_merit) E.out_merit[ti] = (float)(ct.cost + sp.merit_mu * fmax(ct.viol - sp.eps_feas, 0.0));
            if (E.out_iters) E.out_iters[ti] = it;
            if (E.out_stat) E.out_stat[ti] = (float)ct.stat;
        }
        if (E.out_traj) {
            float* out = E.out_traj + ti * E.stride;
            for (int qq = lane; qq < TX * Nm1; qq += 32) {
                const int i = qq / Nm1, k = qq - i * Nm1;
                out[qq] = (k <= N) ? S.xh[i * Np1 + k] + S.xl[i * Np1 + k] : 0.f;
            }
            for (int qq = lane; qq < TU * E.Nmax; qq += 32) {
                const int j = qq / E.Nmax, k = qq - j * E.Nmax;
                out[TX * Nm1 + qq] = (k < N) ? S.us[j * N + k] : 0.f;
            }
        }
        __syncwarp();
    }
}

}  // namespace

size_t timing_smem_per_warp_bytes(int Nmax) { return tsmem_floats(Nmax) * sizeof(float); }

int64_t timing_ws_per_warp_floats(int Nmax) { return (int64_t)kTRec * Nmax; }

int timing_blocks_per_sm(int warps_per_block, int Nmax) {
    const size_t smem = timing_smem_per_warp_bytes(Nmax) * warps_per_block;
    if (cudaFuncSetAttribute(timing_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, timing_kernel, warps_per_block * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_timing(const TimingArgs& a, int total_warps, int warps_per_block, cudaStream_t s) {
    const size_t smem = timing_smem_per_warp_bytes(a.e.Nmax) * warps_per_block;
    cudaError_t e = cudaFuncSetAttribute(timing_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int blocks = (total_warps + warps_per_block - 1) / warps_per_block;
    timing_kernel<<<blocks, warps_per_block * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace comet
