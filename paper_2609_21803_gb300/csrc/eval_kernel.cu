// eval_kernel.cu -- persistent warp-per-TO evaluator of mode-conditioned
// trajectory optimisations (CoMET, Sec. III-C), FP32 with compensated state
// storage and an FP64 certificate.
//
// One warp owns one TO at a time and pulls the next TO index from a device
// counter when it finishes (the resident pool of Sec. III-C, "Reusable pool
// with independent stopping", kept on the device: no host round trip).  One
// iteration of the augmented-Lagrangian Newton / Gauss-Newton method is:
//
//   A  stage-parallel (lane = interval k): dynamics, the fixed masked row
//      layout of Sec. III-C (4 dynamics rows, 1 mode equality, 6
//      inequalities), PHR multiplier estimates, merit / violation /
//      complementarity, the local AL model over (u_k, x_{k+1}, x_k) and the
//      elimination of the u_k block (independent of the value function, so
//      it is taken off the sequential path);
//   B  the state steps dx_0 .. dx_N from the block-tridiagonal system left
//      after phase A (S_k = H_k + rho I + beta A_k^T A_k, Sec. III-C
//      "Fixed-workspace local solves"): the same block Cholesky without
//      pivoting as the backward sweep, taken in a lane-parallel order
//      (lanes fold their stages, a shuffle tree joins them, a root solve,
//      back-substitution); a failed pivot raises damping;
//   C  stage-parallel control steps du_k from the u-block factors and dx;
//   D  parallel trial-step merits: lane = (trial alpha, stage group), alpha
//      in {0, 1, 1/2, ..., 1/64}, Armijo on the largest passing alpha;
//   E  compensated update z += alpha dz and multiplier / penalty updates.
//
// The algorithm (steps, order, constants) is the one the FP64 oracle runs;
// only the arithmetic precision and the parallel schedule differ.

#include <cuda_runtime.h>
#include <cuda/annotated_ptr>
#include <math.h>
#include <stdint.h>

#include "comet_internal.h"

namespace comet {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------ warp helpers

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// error-free sum a + b = s + e (Knuth two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// lower-triangle flat index of (i, j), i >= j
__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// Warm-start staging: one bulk copy (cp.async.bulk, the untiled TMA path)
// completing on the warp's mbarrier.  Waits are bounded (about one second
// of clock cycles) and report whether the phase completed.
constexpr long long kStageWaitCycles = 2000000000ll;
__device__ __forceinline__ uint32_t ek_smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool ek_mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool ek_mbar_wait(uint32_t bar, uint32_t parity) {
    if (ek_mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (ek_mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > kStageWaitCycles) return false;
    }
}
// dst (shared) and src (global) 16-byte aligned, bytes a positive multiple of 16
__device__ __forceinline__ void ek_bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// face geometry: inward normal n, tangent t = rot90(n)
__device__ __forceinline__ void face_nt(int face, float& nx, float& ny) {
    nx = (face == 0) ? 1.f : ((face == 2) ? -1.f : 0.f);
    ny = (face == 1) ? 1.f : ((face == 3) ? -1.f : 0.f);
}

// Pushing modes 0..11 are face (m / 3) x {stick, slide+, slide-} (m % 3);
// mode 12 is free motion (Sec. III-A): the pusher is off the slider, the
// contact force is zero and the slider rests.
constexpr int kModeFree = 12;

struct ModeInfo {
    int face, kind;  // kind 0 stick, 1 slide+, 2 slide-, 3 free motion
    bool smask;      // s-row of d_k masked (the pusher is not on the same face at both ends)
};

__device__ __forceinline__ ModeInfo mode_of(unsigned char b) {
    ModeInfo mi;
    mi.face = b & 3;
    mi.kind = (b >> 2) & 3;
    mi.smask = (b >> 4) & 1;
    return mi;
}

__device__ __forceinline__ ModeInfo mode_info(const uint16_t* modes, int len, int N, int k) {
    ModeInfo mi;
    const int seg = (int)(((long long)k * len) / N);
    const int m = modes[seg];
    const bool free = m == kModeFree;
    mi.face = free ? 0 : m / 3;
    mi.kind = free ? 3 : m - 3 * mi.face;
    // the contact offset may jump when the pusher leaves the face: free
    // motion on either side of knot k+1, or another face next
    mi.smask = free;
    if (!free && k + 1 < N) {
        const int seg1 = (int)(((long long)(k + 1) * len) / N);
        const int m1 = modes[seg1];
        mi.smask = m1 == kModeFree || (m1 / 3) != mi.face;
    }
    return mi;
}

// --------------------------------------------------------------- the rows

// Residual rows of interval k at (x_k, u_k, x_{k+1}) with the exact state
// difference dx = x_{k+1} - x_k.  Values are internally scaled; `phys` is
// the factor that maps a scaled value back to physical units.
//
// The theta row is evaluated in double-float (pairs of FP32 values).  Its
// rate kappa m_z / c^2 is large for a small limit-surface constant c, so the
// per-interval rotation dt * omega and the state difference it balances are
// large beside the defect itself; rounded to FP32, the defect carries noise
// of the order of its converged size, which beta turns into a stationarity
// floor (Sec. III-C, stopping test).  The pair keeps the difference exact.
struct Rows {
    float c[11];
    float phys[11];
    bool on[11];
    // dynamics Jacobian pieces (scaled): d c_r / d x_k, d c_r / d u_k
    float ax[4][4];
    float au[4][3];
    float ay[4];  // d c_r / d x_{k+1, r}
    // linear rows' u-Jacobians (rows 4..8)
    float lu[5][3];
    // dynamics values for the curvature term; kf = force-to-velocity gain
    // of the interval (0 in free motion)
    float f0, f1, ct, st, kf;
};

// kFree: free motion (mode 12) compiled in; problems over the 12 contact
// modes run the variant without it.
// Inputs: xk = x_k and dx = x_{k+1} - x_k rounded to FP32, except dx[2] =
// fl(theta_{k+1,hi} - theta_{k,hi}); ex[0] = the rest of the theta
// difference, ex[1] = s_k - xk[3] (see stage_state).
template <bool kFree>
__device__ __forceinline__ void eval_rows(const DevInstance& P, const ModeInfo& mi, const float xk[4],
                                          const float dx[4], const float ex[2], const float u[3], Rows& R) {
    float nx, ny;
    face_nt(mi.face, nx, ny);
    const float tx = -ny, ty = nx;
    const float a = P.a[mi.face], ell = P.ell[mi.face];
    // free motion: zero force-to-velocity gain, so the slider rests and only
    // the contact offset moves (at the pusher's rate)
    const bool free = kFree && mi.kind == 3;
    const float k = free ? 0.f : P.kappa, ic2 = P.inv_c2, dt = P.dt;
    const float th = xk[2], s = xk[3];
    const float fn = u[0], ft = u[1], sd = u[2];
    float st, ct;
    sincosf(th, &st, &ct);
    // quasi-static pusher-slider on an ellipsoidal limit surface:
    // body twist = kappa * (F_x, F_y, m_z / c^2), m_z = -a f_t - s f_n
    const float vx = k * (fn * nx + ft * tx);
    const float vy = k * (fn * ny + ft * ty);
    const float w = k * (-a * ft - s * fn) * ic2;
    const float f[4] = {ct * vx - st * vy, st * vx + ct * vy, w, sd};
    R.f0 = f[0];
    R.f1 = f[1];
    R.ct = ct;
    R.st = st;
    R.kf = k;
    // Jacobians of f
    const float Fx02 = -st * vx - ct * vy, Fx12 = ct * vx - st * vy, Fx23 = -k * fn * ic2;
    const float Fu[4][3] = {{k * (ct * nx - st * ny), k * (ct * tx - st * ty), 0.f},
                            {k * (st * nx + ct * ny), k * (st * tx + ct * ty), 0.f},
                            {-k * s * ic2, -k * a * ic2, 0.f},
                            {0.f, 0.f, 1.f}};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float is = P.inv_sigma[r];
        R.c[r] = (dx[r] - dt * f[r]) * is;
        R.phys[r] = 1.f / is;
        R.on[r] = true;
#pragma unroll
        for (int j = 0; j < 4; ++j) R.ax[r][j] = (r == j) ? -is : 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) R.au[r][j] = -dt * Fu[r][j] * is;
        R.ay[r] = is;
    }
    {
        // c_2 sigma_2 = dtheta + K (a f_t + s f_n), K = dt kappa / c^2, with
        // error-free products (fma) and sums (two_sum)
        const float kh = free ? 0.f : P.kth_hi, kl = free ? 0.f : P.kth_lo;
        const float p = a * ft, pe = fmaf(a, ft, -p) + P.a_lo[mi.face] * ft;
        const float q = s * fn, qe = fmaf(s, fn, -q) + ex[1] * fn;
        float m, me;
        two_sum(p, q, m, me);
        me += pe + qe;
        const float km = kh * m, kme = fmaf(kh, m, -km) + (kh * me + kl * m);
        float t, te;
        two_sum(dx[2], km, t, te);
        R.c[2] = (t + (te + ex[0] + kme)) * P.inv_sigma[2];
    }
    R.ax[0][2] += -dt * Fx02 * P.inv_sigma[0];
    R.ax[1][2] += -dt * Fx12 * P.inv_sigma[1];
    R.ax[2][3] += -dt * Fx23 * P.inv_sigma[2];
    if (mi.smask) R.on[3] = false;

    const float mu = P.mu, sc = P.sc_cone;
    const bool stick = mi.kind == 0;
    const float sg = (mi.kind == 1) ? -1.f : 1.f;
    // row 4: mode equality.  Free motion: f_n = 0 is the only force row
    // (rows 5..10 off); f_t acts on nothing and the effort cost sets it to 0
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
    // rows 5, 6: friction cone (sticking only)
    R.c[5] = sc * (ft - mu * fn);
    R.lu[1][0] = -sc * mu; R.lu[1][1] = sc; R.lu[1][2] = 0.f;
    R.c[6] = sc * (-ft - mu * fn);
    R.lu[2][0] = -sc * mu; R.lu[2][1] = -sc; R.lu[2][2] = 0.f;
    R.phys[5] = R.phys[6] = 1.f / sc;
    R.on[5] = R.on[6] = stick;
    // row 7: sliding direction
    R.c[7] = sg * sd;
    R.lu[3][0] = 0.f; R.lu[3][1] = 0.f; R.lu[3][2] = sg;
    R.phys[7] = 1.f;
    R.on[7] = !stick && !free;
    // row 8: unilateral contact -f_n <= 0
    R.c[8] = -fn;
    R.lu[4][0] = -1.f; R.lu[4][1] = 0.f; R.lu[4][2] = 0.f;
    R.phys[8] = 1.f;
    R.on[8] = !free;
    // rows 9, 10: contact point on the face, |s_k| <= ell
    R.c[9] = s - ell;
    R.c[10] = -s - ell;
    R.phys[9] = R.phys[10] = 1.f;
    R.on[9] = R.on[10] = !free;
#pragma unroll
    for (int r = 0; r < 11; ++r)
        if (!R.on[r]) R.c[r] = 0.f;
}

// State pieces of interval k from the compensated storage: x_k = h0 + l0,
// x_{k+1} = h1 + l1 (the low parts may carry a trial step).  Returns x_k
// and x_{k+1} - x_k rounded to FP32, with the theta difference and s_k
// split for the theta row: dx[2] + ex[0] = theta_{k+1} - theta_k and
// xk[3] + ex[1] = s_k.
__device__ __forceinline__ void stage_state(const float h0[4], const float h1[4], const float l0[4],
                                            const float l1[4], float xk[4], float dx[4], float ex[2]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        xk[i] = h0[i] + l0[i];
        dx[i] = (h1[i] - h0[i]) + (l1[i] - l0[i]);
    }
    float e;
    two_sum(h1[2], -h0[2], dx[2], e);
    ex[0] = e + (l1[2] - l0[2]);
    two_sum(h0[3], l0[3], xk[3], ex[1]);
}

// Nonzero pattern of dynamics row r over the stage variables (u0..2 at
// 0..2, y = x_{k+1} at 3..6, x_k at 7..10), ascending; -1 pads.  Rows 0, 1
// (x, y): f_n, f_t, their own y, their own x and theta; row 2 (theta): f_n,
// f_t, y_2, theta, s; row 3 (s): the pusher velocity, y_3, s.
__host__ __device__ constexpr int dyn_nz(int r, int a) {
    return r == 0 ? (a == 0 ? 0 : a == 1 ? 1 : a == 2 ? 3 : a == 3 ? 7 : 9)
         : r == 1 ? (a == 0 ? 0 : a == 1 ? 1 : a == 2 ? 4 : a == 3 ? 8 : 9)
         : r == 2 ? (a == 0 ? 0 : a == 1 ? 1 : a == 2 ? 5 : a == 3 ? 9 : 10)
                  : (a == 0 ? 2 : a == 1 ? 6 : a == 2 ? 10 : -1);
}

// PHR augmented-Lagrangian pieces of one row
__device__ __forceinline__ float row_al(bool ineq, float lam, float beta, float inv2b, float c) {
    if (!ineq) return lam * c + 0.5f * beta * c * c;
    const float t = fmaxf(lam + beta * c, 0.f);
    return (t * t - lam * lam) * inv2b;
}

// ------------------------------------------------------------ shared memory

struct Smem {
    unsigned long long* mbar;  // the warp's mbarrier (warm-start staging), 16 bytes reserved
    unsigned char* mb;  // [Nmax] per-interval mode byte: face | kind << 2 | smask << 4
    float* xh;   // [4][Nmax+1] state, high part
    float* xl;   // [4][Nmax+1] state, low part
    float* us;   // [3][Nmax]
    float* lam;  // [3 + 11 Nmax]
    float* dz;   // [7 Nmax + 4] interleaved step
    float* gr;   // [7 Nmax + 4] interleaved AL gradient
};

__host__ __device__ inline size_t smem_floats(int Nmax) {
    const size_t f = 4 + (size_t)(Nmax + 3) / 4 + (size_t)8 * (Nmax + 1) +
                     3 * (size_t)Nmax + 3 + 11 * (size_t)Nmax + 2 * (7 * (size_t)Nmax + 4);
    return (f + 3) / 4 * 4;  // every warp's block starts 16-byte aligned
}

__device__ __forceinline__ Smem carve(float* base, int Nmax) {
    Smem s;
    float* p = base;
    s.mbar = reinterpret_cast<unsigned long long*>(p); p += 4;
    s.mb = reinterpret_cast<unsigned char*>(p); p += (Nmax + 3) / 4;
    s.xh = p; p += 4 * (Nmax + 1);
    s.xl = p; p += 4 * (Nmax + 1);
    s.us = p; p += 3 * Nmax;
    s.lam = p; p += 3 + 11 * Nmax;
    s.dz = p; p += 7 * Nmax + 4;
    s.gr = p;
    return s;
}

// ------------------------------------------------- per-TO solver context

struct Ctx {
    const DevInstance* P;
    uint16_t modes[COMET_MAX_SEGMENTS];
    int len, N, Nmax;
    Smem sm;
    float* rec;  // this warp's stage records (chunk-major, see rec_chunk)
    int lane;
};

// Stage records are stored chunk-major: float4 chunk q (record floats
// 4q .. 4q+3) of stage k sits at rec + 4 (q N_max + k), so that the
// stage-parallel passes (lane = stage) move whole 128-byte lines, while the
// sequential passes still fetch a stage's chunks 16 bytes at a time.
__device__ __forceinline__ float4* rec_chunk(const Ctx& C, int q, int k) {
    return reinterpret_cast<float4*>(C.rec + 4 * ((size_t)q * C.Nmax + k));
}

// Record stores carry the persisting (evict-last) L2 priority: the records
// of all resident warps (about 47 MB at N = 80) fit in L2 and are rewritten
// every iteration, and with the normal priority they were written back to
// DRAM at 1.1 GB per 4,096 TOs; with it, 46 MB, at the same speed.
__device__ __forceinline__ void rec_st(const Ctx& C, int q, int k, float4 v) {
    cuda::annotated_ptr<float4, cuda::access_property::persisting> p(rec_chunk(C, q, k));
    *p = v;
}

// Phase A over all stages.  Computes the violation / stationarity /
// complementarity measures of the current iterate, the AL gradient (into
// sm.gr), and, if `assemble`, the stage records for the sweep.  With
// `update`, the multipliers are first replaced by their PHR estimates at
// beta_old (the dual update of the outer loop).
struct Measures {
    float viol, stat, comp;
    float vphys;  // violation in physical units (rows mapped back by phys)
    float cost;   // objective J at the iterate (scale of the stationarity test)
    bool finite;
};

template <bool kFree, int kUnr = 1>
__device__ Measures phase_a(Ctx& C, float beta, float rho, bool curvature, bool assemble, bool update,
                            float beta_old, bool rhs_from_gr = false) {
    const DevInstance& P = *C.P;
    const int N = C.N, Np1 = C.N + 1, lane = C.lane;
    Smem& S = C.sm;
    float viol = 0.f, comp = 0.f, vph = 0.f, jc = 0.f;
    bool finite = true;
#pragma unroll (kUnr)
    for (int k = lane; k < N; k += 32) {
        const ModeInfo mi = mode_of(S.mb[k]);
        float h0[4], h1[4], l0[4], l1[4], xk[4], dx[4], ex[2], u[3];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            h0[i] = S.xh[i * Np1 + k];
            h1[i] = S.xh[i * Np1 + k + 1];
            l0[i] = S.xl[i * Np1 + k];
            l1[i] = S.xl[i * Np1 + k + 1];
        }
        stage_state(h0, h1, l0, l1, xk, dx, ex);
#pragma unroll
        for (int j = 0; j < 3; ++j) u[j] = S.us[j * N + k];
        Rows R;
        eval_rows<kFree>(P, mi, xk, dx, ex, u, R);
        float* lam = S.lam + 3 + 11 * k;
        float y[11];
        bool act[11];
#pragma unroll
        for (int r = 0; r < 11; ++r) {
            const bool ineq = r >= 5;
            float l = lam[r];
            if (update && R.on[r]) {
                const float t = l + beta_old * R.c[r];
                l = ineq ? fmaxf(t, 0.f) : t;
                lam[r] = l;
            }
            const float t = l + beta * R.c[r];
            act[r] = R.on[r] && (!ineq || t > 0.f);
            y[r] = act[r] ? (ineq ? fmaxf(t, 0.f) : t) : 0.f;
            if (R.on[r]) {
                const float vr = ineq ? fmaxf(R.c[r], 0.f) : fabsf(R.c[r]);
                viol = fmaxf(viol, vr);
                vph = fmaxf(vph, vr * R.phys[r]);
                if (ineq) comp = fmaxf(comp, fabsf(y[r] * R.c[r]));
                if (!isfinite(R.c[r])) finite = false;
            }
        }
        jc += P.w_control * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        // local AL gradient over (x_k, u_k, x_{k+1})
        float gx[4] = {0.f, 0.f, 0.f, 0.f}, gu[3], gy[4];
        const float R2 = 2.f * P.w_control;
#pragma unroll
        for (int j = 0; j < 3; ++j) gu[j] = R2 * u[j];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int j = 0; j < 4; ++j) gx[j] += y[r] * R.ax[r][j];
#pragma unroll
            for (int j = 0; j < 3; ++j) gu[j] += y[r] * R.au[r][j];
            gy[r] = y[r] * R.ay[r];
        }
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
            for (int j = 0; j < 3; ++j) gu[j] += y[4 + q] * R.lu[q][j];
        gx[3] += y[9] - y[10];
        if (rhs_from_gr) {
            // the right-hand side is a given vector per variable (the FP64
            // residual of a refinement step): u_k and x_{k+1} entries go to
            // this stage, x_0's to stage 0
#pragma unroll
            for (int j = 0; j < 3; ++j) gu[j] = S.gr[7 * k + 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                gy[i] = S.gr[7 * (k + 1) + i];
                gx[i] = (k == 0) ? S.gr[i] : 0.f;
            }
        } else {
            // interleaved gradient: x_k slot gets the x_k part here, the x_{k+1}
            // part is parked in dz and added in the pass below
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                S.gr[7 * k + i] = gx[i];
                S.dz[7 * (k + 1) + i] = gy[i];
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) S.gr[7 * k + 4 + j] = gu[j];
        }

        if (assemble) {
            // augmented local matrix over (u0..2, y0..3, x0..3, rhs), lower triangle
            float A[78];
#pragma unroll
            for (int t = 0; t < 78; ++t) A[t] = 0.f;
            // cost and proximal damping
#pragma unroll
            for (int j = 0; j < 3; ++j) A[tri(j, j)] += R2 + rho;
#pragma unroll
            for (int i = 0; i < 4; ++i) A[tri(3 + i, 3 + i)] += rho;
            // beta a a^T over active rows; dynamics rows first, on their fixed
            // nonzero pattern (dyn_nz) over (u0..2, y0..3, x0..3)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float vv[11];
#pragma unroll
                for (int j = 0; j < 3; ++j) vv[j] = R.au[r][j];
#pragma unroll
                for (int i = 0; i < 4; ++i) vv[3 + i] = (i == r) ? R.ay[r] : 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i) vv[7 + i] = R.ax[r][i];
                const float bw = act[r] ? beta : 0.f;
#pragma unroll
                for (int a = 0; a < 5; ++a) {
                    const int i = dyn_nz(r, a);
                    if (i < 0) continue;
                    const float t = bw * vv[i];
#pragma unroll
                    for (int b = 0; b <= a; ++b) A[tri(i, dyn_nz(r, b))] += t * vv[dyn_nz(r, b)];
                }
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const float bw = act[4 + q] ? beta : 0.f;
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j <= i; ++j) A[tri(i, j)] += bw * R.lu[q][i] * R.lu[q][j];
            }
            A[tri(10, 10)] += (act[9] ? beta : 0.f) + (act[10] ? beta : 0.f);
            if (curvature) {
                // Lagrangian curvature of the dynamics rows, -dt sum_r yd_r d^2 f_r,
                // with yd_r the multiplier of the unscaled row
                float nx, ny;
                face_nt(mi.face, nx, ny);
                const float tx = -ny, ty = nx, kk = kFree ? R.kf : P.kappa;  // R.kf = 0 in free motion
                const float yd0 = y[0] * P.inv_sigma[0], yd1 = y[1] * P.inv_sigma[1];
                const float yd2 = y[2] * P.inv_sigma[2];
                const float h_thth = -yd0 * R.f0 - yd1 * R.f1;
                const float h_thfn = yd0 * kk * (-R.st * nx - R.ct * ny) + yd1 * kk * (R.ct * nx - R.st * ny);
                const float h_thft = yd0 * kk * (-R.st * tx - R.ct * ty) + yd1 * kk * (R.ct * tx - R.st * ty);
                const float h_sfn = -yd2 * kk * P.inv_c2;
                A[tri(9, 9)] -= P.dt * h_thth;  // (theta_k, theta_k)
                A[tri(9, 0)] -= P.dt * h_thfn;  // (theta_k, f_n)
                A[tri(9, 1)] -= P.dt * h_thft;  // (theta_k, f_t)
                A[tri(10, 0)] -= P.dt * h_sfn;  // (s_k, f_n)
            }
            // right-hand side row: the gradient (u, y, x)
#pragma unroll
            for (int j = 0; j < 3; ++j) A[tri(11, j)] = gu[j];
#pragma unroll
            for (int i = 0; i < 4; ++i) A[tri(11, 3 + i)] = gy[i];
#pragma unroll
            for (int i = 0; i < 4; ++i) A[tri(11, 7 + i)] = gx[i];
            // eliminate the u block (3 Cholesky steps); a non-positive pivot
            // marks the record (the sweep then reports failure).  The
            // diagonal keeps 1 / l_jj, which is all the control step needs.
            bool pd = true;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float d = A[tri(j, j)];
                pd = pd && (d > 0.f);
                const float il = rsqrtf(fmaxf(d, 1e-30f));
                A[tri(j, j)] = il;
#pragma unroll
                for (int i = j + 1; i < 12; ++i) A[tri(i, j)] *= il;
#pragma unroll
                for (int c = j + 1; c < 12; ++c)
#pragma unroll
                    for (int i = c; i < 12; ++i) A[tri(i, c)] -= A[tri(i, j)] * A[tri(c, j)];
            }
            float rec[kRec];
            rec[0] = A[tri(0, 0)]; rec[1] = A[tri(1, 0)]; rec[2] = A[tri(1, 1)];
            rec[3] = A[tri(2, 0)]; rec[4] = A[tri(2, 1)]; rec[5] = A[tri(2, 2)];
#pragma unroll
            for (int i = 3; i < 12; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) rec[6 + (i - 3) * 3 + j] = A[tri(i, j)];
            rec[33] = pd ? 1.f : -1.f;
            rec[34] = 0.f;
            rec[35] = 0.f;
#pragma unroll
            for (int i = 3; i < 12; ++i)
#pragma unroll
                for (int j = 3; j <= i; ++j)
                    if (!(i == 11 && j == 11)) rec[36 + tri(i - 3, j - 3)] = A[tri(i, j)];
#pragma unroll
            for (int q = 0; q < kRec / 4; ++q)
                rec_st(C, q, k, make_float4(rec[4 * q], rec[4 * q + 1], rec[4 * q + 2], rec[4 * q + 3]));
        }
    }
    __syncwarp();
    // initial-state rows (3, unscaled) and terminal cost
    if (lane < 3) {
        float l = S.lam[lane];
        const float c = (S.xh[lane * Np1] - P.start[lane]) + S.xl[lane * Np1];
        if (update) {
            l = l + beta_old * c;
            S.lam[lane] = l;
        }
        viol = fmaxf(viol, fabsf(c));
        vph = fmaxf(vph, fabsf(c));
        if (!isfinite(c)) finite = false;
    }
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float e = (S.xh[i * Np1 + N] - P.goal[i]) + S.xl[i * Np1 + N];
            jc += P.w_terminal * e * e;
        }
    __syncwarp();
    // combine the x parts of the gradient and take the stationarity measure
    float stat = 0.f;
    for (int k = lane; k <= N && !rhs_from_gr; k += 32) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float g = (k < N) ? S.gr[7 * k + i] : 0.f;
            if (k > 0) g += S.dz[7 * k + i];
            if (k == N && i < 3) g += 2.f * P.w_terminal * ((S.xh[i * Np1 + N] - P.goal[i]) + S.xl[i * Np1 + N]);
            if (k == 0 && i < 3) {
                const float c = (S.xh[i * Np1] - P.start[i]) + S.xl[i * Np1];
                g += S.lam[i] + beta * c;
            }
            S.gr[7 * k + i] = g;
            stat = fmaxf(stat, fabsf(g));
            if (!isfinite(g)) finite = false;
        }
        if (k < N) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float g = S.gr[7 * k + 4 + j];
                stat = fmaxf(stat, fabsf(g));
                if (!isfinite(g)) finite = false;
            }
        }
    }
    __syncwarp();
    Measures m;
    m.viol = warp_max(viol);
    m.stat = warp_max(stat);
    m.comp = warp_max(comp);
    m.vphys = warp_max(vph);
    m.cost = warp_sum(jc);
    m.finite = __all_sync(kFull, finite);
    return m;
}

// Phase B: the step's state part by a lane-parallel elimination of the
// block-tridiagonal system over dx_0 .. dx_N (Sec. III-C "Fixed-workspace
// local solves": after the u block of each stage is eliminated in phase A,
// the stage record holds a quadratic "element" in (dx_{k+1}, dx_k), the
// reduced 9 x 9 lower triangle over (y = x_{k+1}, x = x_k, rhs)).  The paper
// eliminates the x_{k+1} blocks one stage after another (the backward sweep);
// the same block Cholesky is taken here in another order, so that the lanes
// share the chain instead of each lane repeating it:
//   1. lane l owns stages [k0, k1) (k1 - k0 = ceil(N / 32)) and folds them
//      into one element over (x_{k1}, x_{k0}), eliminating its interior
//      nodes left to right;
//   2. a tree over the lanes (log2 of the active lanes levels, the partner's
//      element arriving by shuffles) eliminates the nodes between the lanes'
//      spans, until lane 0 holds an element over (x_N, x_0);
//   3. lane 0 solves that 8 x 8 system for dx_0 and dx_N;
//   4. back-substitution down the tree, then through each lane's interior.
// Eliminating node m between an element E over (m, a) and F over (b, m):
// S = E_mm + F_mm = L L^T, Y = L^{-1} [F_mb | E_ma | r_m], and the element
// over (b, a) is blockdiag(F_bb, E_aa) - Y^T Y; later dx_m =
// -L^{-T} (Y_b dx_b + Y_a dx_a + y_r).  Node m keeps (L, Y) in record floats
// 34..79 (the reduced matrix there is consumed).  The matrix is positive
// definite exactly when every pivot of every elimination is positive, in
// any order (inertia is additive over Schur complements), so the test of
// the backward sweep is unchanged: a non-positive pivot anywhere, or a
// non-positive u-block pivot flagged by phase A, reports failure.
// The terminal cost's value function V_N, v_N enters the last stage's y
// block and the x_0 block (rho I, beta on the three pose rows, their
// multiplier terms) the first stage's x block.  Writes dx_k to dz[7k..7k+3]
// for k = 0..N; returns false if a pivot is not positive.

constexpr int kElem = 44;  // 9 x 9 lower triangle without the (rhs, rhs) entry

// record floats 36..79 (the reduced matrix) of stage k as an element, with
// the boundary terms of the first and the last stage
__device__ __forceinline__ void load_elem(const Ctx& C, int k, float e[kElem], float beta, float rho,
                                          bool rhs_from_gr) {
#pragma unroll
    for (int q = 0; q < 11; ++q) {
        const float4 t = *rec_chunk(C, 9 + q, k);
        e[4 * q] = t.x;
        e[4 * q + 1] = t.y;
        e[4 * q + 2] = t.z;
        e[4 * q + 3] = t.w;
    }
    const DevInstance& P = *C.P;
    const int N = C.N, Np1 = N + 1;
    const Smem& S = C.sm;
    if (k == N - 1) {
        // V_N, v_N of the terminal cost w_T |pose_N - goal|^2 on the y block
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            e[tri(i, i)] += 2.f * P.w_terminal;
            if (!rhs_from_gr)
                e[tri(8, i)] += 2.f * P.w_terminal * ((S.xh[i * Np1 + N] - P.goal[i]) + S.xl[i * Np1 + N]);
        }
    }
    if (k == 0) {
        // the x_0 block: damping, and beta on the initial pose rows
#pragma unroll
        for (int i = 0; i < 4; ++i) e[tri(4 + i, 4 + i)] += rho + (i < 3 ? beta : 0.f);
        if (!rhs_from_gr)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float c = (S.xh[i * Np1] - P.start[i]) + S.xl[i * Np1];
                e[tri(8, 4 + i)] += S.lam[i] + beta * c;
            }
    }
}

// Eliminate the node shared by e (over (y = m, x = a)) and f (over (y = b,
// x = m)); e becomes the element over (y = b, x = a).  Stores (L, Y) of node
// m in record `km` when `store`; returns false on a non-positive pivot.
__device__ __forceinline__ bool combine(const Ctx& C, float e[kElem], const float f[kElem], int km, bool store) {
    // S = E_yy + F_xx and its Cholesky factor (il = 1 / l_jj on the diagonal)
    float L[10];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) L[tri(i, j)] = e[tri(i, j)] + f[tri(4 + i, 4 + j)];
    bool pd = true;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float d = L[tri(j, j)];
#pragma unroll
        for (int q = 0; q < j; ++q) d -= L[tri(j, q)] * L[tri(j, q)];
        pd = pd && d > 0.f;
        const float il = rsqrtf(fmaxf(d, 1e-30f));
        L[tri(j, j)] = il;
#pragma unroll
        for (int i = j + 1; i < 4; ++i) {
            float s = L[tri(i, j)];
#pragma unroll
            for (int q = 0; q < j; ++q) s -= L[tri(i, q)] * L[tri(j, q)];
            L[tri(i, j)] = s * il;
        }
    }
    // Y = L^{-1} [F_mb | E_ma | r_m], columns b0..3, a0..3, rhs
    float Y[4][9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float s = (c < 4) ? f[tri(4 + i, c)] : (c < 8) ? e[tri(4 + (c - 4), i)] : e[tri(8, i)] + f[tri(8, 4 + i)];
#pragma unroll
            for (int q = 0; q < i; ++q) s -= L[tri(i, q)] * Y[q][c];
            Y[i][c] = s * L[tri(i, i)];
        }
    }
    // the element over (y = b, x = a, rhs): blockdiag(F_bb, E_aa) - Y^T Y
    float g[kElem];
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            if (i == 8 && j == 8) continue;
            float s;
            if (i < 4)
                s = f[tri(i, j)];                              // (b, b)
            else if (i < 8)
                s = (j < 4) ? 0.f : e[tri(i, j)];              // (a, b) fill-in, (a, a)
            else
                s = (j < 4) ? f[tri(8, j)] : e[tri(8, j)];     // (rhs, b), (rhs, a)
#pragma unroll
            for (int p = 0; p < 4; ++p) s -= Y[p][i] * Y[p][j];
            g[tri(i, j)] = s;
        }
#pragma unroll
    for (int t = 0; t < kElem; ++t) e[t] = g[t];
    if (store) {
        *reinterpret_cast<float2*>(reinterpret_cast<float*>(rec_chunk(C, 8, km)) + 2) = make_float2(L[0], L[1]);
        rec_st(C, 9, km, make_float4(L[2], L[3], L[4], L[5]));
        rec_st(C, 10, km, make_float4(L[6], L[7], L[8], L[9]));
#pragma unroll
        for (int q = 0; q < 9; ++q)
            rec_st(C, 11 + q, km, make_float4(Y[(4 * q) / 9][(4 * q) % 9], Y[(4 * q + 1) / 9][(4 * q + 1) % 9],
                                              Y[(4 * q + 2) / 9][(4 * q + 2) % 9],
                                              Y[(4 * q + 3) / 9][(4 * q + 3) % 9]));
    }
    return pd;
}

// dx_m = -L^{-T} (Y_b dx_b + Y_a dx_a + y_r) from node m's stored (L, Y)
__device__ __forceinline__ void back_node(const Ctx& C, int km, const float xa[4], const float xb[4], float xm[4]) {
    float v[48];
    const float2 h = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(rec_chunk(C, 8, km)) + 2);
    v[0] = h.x;
    v[1] = h.y;
#pragma unroll
    for (int q = 0; q < 11; ++q) {
        const float4 t = *rec_chunk(C, 9 + q, km);
        v[2 + 4 * q] = t.x;
        v[3 + 4 * q] = t.y;
        v[4 + 4 * q] = t.z;
        v[5 + 4 * q] = t.w;
    }
    const float* L = v;        // 10
    const float* Y = v + 10;   // [4][9]
    float t[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float s = Y[9 * i + 8];
#pragma unroll
        for (int j = 0; j < 4; ++j) s += Y[9 * i + j] * xb[j] + Y[9 * i + 4 + j] * xa[j];
        t[i] = s;
    }
    // L^T xm = -t
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        float s = -t[i];
#pragma unroll
        for (int q = i + 1; q < 4; ++q) s -= L[tri(q, i)] * xm[q];
        xm[i] = s * L[tri(i, i)];
    }
}

__device__ bool phase_b(Ctx& C, float beta, float rho, bool rhs_from_gr = false) {
    const int N = C.N, lane = C.lane;
    Smem& S = C.sm;
    const int per = (N + 31) >> 5;
    const int nl = (N + per - 1) / per;  // lanes that own stages
    const int k0 = min(N, lane * per), k1 = min(N, k0 + per);
    const bool own = lane < nl;
    const int nlev = nl > 1 ? 32 - __clz(nl - 1) : 0;  // tree levels, ceil(log2 nl)
    const int nsteps = (per - 1) + nlev;
    bool pd = true;
    float e[kElem];
#pragma unroll
    for (int t = 0; t < kElem; ++t) e[t] = 0.f;
    if (own) {
        pd = reinterpret_cast<const float*>(rec_chunk(C, 8, k0))[1] > 0.f;
        load_elem(C, k0, e, beta, rho, rhs_from_gr);
    }
    // 1-2. one loop, one elimination call site: steps 0 .. per-2 fold the
    // lane's next stage (the u-block pivot flag of phase A checked on the
    // way), the remaining steps are the tree levels d = 1, 2, 4, ...: lane l
    // (a multiple of 2d) eliminates the first node of lane l + d's span
#pragma unroll 1
    for (int st = 0; st < nsteps; ++st) {
        float f[kElem];
        bool act;
        int km;
        if (st < per - 1) {  // warp-uniform
            km = k0 + 1 + st;
            act = own && km < k1;
            if (act) {
                pd = pd && reinterpret_cast<const float*>(rec_chunk(C, 8, km))[1] > 0.f;
                load_elem(C, km, f, beta, rho, rhs_from_gr);
            }
        } else {
            const int d = 1 << (st - (per - 1));
#pragma unroll
            for (int t = 0; t < kElem; ++t) f[t] = __shfl_down_sync(kFull, e[t], d);
            act = (lane & (2 * d - 1)) == 0 && lane + d < nl;
            km = (lane + d) * per;
        }
        if (act) pd = combine(C, e, f, km, true) && pd;
    }
    // 3. lane 0 solves the root element over (x_N, x_0): an 8 x 8 Cholesky
    float xl[4] = {0.f, 0.f, 0.f, 0.f}, xr[4] = {0.f, 0.f, 0.f, 0.f};
    if (lane == 0) {
        float A[36];
#pragma unroll
        for (int t = 0; t < 36; ++t) A[t] = e[t];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float dd = A[tri(j, j)];
#pragma unroll
            for (int q = 0; q < j; ++q) dd -= A[tri(j, q)] * A[tri(j, q)];
            pd = pd && dd > 0.f;
            const float il = rsqrtf(fmaxf(dd, 1e-30f));
            A[tri(j, j)] = il;
#pragma unroll
            for (int i = j + 1; i < 8; ++i) {
                float s = A[tri(i, j)];
#pragma unroll
                for (int q = 0; q < j; ++q) s -= A[tri(i, q)] * A[tri(j, q)];
                A[tri(i, j)] = s * il;
            }
        }
        float yv[8], x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float s = e[tri(8, i)];
#pragma unroll
            for (int q = 0; q < i; ++q) s -= A[tri(i, q)] * yv[q];
            yv[i] = s * A[tri(i, i)];
        }
#pragma unroll
        for (int i = 7; i >= 0; --i) {
            float s = yv[i];
#pragma unroll
            for (int q = i + 1; q < 8; ++q) s -= A[tri(q, i)] * x[q];
            x[i] = s * A[tri(i, i)];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            xr[i] = -x[i];      // dx_N
            xl[i] = -x[4 + i];  // dx_0
        }
    }
    // 4. back-substitution, one call site: the tree levels top-down (lane l
    // hands lane l + d the node it eliminated and its own right end), then
    // each lane's interior right to left
    float xc[4];  // dx of the node right of the current interior node
#pragma unroll 1
    for (int st = nsteps - 1; st >= 0; --st) {
        const bool tree = st >= per - 1;  // warp-uniform
        const int d = tree ? 1 << (st - (per - 1)) : 0;
        if (st == per - 2)
#pragma unroll
            for (int i = 0; i < 4; ++i) xc[i] = xr[i];
        const bool act = tree ? ((lane & (2 * d - 1)) == 0 && lane + d < nl) : (own && k0 + 1 + st < k1);
        const int km = tree ? (lane + d) * per : k0 + 1 + st;
        float xm[4] = {0.f, 0.f, 0.f, 0.f};
        if (act) back_node(C, km, xl, tree ? xr : xc, xm);
        if (tree) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float pm = __shfl_up_sync(kFull, xm[i], d), pr = __shfl_up_sync(kFull, xr[i], d);
                if ((lane & (2 * d - 1)) == d && lane < nl) {
                    xl[i] = pm;
                    xr[i] = pr;
                }
                if (act) xr[i] = xm[i];
            }
        } else if (act) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                S.dz[7 * km + i] = xm[i];
                xc[i] = xm[i];
            }
        }
    }
    if (own) {
#pragma unroll
        for (int i = 0; i < 4; ++i) S.dz[7 * k0 + i] = xl[i];
        if (lane == nl - 1)
#pragma unroll
            for (int i = 0; i < 4; ++i) S.dz[7 * N + i] = xr[i];
    }
    __syncwarp();
    return __all_sync(kFull, pd);
}

// Phase C: the control steps, stage-parallel from the u-block factors of
// phase A and the state steps of phase B,
//   du_k = -L_u^{-T} (l_{y,u}^T dx_{k+1} + l_{x,u}^T dx_k + l_{rhs,u}^T).
// Returns D = grad . dz.
template <int kUnr = 1>
__device__ float phase_c(Ctx& C) {
    const int N = C.N, lane = C.lane;
    Smem& S = C.sm;
#pragma unroll (kUnr)
    for (int k = lane; k < N; k += 32) {
        // record floats 0..35 as 9 vector loads (u-block factor, 1 / l_jj on
        // its diagonal, and the coupling columns)
        float f[36];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float4 t = *rec_chunk(C, q, k);
            f[4 * q] = t.x;
            f[4 * q + 1] = t.y;
            f[4 * q + 2] = t.z;
            f[4 * q + 3] = t.w;
        }
        float xa[4], xb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            xa[i] = S.dz[7 * k + i];
            xb[i] = S.dz[7 * (k + 1) + i];
        }
        float R[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float s = f[6 + 8 * 3 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i) s += f[6 + i * 3 + j] * xb[i] + f[6 + (4 + i) * 3 + j] * xa[i];
            R[j] = s;
        }
        const float du2 = -R[2] * f[5];
        const float du1 = (-R[1] - f[4] * du2) * f[2];
        const float du0 = (-R[0] - f[1] * du1 - f[3] * du2) * f[0];
        S.dz[7 * k + 4] = du0;
        S.dz[7 * k + 5] = du1;
        S.dz[7 * k + 6] = du2;
    }
    __syncwarp();
    float D = 0.f;
    for (int t = lane; t < 7 * N + 4; t += 32) D += S.gr[t] * S.dz[t];
    return warp_sum(D);
}

// merit contribution of interval k at the trial step alpha
template <bool kFree>
__device__ __forceinline__ float stage_merit(const Ctx& C, int k, float alpha, float beta, float inv2b) {
    const DevInstance& P = *C.P;
    const int N = C.N, Np1 = C.N + 1;
    const Smem& S = C.sm;
    const ModeInfo mi = mode_of(S.mb[k]);
    float h0[4], h1[4], l0[4], l1[4], xk[4], dx[4], ex[2], u[3];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h0[i] = S.xh[i * Np1 + k];
        h1[i] = S.xh[i * Np1 + k + 1];
        l0[i] = S.xl[i * Np1 + k] + alpha * S.dz[7 * k + i];
        l1[i] = S.xl[i * Np1 + k + 1] + alpha * S.dz[7 * (k + 1) + i];
    }
    stage_state(h0, h1, l0, l1, xk, dx, ex);
#pragma unroll
    for (int j = 0; j < 3; ++j) u[j] = S.us[j * N + k] + alpha * S.dz[7 * k + 4 + j];
    Rows R;
    eval_rows<kFree>(P, mi, xk, dx, ex, u, R);
    const float* lam = S.lam + 3 + 11 * k;
    float phi = P.w_control * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
    for (int r = 0; r < 11; ++r)
        if (R.on[r]) phi += row_al(r >= 5, lam[r], beta, inv2b, R.c[r]);
    if (k == 0) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float c = (S.xh[i * Np1] - P.start[i]) + (S.xl[i * Np1] + alpha * S.dz[i]);
            phi += row_al(false, S.lam[i], beta, inv2b, c);
        }
    }
    if (k == N - 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float e = (S.xh[i * Np1 + N] - P.goal[i]) + (S.xl[i * Np1 + N] + alpha * S.dz[7 * N + i]);
            phi += P.w_terminal * e * e;
        }
    }
    return phi;
}

// Phase D: trial merits for alpha in {0, 1, 1/2, ..., 2^-(n_alpha-1)};
// the accepted alpha is the largest one passing the test (0 = rejected).
// Trials run four at a time (lane = trial + 4 x stage group), largest alpha
// first: the second batch {1/8 .. 1/64} is evaluated only when none of
// {1, 1/2, 1/4} passes, which leaves the accepted alpha unchanged.
// Stage merits are summed as FP32 pairs (two_sum), so the tests compare
// phi(alpha) - phi(0) to the predicted decrease without the rounding of
// the total, which near convergence is as large as that decrease.
template <bool kFree, int kUnr = 1>
__device__ float phase_d(const Ctx& C, float beta, float D, const SolverParams& sp) {
    const int lane = C.lane;
    const int sub = lane & 3, grp = lane >> 2;
    const float inv2b = 0.5f / beta;
    float phi0 = 0.f, phi0l = 0.f, slack = 0.f;
#pragma unroll 1
    for (int batch = 0; batch < 2; ++batch) {
        const int a = 4 * batch + sub;  // trial index: alpha = 2^-(a-1), a = 0 -> alpha = 0
        if (batch == 1 && sp.n_alpha < 4) break;
        const float alpha = (a == 0) ? 0.f : ldexpf(1.f, -(a - 1));
        float phi = 0.f, phil = 0.f;
        if (a <= sp.n_alpha)
#pragma unroll (kUnr)
            for (int k = grp; k < C.N; k += 8) {
                float e;
                two_sum(phi, stage_merit<kFree>(C, k, alpha, beta, inv2b), phi, e);
                phil += e;
            }
#pragma unroll
        for (int off = 4; off <= 16; off <<= 1) {
            const float oh = __shfl_xor_sync(kFull, phi, off), ol = __shfl_xor_sync(kFull, phil, off);
            float e;
            two_sum(phi, oh, phi, e);
            phil += ol + e;
        }
        if (batch == 0) {
            phi0 = __shfl_sync(kFull, phi, 0);
            phi0l = __shfl_sync(kFull, phil, 0);
            slack = sp.ls_slack * fabsf(phi0);
        }
        const float dphi = (phi - phi0) + (phil - phi0l);
        bool pass = (a >= 1) && (a <= sp.n_alpha) && (dphi <= sp.armijo_c1 * alpha * D);
        if (a == 1 && fabsf(D) <= slack && dphi <= slack) pass = true;
        const unsigned bal = __ballot_sync(kFull, pass) & 0xfu;
        if (bal) return ldexpf(1.f, -(4 * batch + __ffs(bal) - 2));
    }
    return 0.f;
}

// Phase E: compensated update z += alpha dz
__device__ void phase_e(Ctx& C, float alpha) {
    const int N = C.N, Np1 = C.N + 1, lane = C.lane;
    Smem& S = C.sm;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        for (int k = lane; k < Np1; k += 32) {
            const int t = i * Np1 + k;
            float s, e;
            two_sum(S.xh[t], S.xl[t] + alpha * S.dz[7 * k + i], s, e);
            S.xh[t] = s;
            S.xl[t] = e;
        }
#pragma unroll
    for (int j = 0; j < 3; ++j)
        for (int k = lane; k < N; k += 32) S.us[j * N + k] += alpha * S.dz[7 * k + 4 + j];
    __syncwarp();
}

// FP64 rows of interval kk at the stored iterate (compensated states read as
// double): values c, physical factors ph, presence on, and the local
// Jacobian J[r][0..10] over (x_k[4], u_k[3], x_{k+1}[4]); also the pieces of
// the dynamics curvature.
struct Rows64 {
    double c[11], ph[11];
    bool on[11];
    double J[11][11];
    double f0, f1, ct, st, kf;  // kf: force-to-velocity gain (0 in free motion)
    double x0[4], x1[4], u[3];
};

__device__ void rows_fp64(const Ctx& C, int kk, Rows64& R) {
    const DevInstance& P = *C.P;
    const int N = C.N, Np1 = C.N + 1;
    const Smem& S = C.sm;
    const ModeInfo mi = mode_of(S.mb[kk]);
    for (int i = 0; i < 4; ++i) {
        R.x0[i] = (double)S.xh[i * Np1 + kk] + (double)S.xl[i * Np1 + kk];
        R.x1[i] = (double)S.xh[i * Np1 + kk + 1] + (double)S.xl[i * Np1 + kk + 1];
    }
    for (int j = 0; j < 3; ++j) R.u[j] = (double)S.us[j * N + kk];
    const double nx = (mi.face == 0) ? 1.0 : ((mi.face == 2) ? -1.0 : 0.0);
    const double ny = (mi.face == 1) ? 1.0 : ((mi.face == 3) ? -1.0 : 0.0);
    const double tx = -ny, ty = nx;
    const double a = P.a_d[mi.face], ell = P.ell_d[mi.face];
    const double kp = (mi.kind == 3) ? 0.0 : P.kappa_d, ic2 = P.inv_c2_d, dt = P.dt_d;
    R.kf = kp;
    double st, ct;
    sincos(R.x0[2], &st, &ct);
    const double fn = R.u[0], ft = R.u[1], sd = R.u[2];
    const double vx = kp * (fn * nx + ft * tx), vy = kp * (fn * ny + ft * ty);
    const double f[4] = {ct * vx - st * vy, st * vx + ct * vy, kp * (-a * ft - R.x0[3] * fn) * ic2, sd};
    R.f0 = f[0];
    R.f1 = f[1];
    R.ct = ct;
    R.st = st;
    const double Fx02 = -st * vx - ct * vy, Fx12 = ct * vx - st * vy, Fx23 = -kp * fn * ic2;
    const double Fu[4][3] = {{kp * (ct * nx - st * ny), kp * (ct * tx - st * ty), 0.0},
                             {kp * (st * nx + ct * ny), kp * (st * tx + ct * ty), 0.0},
                             {-kp * R.x0[3] * ic2, -kp * a * ic2, 0.0},
                             {0.0, 0.0, 1.0}};
    const double mu = P.mu_d, sc = P.sc_cone_d;
    const bool stick = mi.kind == 0;
    const double sg = (mi.kind == 1) ? -1.0 : 1.0;
    for (int r = 0; r < 11; ++r) {
        R.on[r] = true;
        R.ph[r] = 1.0;
        for (int j = 0; j < 11; ++j) R.J[r][j] = 0.0;
    }
    for (int r = 0; r < 4; ++r) {
        const double is = 1.0 / P.sigma_d[r];
        R.c[r] = (R.x1[r] - R.x0[r] - dt * f[r]) * is;
        R.ph[r] = P.sigma_d[r];
        R.J[r][r] = -is;
        R.J[r][7 + r] = is;
        for (int j = 0; j < 3; ++j) R.J[r][4 + j] = -dt * Fu[r][j] * is;
    }
    R.J[0][2] += -dt * Fx02 / P.sigma_d[0];
    R.J[1][2] += -dt * Fx12 / P.sigma_d[1];
    R.J[2][3] += -dt * Fx23 / P.sigma_d[2];
    if (mi.smask) R.on[3] = false;
    if (mi.kind == 3) {
        // free motion: f_n = 0 is the only force row
        R.c[4] = fn;
        R.J[4][4] = 1.0;
        for (int r = 5; r < 11; ++r) R.on[r] = false;
    } else {
        if (stick) {
            R.c[4] = sd;
            R.J[4][6] = 1.0;
        } else {
            R.c[4] = sc * (ft + sg * mu * fn);
            R.J[4][4] = sc * sg * mu;
            R.J[4][5] = sc;
            R.ph[4] = 1.0 / sc;
        }
        R.c[5] = sc * (ft - mu * fn);
        R.J[5][4] = -sc * mu;
        R.J[5][5] = sc;
        R.c[6] = sc * (-ft - mu * fn);
        R.J[6][4] = -sc * mu;
        R.J[6][5] = -sc;
        R.ph[5] = R.ph[6] = 1.0 / sc;
        R.on[5] = R.on[6] = stick;
        R.c[7] = sg * sd;
        R.J[7][6] = sg;
        R.on[7] = !stick;
        R.c[8] = -fn;
        R.J[8][4] = -1.0;
        R.c[9] = R.x0[3] - ell;
        R.J[9][3] = 1.0;
        R.c[10] = -R.x0[3] - ell;
        R.J[10][3] = -1.0;
    }
    for (int r = 0; r < 11; ++r)
        if (!R.on[r]) {
            R.c[r] = 0.0;
            for (int j = 0; j < 11; ++j) R.J[r][j] = 0.0;
        }
}

// FP64 certificate (Eq. inexact_mode_value in physical units, KKT residual)
struct Cert {
    double cost, viol, stat;
    bool finite;
};

__device__ Cert certify(const Ctx& C, float beta) {
    const DevInstance& P = *C.P;
    const int N = C.N, Np1 = C.N + 1, lane = C.lane;
    const Smem& S = C.sm;
    double cost = 0.0, viol = 0.0, stat = 0.0;
    bool finite = true;
    // gradient pieces are accumulated per knot: lane handles knots k and
    // recomputes the two adjacent intervals (k-1 as x_{k+1}, k as x_k)
    for (int k = lane; k <= N; k += 32) {
        double g[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
            const int kk = (side == 0) ? k - 1 : k;  // interval index
            if (kk < 0 || kk >= N) continue;
            Rows64 R;
            rows_fp64(C, kk, R);
            const float* lam = S.lam + 3 + 11 * kk;
            for (int r = 0; r < 11; ++r) {
                if (!R.on[r]) continue;
                const bool ineq = r >= 5;
                const double t = (double)lam[r] + (double)beta * R.c[r];
                const double y = ineq ? fmax(t, 0.0) : t;
                if (side == 1) {  // count each interval once
                    const double vr = ineq ? fmax(R.c[r], 0.0) : fabs(R.c[r]);
                    viol = fmax(viol, vr * R.ph[r]);
                    if (!isfinite(R.c[r])) finite = false;
                }
                // gradient: side 0 contributes the x_{k+1} columns, side 1 the x_k and u_k ones
                if (side == 0)
                    for (int i = 0; i < 4; ++i) g[i] += y * R.J[r][7 + i];
                else
                    for (int i = 0; i < 7; ++i) g[i] += y * R.J[r][i];
            }
            if (side == 1) {
                for (int j = 0; j < 3; ++j) {
                    g[4 + j] += 2.0 * P.w_control_d * R.u[j];
                    cost += P.w_control_d * R.u[j] * R.u[j];
                }
            }
        }
        if (k == N)
            for (int i = 0; i < 3; ++i) {
                const double e = (double)S.xh[i * Np1 + N] + (double)S.xl[i * Np1 + N] - P.goal_d[i];
                g[i] += 2.0 * P.w_terminal_d * e;
                cost += P.w_terminal_d * e * e;
            }
        if (k == 0)
            for (int i = 0; i < 3; ++i) {
                const double c = (double)S.xh[i * Np1] + (double)S.xl[i * Np1] - P.start_d[i];
                g[i] += (double)S.lam[i] + (double)beta * c;
                viol = fmax(viol, fabs(c));
            }
        const int nv = (k < N) ? 7 : 4;
        for (int i = 0; i < nv; ++i) {
            stat = fmax(stat, fabs(g[i]));
            if (!isfinite(g[i])) finite = false;
        }
    }
    Cert ct;
    ct.cost = warp_sum_d(cost);
    ct.viol = warp_max_d(viol);
    ct.stat = warp_max_d(stat);
    ct.finite = __all_sync(kFull, finite) && isfinite(ct.cost);
    return ct;
}

// FP64 residual of the step for one iterative-refinement pass:
//   res = g + (H + rho I) dz
// with g the AL gradient and H the local model that was factored (the
// Gauss-Newton part, plus the dynamics curvature when `curvature`), per
// variable into S.gr (x_k at 7k .. 7k+3, u_k at 7k+4 .. 7k+6).
__device__ void residual_fp64(Ctx& C, float beta_f, float rho_f, bool curvature) {
    const DevInstance& P = *C.P;
    const int N = C.N, Np1 = C.N + 1, lane = C.lane;
    Smem& S = C.sm;
    const double beta = beta_f, rho = rho_f;
    for (int k = lane; k <= N; k += 32) {
        double res[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int side = 0; side < 2; ++side) {
            const int kk = (side == 0) ? k - 1 : k;
            if (kk < 0 || kk >= N) continue;
            Rows64 R;
            rows_fp64(C, kk, R);
            double dl[11];
            for (int i = 0; i < 4; ++i) {
                dl[i] = S.dz[7 * kk + i];
                dl[7 + i] = S.dz[7 * (kk + 1) + i];
            }
            for (int j = 0; j < 3; ++j) dl[4 + j] = S.dz[7 * kk + 4 + j];
            const float* lam = S.lam + 3 + 11 * kk;
            for (int r = 0; r < 11; ++r) {
                if (!R.on[r]) continue;
                const bool ineq = r >= 5;
                const double t = (double)lam[r] + beta * R.c[r];
                if (ineq && !(t > 0.0)) continue;
                double adz = 0.0;
                for (int j = 0; j < 11; ++j) adz += R.J[r][j] * dl[j];
                const double w = t + beta * adz;  // y_r + beta a_r . dz
                if (side == 0)
                    for (int i = 0; i < 4; ++i) res[i] += w * R.J[r][7 + i];
                else
                    for (int i = 0; i < 7; ++i) res[i] += w * R.J[r][i];
            }
            if (side == 0) {
                for (int i = 0; i < 4; ++i) res[i] += rho * dl[7 + i];  // damping of x_{k+1}
            } else {
                for (int j = 0; j < 3; ++j) res[4 + j] += 2.0 * P.w_control_d * (R.u[j] + dl[4 + j]) + rho * dl[4 + j];
                if (curvature) {
                    // -dt sum_r yd_r d^2 f_r over (x_k, u_k), yd the unscaled multipliers
                    double yd[3];
                    for (int r = 0; r < 3; ++r) {
                        const double t = (double)lam[r] + beta * R.c[r];
                        yd[r] = R.on[r] ? t / P.sigma_d[r] : 0.0;
                    }
                    const ModeInfo mi = mode_of(S.mb[kk]);
                    const double nx = (mi.face == 0) ? 1.0 : ((mi.face == 2) ? -1.0 : 0.0);
                    const double ny = (mi.face == 1) ? 1.0 : ((mi.face == 3) ? -1.0 : 0.0);
                    const double tx = -ny, ty = nx, kp = R.kf, dt = P.dt_d;  // kf = 0 in free motion
                    const double h_thth = -yd[0] * R.f0 - yd[1] * R.f1;
                    const double h_thfn = yd[0] * kp * (-R.st * nx - R.ct * ny) + yd[1] * kp * (R.ct * nx - R.st * ny);
                    const double h_thft = yd[0] * kp * (-R.st * tx - R.ct * ty) + yd[1] * kp * (R.ct * tx - R.st * ty);
                    const double h_sfn = -yd[2] * kp * P.inv_c2_d;
                    res[2] -= dt * (h_thth * dl[2] + h_thfn * dl[4] + h_thft * dl[5]);
                    res[4] -= dt * (h_thfn * dl[2] + h_sfn * dl[3]);
                    res[5] -= dt * h_thft * dl[2];
                    res[3] -= dt * h_sfn * dl[4];
                }
            }
        }
        if (k == N)
            for (int i = 0; i < 3; ++i) {
                const double e = (double)S.xh[i * Np1 + N] + (double)S.xl[i * Np1 + N] - P.goal_d[i];
                res[i] += 2.0 * P.w_terminal_d * (e + (double)S.dz[7 * N + i]);
            }
        if (k == 0) {
            for (int i = 0; i < 3; ++i) {
                const double c = (double)S.xh[i * Np1] + (double)S.xl[i * Np1] - P.start_d[i];
                res[i] += (double)S.lam[i] + beta * (c + (double)S.dz[i]);
            }
            for (int i = 0; i < 4; ++i) res[i] += rho * (double)S.dz[i];
        }
        const int nv = (k < N) ? 7 : 4;
        for (int i = 0; i < nv; ++i) S.gr[7 * k + i] = (float)res[i];
    }
    __syncwarp();
}

// One step of iterative refinement of the Riccati solve (at high penalty):
// the FP64 residual res = g + (H + rho I) dz of the FP32 step is solved
// with the same model (same factorisation path) and the correction added,
// dz <- dz + delta with (H + rho I) delta = -res.  Once the records hold
// the residual, sm.gr is free and keeps the first step meanwhile.
template <bool kFree>
__device__ void refine_step(Ctx& C, float beta, float rho, bool curvature) {
    Smem& S = C.sm;
    const int nz = 7 * C.N + 4;
    residual_fp64(C, beta, rho, curvature);
    phase_a<kFree>(C, beta, rho, curvature, true, false, beta, /*rhs_from_gr=*/true);
    for (int t = C.lane; t < nz; t += 32) S.gr[t] = S.dz[t];
    __syncwarp();
    if (phase_b(C, beta, rho, /*rhs_from_gr=*/true)) {
        phase_c(C);
        for (int t = C.lane; t < nz; t += 32) S.dz[t] += S.gr[t];
    } else {
        for (int t = C.lane; t < nz; t += 32) S.dz[t] = S.gr[t];
    }
    __syncwarp();
}

// ------------------------------------------------------------------ kernel

// kRefine: the variant with the FP64 refinement step compiled in; the
// launch picks it only when the penalty can exceed refine_beta, so the
// default kernel carries none of that code (a smaller instruction footprint).
// At most 3 resident CTAs of 4 warps per SM: the register cap is then 168,
// where the elimination of phase B and the assembly of phase A run without
// most of the local-memory spills a 128-register cap costs (12 warps per SM
// at 168 registers were 7 % faster than 16 at 128 on the 4-segment
// enumeration, with DRAM write-back 7 times lower).
// kUnr: stages per trip of the stage-parallel loops (phases A, C and D
// unrolled 1 or 2 times; the autotuner picks it with the launch shape).
template <bool kRefine, bool kFree, int kUnr = 1>
__global__ void __launch_bounds__(128, 3) eval_kernel(EvalArgs A) {
    extern __shared__ float smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int warp_global = blockIdx.x * (blockDim.x >> 5) + wib;
    const size_t per_warp = smem_floats(A.Nmax);
    Ctx C;
    C.lane = lane;
    C.Nmax = A.Nmax;
    C.sm = carve(smem_raw + per_warp * wib, A.Nmax);
    C.rec = A.ws + (size_t)warp_global * A.ws_per_warp;
    const SolverParams& sp = A.sp;
    const int64_t n_tos = A.d_n ? min(*A.d_n, A.n) : A.n;
    const uint32_t wbar = ek_smem_u32(C.sm.mbar);
    uint32_t wphase = 0;  // parity of the warp's next staging phase
    if (A.warm) {
        if (lane == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(wbar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncwarp();
    }

    for (;;) {
        unsigned int t = 0;
        if (lane == 0) t = atomicAdd(A.queue, 1u);
        t = __shfl_sync(kFull, t, 0);
        if ((int64_t)t >= n_tos) break;
        const int64_t ti = A.perm ? (int64_t)A.perm[t] : (int64_t)t;
        // ---- load the order and validate it
        const comet_mode_seq sq = A.seqs[ti];
        bool bad = sq.instance < 0 || sq.instance >= A.n_inst;
        const DevInstance* P = bad ? A.inst : A.inst + sq.instance;
        const int len = sq.len;
        bad = bad || len < 1 || len > P->Lmax || len > COMET_MAX_SEGMENTS;
        if (!bad)
            for (int i = 0; i < len; ++i) bad = bad || sq.modes[i] >= P->n_modes;
        if (bad) {
            if (lane == 0) {
                atomicExch(A.bad_input, 1);
                A.out_status[ti] = COMET_TO_NONFINITE;
                A.out_cost[ti] = __int_as_float(0x7fc00000);
                if (A.out_iters) A.out_iters[ti] = 0;
                if (A.out_viol) A.out_viol[ti] = __int_as_float(0x7fc00000);
                if (A.out_merit) A.out_merit[ti] = __int_as_float(0x7fc00000);
                if (A.out_stat) A.out_stat[ti] = __int_as_float(0x7fc00000);
            }
            continue;
        }
        C.P = P;
        C.len = len;
        C.N = P->K * len;
        for (int i = 0; i < COMET_MAX_SEGMENTS; ++i) C.modes[i] = sq.modes[i];
        const int N = C.N, Np1 = N + 1;
        Smem& S = C.sm;
        // ---- initial iterate: warm start or the cold start
        const float* warm = A.warm ? A.warm + ti * A.stride : nullptr;
        const int Nm1 = A.Nmax + 1;
        if (warm) {
            // stage the record in the step / gradient buffers (free until
            // the first iteration): float j at stg[j], with stg congruent to
            // the record modulo 16 bytes, so that its 16-byte aligned
            // interior arrives by one bulk copy; the head and tail (at most
            // 3 floats each) by plain loads
            const uintptr_t src = reinterpret_cast<uintptr_t>(warm);
            const int nrec = (int)A.stride;
            const uintptr_t a0 = (src + 15) & ~(uintptr_t)15, a1 = (src + 4 * (uintptr_t)nrec) & ~(uintptr_t)15;
            const bool bulk = a1 > a0;
            float* stg = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(S.dz) + 15) & ~(uintptr_t)15) +
                         ((src & 15) >> 2);
            const int h_end = bulk ? (int)((a0 - src) >> 2) : nrec, t_begin = bulk ? (int)((a1 - src) >> 2) : nrec;
            __syncwarp();
            if (bulk && lane == 0 && !A.stall_staging)
                ek_bulk_copy(ek_smem_u32(stg) + (uint32_t)(a0 - src), reinterpret_cast<const void*>(a0),
                             (uint32_t)(a1 - a0), wbar);
            for (int j = lane; j < h_end; j += 32) stg[j] = warm[j];
            for (int j = t_begin + lane; j < nrec; j += 32) stg[j] = warm[j];
            bool ok = true;
            if (bulk) {
                ok = ek_mbar_wait(wbar, wphase);
                wphase ^= 1u;
            }
            if (!__all_sync(kFull, ok)) {
                // the copy did not complete: flag it, give the copy a second
                // bounded wait, and leave
                if (lane == 0) {
                    atomicExch(A.bad_input, 2);
                    A.out_status[ti] = COMET_TO_NONFINITE;
                    A.out_cost[ti] = __int_as_float(0x7fc00000);
                }
                ek_mbar_wait(wbar, wphase ^ 1u);
                return;
            }
            __syncwarp();
            warm = stg;
        }
        for (int q = lane; q < 4 * Np1; q += 32) {
            const int i = q / Np1, k = q - i * Np1;
            float x;
            if (warm) {
                x = warm[i * Nm1 + k];
            } else if (i < 3) {
                const float al = (float)k / (float)N;
                x = (1.f - al) * P->start[i] + al * P->goal[i];
            } else {
                x = 0.f;
            }
            S.xh[q] = x;
            S.xl[q] = 0.f;
        }
        for (int q = lane; q < 3 * N; q += 32) {
            const int j = q / N, k = q - j * N;
            S.us[q] = warm ? warm[4 * Nm1 + j * A.Nmax + k] : 0.f;
        }
        for (int q = lane; q < 3 + 11 * N; q += 32) S.lam[q] = 0.f;
        for (int k = lane; k < N; k += 32) {
            const ModeInfo mi = mode_info(C.modes, len, N, k);
            S.mb[k] = (unsigned char)(mi.face | (mi.kind << 2) | ((mi.smask ? 1 : 0) << 4));
        }
        __syncwarp();

        float beta = sp.beta0, rho = sp.rho0, eta = INFINITY;
        int inner = 0, it = 0, status = COMET_TO_MAX_ITER, curv_hold = 0;
        bool nonfinite = false;
        for (it = 0; it < sp.max_iters; ++it) {
            const bool curv = curv_hold == 0;
            if (!curv) --curv_hold;
            // One iteration is a sequence of (assemble, sweep) trips through a
            // single call site of each phase (one inlined copy of the largest
            // code in the hot loop):
            //   MEASURE  the measures and the model at the current iterate;
            //   UPDATE   after a solved subproblem: dual update at beta_old,
            //            then the model at the new (lam, beta);
            //   RETRY    Gauss-Newton reassembly after a failed sweep.
            // The step model is Newton with the dynamics curvature, then
            // Gauss-Newton with the same damping, then rising damping.
            enum { kMeasure, kUpdate, kRetry };
            int trip = kMeasure, retries = 0;
            bool model_curv = curv, fac = false, done = false;
            float beta_old = beta;
            for (;;) {
                const Measures m = phase_a<kFree, kUnr>(C, beta, rho, model_curv, true, trip == kUpdate, beta_old);
                if (trip == kMeasure) {
                    if (!m.finite) {
                        status = COMET_TO_NONFINITE;
                        nonfinite = true;
                        done = true;
                        break;
                    }
                    // stop test (Sec. III-C): scaled rows within eps_primal,
                    // rows in physical units within half eps_feas, and
                    // stationarity relative to max(1, |J|)
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
                fac = phase_b(C, beta, rho);
                if (fac) break;
                if (model_curv) {
                    // indefinite with the curvature: Gauss-Newton for the next
                    // curv_skip iterations, starting now at the same damping
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
            const float D = phase_c<kUnr>(C);
            if (kRefine && beta > sp.refine_beta) refine_step<kFree>(C, beta, rho, model_curv);
            const float alpha = phase_d<kFree, kUnr>(C, beta, D, sp);
            if (alpha > 0.f) {
                phase_e(C, alpha);
                rho = fmaxf(sp.rho_min, rho / 10.f);
            } else {
                rho = fminf(sp.rho_max, rho * 10.f);
            }
        }
        // ---- FP64 certificate and outputs
        const Cert ct = certify(C, beta);
        if (!ct.finite) nonfinite = true;
        if (nonfinite) status = COMET_TO_NONFINITE;
        if (status == COMET_TO_CONVERGED && !(ct.viol <= sp.eps_feas)) status = COMET_TO_INFEASIBLE;
        if (lane == 0) {
            A.out_status[ti] = status;
            A.out_cost[ti] = (float)ct.cost;
            if (A.out_viol) A.out_viol[ti] = (float)ct.viol;
            if (A.out_merit) A.out_merit[ti] = (float)(ct.cost + sp.merit_mu * fmax(ct.viol - sp.eps_feas, 0.0));
            if (A.out_iters) A.out_iters[ti] = it;
            if (A.out_stat) A.out_stat[ti] = (float)ct.stat;
        }
        if (A.out_traj) {
            float* out = A.out_traj + ti * A.stride;
            for (int q = lane; q < 4 * Nm1; q += 32) {
                const int i = q / Nm1, k = q - i * Nm1;
                out[q] = (k <= N) ? S.xh[i * Np1 + k] + S.xl[i * Np1 + k] : 0.f;
            }
            for (int q = lane; q < 3 * A.Nmax; q += 32) {
                const int j = q / A.Nmax, k = q - j * A.Nmax;
                out[4 * Nm1 + q] = (k < N) ? S.us[j * N + k] : 0.f;
            }
        }
        __syncwarp();
    }
}

}  // namespace

size_t smem_per_warp_bytes(int Nmax) { return smem_floats(Nmax) * sizeof(float); }

namespace {
// every instantiation of the evaluator: (refinement, free motion, unroll;
// the refinement variants run unrolled once)
cudaError_t set_smem_all(size_t smem) {
    const int b = (int)smem;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(eval_kernel<false, false, 1>, at, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eval_kernel<true, false, 1>, at, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eval_kernel<false, true, 1>, at, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eval_kernel<true, true, 1>, at, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eval_kernel<false, false, 2>, at, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eval_kernel<false, true, 2>, at, b);
    return e;
}
}  // namespace

int eval_blocks_per_sm(int warps_per_block, size_t smem_per_block) {
    int nb = 0;
    if (set_smem_all(smem_per_block) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    // the variants share the register cap and shared memory, so one
    // occupancy query serves all
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eval_kernel<false, false, 1>, warps_per_block * 32,
                                                      smem_per_block) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_eval(const EvalArgs& a, int total_warps, int warps_per_block, cudaStream_t s) {
    const size_t smem = smem_per_warp_bytes(a.Nmax) * warps_per_block;
    // the attribute is raised to the largest size seen on this device; it is
    // not a stream operation, so raising it outside of a capture keeps
    // launches capturable (problem creation raises it first)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static size_t raised[64] = {};
    if (dev < 64 && raised[dev] < smem) {
        e = set_smem_all(smem);
        if (e != cudaSuccess) return e;
        raised[dev] = smem;
    }
    const int blocks = (total_warps + warps_per_block - 1) / warps_per_block;
    const bool refine = a.sp.refine && a.sp.refine_beta < a.sp.beta_max;
    const bool unr2 = a.unroll == 2 && !refine;
    const unsigned threads = warps_per_block * 32;
    if (a.sp.free_motion) {
        if (refine)
            eval_kernel<true, true, 1><<<blocks, threads, smem, s>>>(a);
        else if (unr2)
            eval_kernel<false, true, 2><<<blocks, threads, smem, s>>>(a);
        else
            eval_kernel<false, true, 1><<<blocks, threads, smem, s>>>(a);
    } else {
        if (refine)
            eval_kernel<true, false, 1><<<blocks, threads, smem, s>>>(a);
        else if (unr2)
            eval_kernel<false, false, 2><<<blocks, threads, smem, s>>>(a);
        else
            eval_kernel<false, false, 1><<<blocks, threads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace comet
