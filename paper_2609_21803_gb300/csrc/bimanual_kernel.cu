// bimanual_kernel.cu -- persistent evaluator of the bimanual variant: a box
// in the vertical plane flipped by two point hands on a ground contact
// (state x, z, theta, s_L, s_R; control twist, hand forces and sliding
// rates, ground force and centre of pressure; 507 modes = 3 ground x 13 x 13
// hand modes), one CTA of 128 threads per TO.
//
// The solver is the method of Sec. III-C with the Gauss-Newton model (the
// same steps as the pushing evaluator): PHR augmented Lagrangian, a
// backward sweep over w_k = (u_k, x_{k+1}) (17 x 17 S_k, Cholesky without
// pivoting, damping retries), trial steps alpha = 2^-i with the Armijo test,
// multiplier / penalty updates, the KKT stop test, and an FP64 certificate
// of v_hat (Eq. inexact_mode_value) and the KKT residual.
//
// Work per iteration:
//   A  a warp per stage, a lane per constraint row (32 rows): rows and their
//      Jacobians from one stage context; the AL model over (u, x_{k+1}, x_k)
//      built in registers, a model row per lane, from each row's nonzero
//      pattern; the 12 u columns eliminated there (shuffles for the pivot
//      column); records to the CTA's workspace (L2-resident)
//   B  one warp: the sequential sweep eliminating the 5 x_{k+1} columns, the
//      next stage's record prefetched into registers
//   gains and control steps stage-parallel, the forward chain on 5 lanes
//   D  8 trial steps x stages over all threads, sums in shared memory
//   E  compensated state update

#include <cuda_runtime.h>
#include <cuda/annotated_ptr>
#include <math.h>
#include <stdint.h>

#include "comet.h"
#include "comet_internal.h"

namespace comet {
namespace {

constexpr unsigned kFullB = 0xffffffffu;
constexpr int NX = 5, NU = 12, NR = 32, NL = 22, NWV = 17;
constexpr int NE = 23;               // elimination order (u 12, y 5, x 5, rhs)
constexpr int NRED = 11;             // reduced block (y 5, x 5, rhs)
constexpr int NTRI_RED = NRED * (NRED + 1) / 2;  // 66
// record layout (floats)
constexpr int R_LUU = 0;     // 78: u-block factor, lower triangle
constexpr int R_CPL = 78;    // 132: coupling rows (y, x, rhs) x 12 u columns
constexpr int R_PD = 210;    // u-block pivots positive
constexpr int R_RED = 212;   // 66: reduced (y, x, rhs) block
constexpr int R_YF = 280;    // 15 + 30 raw y-factor (+3 pad), then 30 gains
static_assert(R_YF + 48 <= kBimRec, "record layout");
static_assert(R_YF % 4 == 0 && kBimRec % 4 == 0, "vector access to the raw factor");
// sweep copy ring: record floats 208..279 (the u-block flag at 210, the
// reduced block at 212..277), kBRing stages ahead
constexpr int R_SLOT = 208, kBSlot = 72, kBRing = 6;
static_assert(R_SLOT + 2 == R_PD && R_SLOT + 4 == R_RED && R_SLOT + kBSlot >= R_RED + NTRI_RED, "ring slot");

// local variables: x_k 0..4, u_k 5..16, x_{k+1} 17..21
enum { VX = 0, VZ, VTH, VSL, VSR, UXD, UZD, UTHD, UFNL, UFTL, USDL, UFNR, UFTR, USDR, ULN, ULT, UPC, VX1 };

__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// asynchronous global -> shared copies of 16 bytes with commit groups (the
// waits are hardware waits on the issuing thread's own groups)
__device__ __forceinline__ void bcp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void bcp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bcp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bcp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// reciprocal from the SFU (rcp.approx, about 1 ulp); the damped pivots are
// never subnormal
__device__ __forceinline__ float brcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// elimination position of local variable v; rhs = 22
__host__ __device__ constexpr int epos(int v) { return v >= 17 ? v - 5 : (v >= 5 ? v - 5 : v + 17); }
// local variable of elimination position e (e < 22)
__host__ __device__ constexpr int evar(int e) { return e < 17 ? e + 5 : e - 17; }


template <typename T>
struct BInst {
    T ax, az, mg, lbar, mu_g, mu_h, cg, ch, dt;
    T start[3], goal[3];
    T wT, wc, wf;  // control weights: wc (twist, sliding rates, p_c), wf (forces)
    int K;
};

// weight of control j (forces: f_n, f_t of both hands, lam_n, lam_t)
template <typename T>
__device__ __forceinline__ T rweight(const BInst<T>& P, int j) {
    return (j == 3 || j == 4 || j == 6 || j == 7 || j == 9 || j == 10) ? P.wf : P.wc;
}

template <typename T>
__device__ void load_inst(const DevInstance& d, BInst<T>& P) {
    const bool dbl = sizeof(T) == 8;
    P.ax = dbl ? (T)d.a_d[0] : (T)d.a[0];
    P.az = dbl ? (T)d.a_d[1] : (T)d.a[1];
    const T mass = dbl ? (T)d.mass_d : (T)d.mass;
    P.mg = mass * (T)9.81;
    P.lbar = P.ax > P.az ? P.ax : P.az;
    P.mu_g = dbl ? (T)d.ground_mu_d : (T)d.ground_mu;
    P.mu_h = dbl ? (T)d.mu_d : (T)d.mu;
    P.cg = sqrt(1 + P.mu_g * P.mu_g);
    P.ch = sqrt(1 + P.mu_h * P.mu_h);
    P.dt = dbl ? (T)d.dt_d : (T)d.dt;
    for (int i = 0; i < 3; ++i) {
        P.start[i] = dbl ? (T)d.start_d[i] : (T)d.start[i];
        P.goal[i] = dbl ? (T)d.goal_d[i] : (T)d.goal[i];
    }
    P.wT = dbl ? (T)d.w_terminal_d : (T)d.w_terminal;
    const T wc = dbl ? (T)d.w_control_d : (T)d.w_control;
    P.wc = wc;
    P.wf = wc / (P.mg * P.mg);
    P.K = d.K;
}

// per-stage quantities shared by the rows
template <typename T>
struct BStage {
    T cth, sth;
    int g, h[2];
    T n[2][2], t[2][2], a[2], ell[2];
    T Fwx, Fwz, tau;      // wrench sums (without gravity's force)
    T rcx, rcz, w, dw;    // pivot corner offset, support half-width
};

template <typename T>
__device__ void stage_ctx(const BInst<T>& P, int mode, const T* x, const T* u, BStage<T>& S) {
    S.g = mode / 169;
    S.h[0] = (mode / 13) % 13;
    S.h[1] = mode % 13;
    const T th = x[VTH];
    if (sizeof(T) == 8) {
        double s, c;
        sincos((double)th, &s, &c);
        S.cth = (T)c;
        S.sth = (T)s;
    } else {
        float s, c;
        sincosf((float)th, &s, &c);
        S.cth = (T)c;
        S.sth = (T)s;
    }
    const T cth = S.cth, sth = S.sth;
    S.Fwx = u[ULT - 5];
    S.Fwz = u[ULN - 5];
    S.tau = u[UPC - 5] * u[ULN - 5] + x[VZ] * u[ULT - 5];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int h = S.h[side];
        const int f = h == 0 ? 0 : (h - 1) / 3;
        const T nx = (f == 0) ? (T)1 : ((f == 2) ? (T)-1 : (T)0);
        const T nz = (f == 1) ? (T)1 : ((f == 3) ? (T)-1 : (T)0);
        S.n[side][0] = nx;
        S.n[side][1] = nz;
        S.t[side][0] = -nz;
        S.t[side][1] = nx;
        S.a[side] = (f % 2 == 0) ? P.ax : P.az;
        S.ell[side] = (f % 2 == 0) ? P.az : P.ax;
        if (h == 0) continue;
        const T fn = u[(side ? UFNR : UFNL) - 5], ft = u[(side ? UFTR : UFTL) - 5];
        const T s = x[side ? VSR : VSL];
        const T bx = fn * nx + ft * (-nz), bz = fn * nz + ft * nx;
        S.Fwx += cth * bx - sth * bz;
        S.Fwz += sth * bx + cth * bz;
        S.tau += -S.a[side] * ft - s * fn;
    }
    S.rcx = -P.ax * cth + P.az * sth;
    S.rcz = -P.ax * sth - P.az * cth;
    S.w = P.ax * cth * cth + P.az * sth * sth;
    S.dw = 2 * sth * cth * (P.az - P.ax);
}

// hand rows of one side (q = 0..7): force, sliding rate and offset
__host__ __device__ constexpr int bnz_hand(bool right, int q, int a) {
    return (q == 0 || q == 3) ? (a == 0 ? (right ? UFNR : UFNL) : a == 1 ? (right ? UFTR : UFTL)
                                 : a == 2 ? (right ? USDR : USDL) : -1)
         : q == 1 ? (a == 0 ? (right ? UFTR : UFTL) : -1)
         : q == 2 ? (a == 0 ? (right ? USDR : USDL) : -1)
         : q == 4 ? (a == 0 ? (right ? UFNR : UFNL) : a == 1 ? (right ? UFTR : UFTL) : -1)
         : q == 5 ? (a == 0 ? (right ? UFNR : UFNL) : -1)
                  : (a == 0 ? (right ? VSR : VSL) : -1);
}

// Local variables that row r can depend on, over all modes (a superset of
// the nonzeros brow writes), ascending; -1 pads.  Kinematic rows: x_k,r,
// the rate and x_{k+1},r; wrench rows: the force components, the angle and
// (torque) z, the hands' offsets and the centre of pressure; ground rows:
// the twist, the ground force and p_c, the angle where the pivot enters;
// hand rows: that hand's force, sliding rate and offset.
__host__ __device__ constexpr int bnz(int r, int a) {
    return r < 5 ? (a == 0 ? r : a == 1 ? (r < 3 ? UXD + r : (r == 3 ? USDL : USDR)) : a == 2 ? VX1 + r : -1)
         : r == 5 ? (a == 0 ? VTH : a == 1 ? UFNL : a == 2 ? UFTL : a == 3 ? UFNR : a == 4 ? UFTR : a == 5 ? ULT : -1)
         : r == 6 ? (a == 0 ? VTH : a == 1 ? UFNL : a == 2 ? UFTL : a == 3 ? UFNR : a == 4 ? UFTR : a == 5 ? ULN : -1)
         : r == 7 ? (a == 0 ? VZ : a == 1 ? VSL : a == 2 ? VSR : a == 3 ? UFNL : a == 4 ? UFTL : a == 5 ? UFNR
                     : a == 6 ? UFTR : a == 7 ? ULN : a == 8 ? ULT : a == 9 ? UPC : -1)
         : r == 8 ? (a == 0 ? VTH : a == 1 ? UXD : a == 2 ? UZD : a == 3 ? UTHD : -1)
         : r == 9 ? (a == 0 ? VTH : a == 1 ? UZD : a == 2 ? UTHD : -1)
         : r == 10 ? (a == 0 ? VTH : a == 1 ? UTHD : a == 2 ? ULN : a == 3 ? ULT : a == 4 ? UPC : -1)
         : r == 11 ? (a == 0 ? UXD : a == 1 ? ULN : a == 2 ? ULT : -1)
         : r == 12 ? (a == 0 ? ULN : a == 1 ? ULT : -1)
         : r == 13 ? (a == 0 ? ULN : -1)
         : r <= 15 ? (a == 0 ? VTH : a == 1 ? UPC : -1)
         : bnz_hand(r >= 24, r - (r >= 24 ? 24 : 16), a);
}

// Row r of an interval: scaled value c, presence, inequality flag, the
// physical factor (physical = c / scale) and, with WJ, the Jacobian over the
// 22 local variables.  dx = x_{k+1} - x_k (kinematic rows; computed from the
// compensated states by the caller).
template <typename T, bool WJ>
__device__ void brow(int r, const BInst<T>& P, const BStage<T>& S, bool mL, bool mR, const T* x, const T* u,
                     const T* dx, T& c, T* J, bool& on, bool& ineq, T& scale) {
    // internally the force rows are divided by m g and the torque row by
    // m g l; scale maps a row back to physical units (physical = c / scale:
    // N, N m, W, m, m/s), as v_hat is scored (Sec. III-C "Stopping and
    // scoring")
    c = 0;
    on = true;
    ineq = (r >= 11 && r <= 15) || (r >= 19 && r <= 23) || (r >= 27);
    scale = 1;
    if (WJ)
        for (int j = 0; j < NL; ++j) J[j] = 0;
    const T mg = P.mg;
    if (r < 5) {
        const int vel = (r < 3) ? UXD + r : (r == 3 ? USDL : USDR);
        const T dxr = (r == 0) ? dx[0] : (r == 1) ? dx[1] : (r == 2) ? dx[2] : (r == 3) ? dx[3] : dx[4];
        const T ur = (r == 0) ? u[0] : (r == 1) ? u[1] : (r == 2) ? u[2] : (r == 3) ? u[USDL - 5] : u[USDR - 5];
        c = dxr - P.dt * ur;
        if (WJ) {
            J[r] = -1;
            J[VX1 + r] = 1;
            J[vel] = -P.dt;
        }
        if ((r == 3 && mL) || (r == 4 && mR)) on = false;
    } else if (r < 8) {
        const T sc = (r == 7) ? 1 / (mg * P.lbar) : 1 / mg;
        scale = sc;
        if (r == 5) c = S.Fwx * sc;
        if (r == 6) c = (S.Fwz - mg) * sc;
        if (r == 7) c = S.tau * sc;
        if (WJ) {
            const T cth = S.cth, sth = S.sth;
            if (r == 5) J[ULT] = sc;
            if (r == 6) J[ULN] = sc;
            if (r == 7) {
                J[UPC] = u[ULN - 5] * sc;
                J[ULN] = u[UPC - 5] * sc;
                J[VZ] = u[ULT - 5] * sc;
                J[ULT] = x[VZ] * sc;
            }
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                if (S.h[side] == 0) continue;
                const int ufn = side ? UFNR : UFNL, uft = side ? UFTR : UFTL, vs = side ? VSR : VSL;
                const T nx = S.n[side][0], nz = S.n[side][1], tx = S.t[side][0], tz = S.t[side][1];
                const T fn = u[ufn - 5], ft = u[uft - 5];
                const T bx = fn * nx + ft * tx, bz = fn * nz + ft * tz;
                const T wx = cth * bx - sth * bz, wz = sth * bx + cth * bz;
                if (r == 5) {
                    J[VTH] += -wz * sc;
                    J[ufn] = (cth * nx - sth * nz) * sc;
                    J[uft] = (cth * tx - sth * tz) * sc;
                } else if (r == 6) {
                    J[VTH] += wx * sc;
                    J[ufn] = (sth * nx + cth * nz) * sc;
                    J[uft] = (sth * tx + cth * tz) * sc;
                } else {
                    J[uft] = -S.a[side] * sc;
                    J[ufn] = -(side ? x[VSR] : x[VSL]) * sc;
                    J[vs] = -fn * sc;
                }
            }
        }
    } else if (r < 16) {
        const T xd = u[0], zd = u[1], thd = u[2], ln = u[ULN - 5], lt = u[ULT - 5], pc = u[UPC - 5];
        const T mu = P.mu_g;
        if (r == 8) {
            if (S.g == 0) {
                c = xd;
                if (WJ) J[UXD] = 1;
            } else if (S.g == 1) {
                c = zd;
                if (WJ) J[UZD] = 1;
            } else {
                c = xd - thd * S.rcz;
                if (WJ) {
                    J[UXD] = 1;
                    J[UTHD] = -S.rcz;
                    J[VTH] = -thd * S.rcx;
                }
            }
        } else if (r == 9) {
            if (S.g == 0) {
                c = zd;
                if (WJ) J[UZD] = 1;
            } else if (S.g == 1) {
                c = thd;
                if (WJ) J[UTHD] = 1;
            } else {
                c = zd + thd * S.rcx;
                if (WJ) {
                    J[UZD] = 1;
                    J[UTHD] = S.rcx;
                    J[VTH] = -thd * S.rcz;
                }
            }
        } else if (r == 10) {
            if (S.g == 0) {
                c = thd;
                if (WJ) J[UTHD] = 1;
            } else if (S.g == 1) {
                const T s2 = 1 / (mg * mg);
                // factored, so that the difference near the edge is formed
                // before the product (no cancellation of two squares)
                c = ((lt - mu * ln) * (lt + mu * ln)) * s2;
                // physical: the friction force's distance from the cone
                // edge, |lam_t| - mu |lam_n| [N]
                const T den = fabs(lt) + mu * fabs(ln);
                scale = den > (T)0 ? den * s2 : (T)1;
                if (WJ) {
                    J[ULT] = 2 * lt * s2;
                    J[ULN] = -2 * mu * mu * ln * s2;
                }
            } else {
                c = pc - S.rcx;
                if (WJ) {
                    J[UPC] = 1;
                    J[VTH] = S.rcz;
                }
            }
        } else if (r == 11 || r == 12) {
            if (S.g != 1) {
                const T sc = 1 / (mg * P.cg), sg = (r == 11) ? (T)1 : (T)-1;
                scale = sc;
                c = (sg * lt - mu * ln) * sc;
                if (WJ) {
                    J[ULT] = sg * sc;
                    J[ULN] = -mu * sc;
                }
            } else if (r == 11) {
                const T sc = 1 / mg;
                scale = sc;  // W
                c = lt * xd * sc;
                if (WJ) {
                    J[ULT] = xd * sc;
                    J[UXD] = lt * sc;
                }
            } else {
                on = false;
            }
        } else if (r == 13) {
            scale = 1 / mg;
            c = -ln / mg;
            if (WJ) J[ULN] = -1 / mg;
        } else {
            if (S.g == 2) {
                on = false;
            } else {
                const T sg = (r == 14) ? (T)1 : (T)-1;
                c = sg * pc - S.w;
                if (WJ) {
                    J[UPC] = sg;
                    J[VTH] = -S.dw;
                }
            }
        }
    } else {
        const bool side = r >= 24;
        const int q = r - (side ? 24 : 16);
        const int h = side ? S.h[1] : S.h[0];
        const int ufn = side ? UFNR : UFNL, uft = side ? UFTR : UFTL, usd = side ? USDR : USDL;
        const int vs = side ? VSR : VSL;
        const T fn = side ? u[UFNR - 5] : u[UFNL - 5], ft = side ? u[UFTR - 5] : u[UFTL - 5];
        const T sd = side ? u[USDR - 5] : u[USDL - 5], s = side ? x[VSR] : x[VSL];
        const T ell = side ? S.ell[1] : S.ell[0];
        if (h == 0) {
            if (q == 0) {
                scale = 1 / mg;
                c = fn / mg;
                if (WJ) J[ufn] = 1 / mg;
            } else if (q == 1) {
                scale = 1 / mg;
                c = ft / mg;
                if (WJ) J[uft] = 1 / mg;
            } else if (q == 2) {
                c = sd;
                if (WJ) J[usd] = 1;
            } else {
                on = false;
            }
        } else {
            const int kind = (h - 1) % 3;
            const T muh = P.mu_h, sch = 1 / (mg * P.ch);
            if (q == 1 || q == 2) {
                on = false;
            } else if (q == 0) {
                if (kind == 0) {
                    c = sd;
                    if (WJ) J[usd] = 1;
                } else {
                    const T sg = (kind == 1) ? (T)-1 : (T)1;
                    scale = sch;
                    c = (ft + sg * muh * fn) * sch;
                    if (WJ) {
                        J[uft] = sch;
                        J[ufn] = sg * muh * sch;
                    }
                }
            } else if (q == 3) {
                if (kind == 0) {
                    scale = sch;
                    c = (ft - muh * fn) * sch;
                    if (WJ) {
                        J[uft] = sch;
                        J[ufn] = -muh * sch;
                    }
                } else {
                    const T sg = (kind == 1) ? (T)-1 : (T)1;
                    c = sg * sd;
                    if (WJ) J[usd] = sg;
                }
            } else if (q == 4) {
                if (kind == 0) {
                    scale = sch;
                    c = (-ft - muh * fn) * sch;
                    if (WJ) {
                        J[uft] = -sch;
                        J[ufn] = -muh * sch;
                    }
                } else {
                    on = false;
                }
            } else if (q == 5) {
                scale = 1 / mg;
                c = -fn / mg;
                if (WJ) J[ufn] = -1 / mg;
            } else {
                const T sg = (q == 6) ? (T)1 : (T)-1;
                c = sg * s - ell;
                if (WJ) J[vs] = sg;
            }
        }
    }
    if (!on) {
        c = 0;
        if (WJ)
            for (int j = 0; j < NL; ++j) J[j] = 0;
    }
}

__device__ __forceinline__ float bwarp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFullB, v, o));
    return v;
}
__device__ __forceinline__ float bwarp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullB, v, o);
    return v;
}

__device__ __forceinline__ void two_sum_b(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

struct BSmem {
    float *xh, *xl, *us, *lam, *dz, *gr;
    int* mi;     // per interval: mode | maskL << 10 | maskR << 11
    float *Jw, *yw;       // per warp: [32][22], [32]
    float* ring;          // sweep copy ring [kBRing][kBSlot] (16-byte aligned)
    float* red;           // reductions / broadcasts [64]
};

__host__ __device__ inline size_t bsmem_floats(int Nmax) {
    const size_t f = (size_t)10 * (Nmax + 1) + (size_t)NU * Nmax + 3 + (size_t)NR * Nmax +
                     2 * ((size_t)NWV * Nmax + NX) + (size_t)Nmax + 4 * (NR * NL + NR) + kBRing * kBSlot + 64;
    return (f + 3) / 4 * 4;
}

__device__ BSmem bcarve(float* p, int Nmax) {
    BSmem s;
    s.ring = p; p += kBRing * kBSlot;  // first: 16-byte aligned
    s.xh = p; p += NX * (Nmax + 1);
    s.xl = p; p += NX * (Nmax + 1);
    s.us = p; p += NU * Nmax;
    s.lam = p; p += 3 + NR * Nmax;
    s.dz = p; p += NWV * Nmax + NX;
    s.gr = p; p += NWV * Nmax + NX;
    s.mi = reinterpret_cast<int*>(p); p += Nmax;
    s.Jw = p; p += 4 * NR * NL;
    s.yw = p; p += 4 * NR;
    s.red = p;
    return s;
}

struct BCtx {
    const DevInstance* D;
    BInst<float> P;
    BSmem S;
    float* rec;
    int N, Np1, len;
    int tid, warp, lane;
};

// compensated local variables of stage k at step alpha along dz
// (at alpha = 0 the step is not read: phase A runs before the first step of
// a TO exists, and its buffer also parks gradient parts during phase A)
__device__ __forceinline__ void load_stage(const BCtx& C, int k, float alpha, float* x, float* u, float* dx) {
    const int Np1 = C.Np1, N = C.N;
    const BSmem& S = C.S;
    const bool step = alpha != 0.f;
#pragma unroll
    for (int i = 0; i < NX; ++i) {
        const float h0 = S.xh[i * Np1 + k], h1 = S.xh[i * Np1 + k + 1];
        const float l0 = S.xl[i * Np1 + k] + (step ? alpha * S.dz[NWV * k + i] : 0.f);
        const float l1 = S.xl[i * Np1 + k + 1] + (step ? alpha * S.dz[NWV * (k + 1) + i] : 0.f);
        x[i] = h0 + l0;
        dx[i] = (h1 - h0) + (l1 - l0);
    }
#pragma unroll
    for (int j = 0; j < NU; ++j) u[j] = S.us[j * N + k] + (step ? alpha * S.dz[NWV * k + NX + j] : 0.f);
}

struct BMeasures {
    float viol, stat, comp;
    float vphys;  // violation in physical units (rows mapped back by c / scale)
    float cost;   // objective J at the iterate (scale of the stationarity test)
    bool finite;
};

// Phase A: rows, multipliers (PHR update at beta_old with `update`), the
// measures, the AL gradient into gr (x_{k+1} parts parked in dz), and, with
// `assemble`, the stage records (u block eliminated).
__device__ BMeasures bphase_a(BCtx& C, float beta, float rho, bool assemble, bool update, float beta_old) {
    BSmem& S = C.S;
    const BInst<float>& P = C.P;
    const int N = C.N, lane = C.lane, warp = C.warp;
    float* Jw = S.Jw + warp * NR * NL;
    float* yw = S.yw + warp * NR;
    float viol = 0.f, comp = 0.f, vph = 0.f, jc = 0.f;
    bool finite = true;
#pragma unroll 1
    for (int k = warp; k < N; k += 4) {
        float x[NX], u[NU], dx[NX];
        load_stage(C, k, 0.f, x, u, dx);
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < NU; ++j) jc += rweight(P, j) * u[j] * u[j];
        }
        const int mi = S.mi[k];
        BStage<float> St;
        stage_ctx(P, mi & 1023, x, u, St);
        // the row's Jacobian goes straight into its shared-memory row (a
        // register array indexed at run time would live in local memory)
        float* Jr = Jw + lane * NL;
        float c, sc;
        bool on, iq;
        brow<float, true>(lane, P, St, (mi >> 10) & 1, (mi >> 11) & 1, x, u, dx, c, Jr, on, iq, sc);
        float* lam = S.lam + 3 + NR * k;
        float l = lam[lane];
        if (update && on) {
            const float t = l + beta_old * c;
            l = iq ? fmaxf(t, 0.f) : t;
            lam[lane] = l;
        }
        const float t = l + beta * c;
        const bool act = on && (!iq || t > 0.f);
        const float y = act ? (iq ? fmaxf(t, 0.f) : t) : 0.f;
        if (on) {
            const float vr = iq ? fmaxf(c, 0.f) : fabsf(c);
            viol = fmaxf(viol, vr);
            vph = fmaxf(vph, vr / sc);
            if (iq) comp = fmaxf(comp, fabsf(y * c));
            if (!isfinite(c)) finite = false;
        }
        if (!act)
            for (int j = 0; j < NL; ++j) Jr[j] = 0.f;
        yw[lane] = y;
        __syncwarp();
        // AL gradient over the local variables (lane = variable)
        float gval = 0.f;
        if (lane < NL) {
            float g = 0.f;
            for (int r = 0; r < NR; ++r) g += yw[r] * Jw[r * NL + lane];
            if (lane >= 5 && lane < 17) g += 2.f * rweight(P, lane - 5) * S.us[(lane - 5) * N + k];
            if (lane < 17)
                S.gr[NWV * k + lane] = g;
            else
                S.dz[NWV * (k + 1) + lane - 17] = g;
            gval = g;
        }
        if (assemble) {
            // the model in registers, a row per lane: lane i < 22 holds row i
            // of the lower triangle over (u, y, x) in elimination order (and
            // lane 22 the rhs row).  Row i = sum_r J_r[v_i] J_r over the
            // active rows in row order; for row r only the columns of its
            // pattern (bnz) are added, the others being exact zeros: the
            // lane's own entry times a broadcast Jacobian value
            const int vi = lane < NL ? evar(lane) : 0;
            float row[NE];
#pragma unroll
            for (int cc = 0; cc < NE; ++cc) row[cc] = 0.f;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float a = lane < NL ? Jw[r * NL + vi] : 0.f;
#pragma unroll
                for (int q = 0; q < 10; ++q) {
                    if (bnz(r, q) < 0) break;
                    row[epos(bnz(r, q))] += a * Jw[r * NL + bnz(r, q)];
                }
            }
            // beta, then the cost and damping on the diagonal (u: cost +
            // rho, x_{k+1}: rho); the gradient as the rhs row (lane 22)
#pragma unroll
            for (int cc = 0; cc < NE - 1; ++cc) {
                row[cc] *= beta;
                if (lane == cc) {
                    if (cc < 12) row[cc] += 2.f * rweight(P, cc) + rho;
                    else if (cc < 17) row[cc] += rho;
                }
            }
#pragma unroll
            for (int cc = 0; cc < NE - 1; ++cc) {
                const float gv = __shfl_sync(kFullB, gval, evar(cc));
                if (lane == NE - 1) row[cc] = gv;
            }
            // eliminate the u block (12 Cholesky columns) in registers: lane
            // i < 23 holds row i of the lower triangle (entries 0..i); the
            // pivot comes from lane j and the column entry L_cj from lane c
            // by shuffles.  A non-positive pivot marks the record.
            bool pd = true;
#pragma unroll
            for (int j = 0; j < 12; ++j) {
                const float d = __shfl_sync(kFullB, row[j], j);
                pd = pd && (d > 0.f);
                const float l = sqrtf(fmaxf(d, 1e-30f));
                const float il = 1.f / l;
                if (lane == j) row[j] = l;
                if (lane > j) row[j] *= il;
#pragma unroll
                for (int cc = j + 1; cc < NE; ++cc) {
                    const float lcj = __shfl_sync(kFullB, row[j], cc);
                    if (lane >= cc) row[cc] -= row[j] * lcj;
                }
            }
            // records from the rows: the u factor (rows 0..11), the coupling
            // rows (12..22) x u columns, the reduced (y, x, rhs) block
            // record stores with the persisting (evict-last) L2 priority: the
            // CTAs' workspaces fit in L2 and are rewritten every iteration
            cuda::annotated_ptr<float, cuda::access_property::persisting> rec(C.rec + (size_t)k * kBimRec);
            if (lane < 12) {
#pragma unroll
                for (int cc = 0; cc < 12; ++cc)
                    if (cc <= lane) rec[R_LUU + tri(lane, cc)] = row[cc];
            } else if (lane < NE) {
                const int p = lane - 12;
#pragma unroll
                for (int cc = 0; cc < 12; ++cc) rec[R_CPL + 12 * p + cc] = row[cc];
#pragma unroll
                for (int cc = 12; cc < NE; ++cc)
                    if (cc <= lane) rec[R_RED + tri(p, cc - 12)] = row[cc];
            }
            if (lane == 0) rec[R_PD] = pd ? 1.f : -1.f;
        }
        __syncwarp();
    }
    __syncthreads();
    // initial pose rows and the combined gradient
    const int tid = C.tid, Np1 = C.Np1;
    float stat = 0.f;
    if (tid < 3) {
        float l = S.lam[tid];
        const float c = (S.xh[tid * Np1] - P.start[tid]) + S.xl[tid * Np1];
        if (update) {
            l = l + beta_old * c;
            S.lam[tid] = l;
        }
        viol = fmaxf(viol, fabsf(c));
        vph = fmaxf(vph, fabsf(c));
        if (!isfinite(c)) finite = false;
    }
    if (tid == 0)
        for (int i = 0; i < 3; ++i) {
            const float e = (S.xh[i * Np1 + N] - P.goal[i]) + S.xl[i * Np1 + N];
            jc += P.wT * e * e;
        }
    __syncthreads();
    for (int k = tid; k <= N; k += kBimThreads) {
        for (int i = 0; i < NX; ++i) {
            float g = (k < N) ? S.gr[NWV * k + i] : 0.f;
            if (k > 0) g += S.dz[NWV * k + i];
            if (k == N && i < 3) g += 2.f * P.wT * ((S.xh[i * Np1 + N] - P.goal[i]) + S.xl[i * Np1 + N]);
            if (k == 0 && i < 3) g += S.lam[i] + beta * ((S.xh[i * Np1] - P.start[i]) + S.xl[i * Np1]);
            S.gr[NWV * k + i] = g;
            stat = fmaxf(stat, fabsf(g));
            if (!isfinite(g)) finite = false;
        }
        if (k < N)
            for (int j = 0; j < NU; ++j) {
                const float g = S.gr[NWV * k + NX + j];
                stat = fmaxf(stat, fabsf(g));
                if (!isfinite(g)) finite = false;
            }
    }
    // block reductions
    viol = bwarp_max(viol);
    stat = bwarp_max(stat);
    comp = bwarp_max(comp);
    vph = bwarp_max(vph);
    jc = bwarp_sum(jc);
    const bool fin = __all_sync(kFullB, finite);
    __syncthreads();
    if (C.lane == 0) {
        S.red[C.warp] = viol;
        S.red[4 + C.warp] = stat;
        S.red[8 + C.warp] = comp;
        S.red[12 + C.warp] = fin ? 1.f : 0.f;
        S.red[24 + C.warp] = vph;
        S.red[28 + C.warp] = jc;
    }
    __syncthreads();
    BMeasures m;
    m.viol = fmaxf(fmaxf(S.red[0], S.red[1]), fmaxf(S.red[2], S.red[3]));
    m.stat = fmaxf(fmaxf(S.red[4], S.red[5]), fmaxf(S.red[6], S.red[7]));
    m.comp = fmaxf(fmaxf(S.red[8], S.red[9]), fmaxf(S.red[10], S.red[11]));
    m.finite = S.red[12] > 0.f && S.red[13] > 0.f && S.red[14] > 0.f && S.red[15] > 0.f;
    m.vphys = fmaxf(fmaxf(S.red[24], S.red[25]), fmaxf(S.red[26], S.red[27]));
    m.cost = (S.red[28] + S.red[29]) + (S.red[30] + S.red[31]);
    __syncthreads();
    return m;
}

// Sweep over k = N-1 .. 0 on warp 0.  Every lane runs the whole stage in
// registers (the sequential chain is short and dependent): the reduced
// 11 x 11 lower triangle (rows y 0..4, x 0..4, rhs) arrives from the record
// through a cp.async ring kBRing stages ahead and is read as shared-memory
// broadcasts, V_{k+1} and v_{k+1} stay in registers, the 5 y columns are
// eliminated with SFU reciprocal pivots, and lane 0 writes the raw y-factor
// columns (15 y-y entries, then the (x, rhs) rows) for the gains.  Then the
// x_0 block; publishes the factorisation status to all threads and dx0 into
// red[16..20].
__device__ bool bphase_b(BCtx& C, float beta, float rho) {
    BSmem& S = C.S;
    const BInst<float>& P = C.P;
    const int N = C.N, Np1 = C.Np1, lane = C.lane;
    if (C.warp == 0) {
        float V[15], v[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
#pragma unroll
            for (int j = 0; j <= i; ++j) V[tri(i, j)] = (i == j && i < 3) ? 2.f * P.wT : 0.f;
            v[i] = i < 3 ? 2.f * P.wT * ((S.xh[i * Np1 + N] - P.goal[i]) + S.xl[i * Np1 + N]) : 0.f;
        }
#pragma unroll
        for (int d = 0; d < kBRing; ++d) {
            const int kk = N - 1 - d;
            if (kk >= 0 && lane < kBSlot / 4)
                bcp_async16(S.ring + d * kBSlot + 4 * lane, C.rec + (size_t)kk * kBimRec + R_SLOT + 4 * lane);
            bcp_async_commit();
        }
        bool ok = true;
        int slot = kBRing - 1;  // ring slot of stage k: (N - 1 - k) mod kBRing
#pragma unroll 1
        for (int k = N - 1; k >= 0; --k) {
            slot = (slot == kBRing - 1) ? 0 : slot + 1;
            bcp_async_wait<kBRing - 1>();
            __syncwarp();
            const float4* sl = reinterpret_cast<const float4*>(S.ring + slot * kBSlot);
            const float4 hd = sl[0];  // record floats 208..211: the u-block flag at 210
            float m[68];
#pragma unroll
            for (int q = 0; q < 17; ++q) {
                const float4 t = sl[1 + q];
                m[4 * q] = t.x;
                m[4 * q + 1] = t.y;
                m[4 * q + 2] = t.z;
                m[4 * q + 3] = t.w;
            }
            bool pd = hd.z > 0.f;
            __syncwarp();
            {
                const int kk = k - kBRing;
                if (kk >= 0 && lane < kBSlot / 4)
                    bcp_async16(S.ring + slot * kBSlot + 4 * lane, C.rec + (size_t)kk * kBimRec + R_SLOT + 4 * lane);
                bcp_async_commit();
            }
#pragma unroll
            for (int t = 0; t < 15; ++t) m[t] += V[t];
#pragma unroll
            for (int j = 0; j < 5; ++j) m[tri(10, j)] += v[j];
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const float p = m[tri(j, j)];
                pd = pd && (p > 0.f);
                const float ip = brcp_approx(p);
#pragma unroll
                for (int i = j + 1; i < 11; ++i) {
                    const float a = m[tri(i, j)] * ip;
#pragma unroll
                    for (int l = j + 1; l <= i; ++l)
                        if (!(i == 10 && l == 10)) m[tri(i, l)] -= a * m[tri(l, j)];
                }
            }
            if (!__all_sync(kFullB, pd)) {
                ok = false;
                break;
            }
            if (lane == 0) {
                // 45 raw factor entries (+3 pad) as 12 vector stores
                float o[48];
#pragma unroll
                for (int t = 0; t < 15; ++t) o[t] = m[t];
#pragma unroll
                for (int c = 0; c < 6; ++c)
#pragma unroll
                    for (int j = 0; j < 5; ++j) o[15 + 5 * c + j] = m[tri(5 + c, j)];
                o[45] = o[46] = o[47] = 0.f;
                cuda::annotated_ptr<float4, cuda::access_property::persisting> r4(
                    reinterpret_cast<float4*>(C.rec + (size_t)k * kBimRec + R_YF));
#pragma unroll
                for (int q = 0; q < 12; ++q) r4[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
            }
#pragma unroll
            for (int i = 0; i < 5; ++i) {
#pragma unroll
                for (int j = 0; j <= i; ++j) V[tri(i, j)] = m[tri(5 + i, 5 + j)];
                v[i] = m[tri(10, 5 + i)];
            }
        }
        bcp_async_wait_all();
        __syncwarp();
        // x_0 block (every lane), Cholesky with reciprocal pivots
        bool pd0 = ok;
        float d0[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (ok) {
            float H[5][5], g[5], L[5][5], il[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
#pragma unroll
                for (int j = 0; j < 5; ++j) H[i][j] = V[i >= j ? tri(i, j) : tri(j, i)];
                H[i][i] += rho;
                g[i] = v[i];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                H[i][i] += beta;
                g[i] += S.lam[i] + beta * ((S.xh[i * Np1] - P.start[i]) + S.xl[i * Np1]);
            }
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                float d = H[j][j];
#pragma unroll
                for (int q = 0; q < j; ++q) d -= L[j][q] * L[j][q];
                pd0 = pd0 && d > 0.f;
                il[j] = rsqrtf(fmaxf(d, 1e-30f));
#pragma unroll
                for (int i = j + 1; i < 5; ++i) {
                    float s = H[i][j];
#pragma unroll
                    for (int q = 0; q < j; ++q) s -= L[i][q] * L[j][q];
                    L[i][j] = s * il[j];
                }
            }
            float yv[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                float s = g[i];
#pragma unroll
                for (int q = 0; q < i; ++q) s -= L[i][q] * yv[q];
                yv[i] = s * il[i];
            }
#pragma unroll
            for (int i = 4; i >= 0; --i) {
                float s = yv[i];
#pragma unroll
                for (int q = i + 1; q < 5; ++q) s -= L[q][i] * d0[q];
                d0[i] = s * il[i];
            }
        }
        if (lane == 0) {
            if (ok)
                for (int i = 0; i < 5; ++i) S.red[16 + i] = -d0[i];
            S.red[21] = pd0 ? 1.f : 0.f;
        }
    }
    __syncthreads();
    const bool res = S.red[21] > 0.f;
    __syncthreads();
    return res;
}

// gains K_y = -L_y^{-T} [l_{x,y} | l_{rhs,y}] (5 x 6) per stage
__device__ void bphase_gains(BCtx& C) {
#pragma unroll 1
    for (int k = C.tid; k < C.N; k += kBimThreads) {
        float* rec = C.rec + (size_t)k * kBimRec;
        // raw factor: 15 y-y entries, then the (x, rhs) rows, as vector loads
        float m[48];
        const float4* r4 = reinterpret_cast<const float4*>(rec + R_YF);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const float4 t = r4[q];
            m[4 * q] = t.x;
            m[4 * q + 1] = t.y;
            m[4 * q + 2] = t.z;
            m[4 * q + 3] = t.w;
        }
        float ly[5][5], il[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            il[j] = rsqrtf(m[tri(j, j)]);
#pragma unroll
            for (int i = j + 1; i < 5; ++i) ly[i][j] = m[tri(i, j)] * il[j];
#pragma unroll
            for (int c = 0; c < 6; ++c) m[15 + 5 * c + j] *= il[j];
        }
        // K (row i at R_YF + 6 i), two pad floats, as vector stores
        float o[32];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
#pragma unroll
            for (int i = 4; i >= 0; --i) {
                float s = -m[15 + 5 * c + i];
#pragma unroll
                for (int q = i + 1; q < 5; ++q) s -= ly[q][i] * o[6 * q + c];
                o[6 * i + c] = s * il[i];
            }
        }
        o[30] = o[31] = 0.f;
        cuda::annotated_ptr<float4, cuda::access_property::persisting> w4(reinterpret_cast<float4*>(rec + R_YF));
#pragma unroll
        for (int q = 0; q < 8; ++q) w4[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    }
    __syncthreads();
}

// forward pass: the chain on 5 lanes of warp 0, then the control steps;
// returns D = grad . dz
__device__ float bphase_c(BCtx& C) {
    BSmem& S = C.S;
    const int N = C.N;
    if (C.warp == 0) {
        float dxi = (C.lane < 5) ? S.red[16 + C.lane] : 0.f;
        if (C.lane < 5) S.dz[C.lane] = dxi;
        float dxv[5];
        #pragma unroll
        for (int i = 0; i < 5; ++i) dxv[i] = __shfl_sync(kFullB, dxi, i);
#pragma unroll 1
        for (int k = 0; k < N; ++k) {
            float w = 0.f;
            if (C.lane < 5) {
                const float* g = C.rec + (size_t)k * kBimRec + R_YF + 6 * C.lane;
                w = g[5];
                #pragma unroll
                for (int j = 0; j < 5; ++j) w += g[j] * dxv[j];
                S.dz[NWV * (k + 1) + C.lane] = w;
            }
            #pragma unroll
            for (int i = 0; i < 5; ++i) dxv[i] = __shfl_sync(kFullB, w, i);
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int k = C.tid; k < N; k += kBimThreads) {
        const float* rec = C.rec + (size_t)k * kBimRec;
        float xa[5], xb[5];
        #pragma unroll
        for (int i = 0; i < 5; ++i) {
            xa[i] = S.dz[NWV * k + i];
            xb[i] = S.dz[NWV * (k + 1) + i];
        }
        float R[NU];
        #pragma unroll
        for (int j = 0; j < NU; ++j) {
            float s = rec[R_CPL + 10 * 12 + j];
            #pragma unroll
            for (int i = 0; i < 5; ++i) s += rec[R_CPL + i * 12 + j] * xb[i] + rec[R_CPL + (5 + i) * 12 + j] * xa[i];
            R[j] = s;
        }
        float du[NU];
        #pragma unroll
        for (int j = NU - 1; j >= 0; --j) {
            float s = -R[j];
            #pragma unroll
            for (int i = j + 1; i < NU; ++i) s -= rec[R_LUU + tri(i, j)] * du[i];
            du[j] = s / rec[R_LUU + tri(j, j)];
        }
        #pragma unroll
        for (int j = 0; j < NU; ++j) S.dz[NWV * k + NX + j] = du[j];
    }
    __syncthreads();
    float D = 0.f;
    for (int t = C.tid; t < NWV * N + NX; t += kBimThreads) D += S.gr[t] * S.dz[t];
    D = bwarp_sum(D);
    if (C.lane == 0) S.red[24 + C.warp] = D;
    __syncthreads();
    const float Dt = S.red[24] + S.red[25] + S.red[26] + S.red[27];
    __syncthreads();
    return Dt;
}

__device__ __forceinline__ float brow_al(bool ineq, float lam, float beta, float inv2b, float c) {
    if (!ineq) return lam * c + 0.5f * beta * c * c;
    const float t = fmaxf(lam + beta * c, 0.f);
    return (t * t - lam * lam) * inv2b;
}

// trial merits for alpha in {0, 1, ..., 2^-6}; returns the accepted alpha
__device__ float bphase_d(BCtx& C, float beta, float D, const SolverParams& sp) {
    BSmem& S = C.S;
    const BInst<float>& P = C.P;
    const int N = C.N, Np1 = C.Np1;
    // Trials four at a time (thread = trial + 4 x stage group, 32 groups),
    // largest alpha first: {1/8 .. 1/64} only when none of {1, 1/2, 1/4}
    // passes, which leaves the accepted alpha (the largest passing) unchanged.
    const int sub = C.tid & 3, grp = C.tid >> 2;
    const float inv2b = 0.5f / beta;
    float phi0 = 0.f, slack = 0.f, acc = 0.f;
#pragma unroll 1
    for (int batch = 0; batch < 2; ++batch) {
        if (batch == 1 && sp.n_alpha < 4) break;
        const int a = 4 * batch + sub;
        const float alpha = (a == 0) ? 0.f : ldexpf(1.f, -(a - 1));
        float phi = 0.f;
        if (a <= sp.n_alpha) {
#pragma unroll 1
            for (int k = grp; k < N; k += 32) {
                float x[NX], u[NU], dx[NX];
                load_stage(C, k, alpha, x, u, dx);
                const int mi = S.mi[k];
                BStage<float> St;
                stage_ctx(P, mi & 1023, x, u, St);
                const float* lam = S.lam + 3 + NR * k;
                for (int j = 0; j < NU; ++j) phi += rweight(P, j) * u[j] * u[j];
                for (int r = 0; r < NR; ++r) {
                    float c, sc;
                    bool on, iq;
                    brow<float, false>(r, P, St, (mi >> 10) & 1, (mi >> 11) & 1, x, u, dx, c, nullptr, on, iq, sc);
                    if (on) phi += brow_al(iq, lam[r], beta, inv2b, c);
                }
                if (k == 0)
                    for (int i = 0; i < 3; ++i) {
                        const float c = (S.xh[i * Np1] - P.start[i]) + (S.xl[i * Np1] + alpha * S.dz[i]);
                        phi += brow_al(false, S.lam[i], beta, inv2b, c);
                    }
                if (k == N - 1)
                    for (int i = 0; i < 3; ++i) {
                        const float e =
                            (S.xh[i * Np1 + N] - P.goal[i]) + (S.xl[i * Np1 + N] + alpha * S.dz[NWV * N + i]);
                        phi += P.wT * e * e;
                    }
            }
        }
        // threads with the same trial: xor 4, 8, 16 inside the warp, then the warps
        phi += __shfl_xor_sync(kFullB, phi, 4);
        phi += __shfl_xor_sync(kFullB, phi, 8);
        phi += __shfl_xor_sync(kFullB, phi, 16);
        if (C.lane < 4) S.red[32 + C.warp * 4 + C.lane] = phi;
        __syncthreads();
        if (C.tid == 0) {
            float ph[4];
            for (int q = 0; q < 4; ++q) ph[q] = S.red[32 + q] + S.red[36 + q] + S.red[40 + q] + S.red[44 + q];
            if (batch == 0) {
                phi0 = ph[0];
                slack = sp.ls_slack * fabsf(phi0);
            }
            const bool flat = fabsf(D) <= slack;
            float take = 0.f;
            for (int q = (batch == 0) ? 1 : 0; q < 4; ++q) {
                const int aq = 4 * batch + q;
                if (aq > sp.n_alpha) break;
                const float al = ldexpf(1.f, -(aq - 1));
                if (ph[q] <= phi0 + sp.armijo_c1 * al * D || (aq == 1 && flat && ph[q] <= phi0 + slack)) {
                    take = al;
                    break;
                }
            }
            S.red[30] = take;
        }
        __syncthreads();
        acc = S.red[30];
        __syncthreads();
        if (acc > 0.f) break;
    }
    return acc;
}

__device__ void bphase_e(BCtx& C, float alpha) {
    BSmem& S = C.S;
    const int N = C.N, Np1 = C.Np1;
    for (int t = C.tid; t < NX * Np1; t += kBimThreads) {
        const int i = t / Np1, k = t - i * Np1;
        float s, e;
        two_sum_b(S.xh[t], S.xl[t] + alpha * S.dz[NWV * k + i], s, e);
        S.xh[t] = s;
        S.xl[t] = e;
    }
    for (int t = C.tid; t < NU * N; t += kBimThreads) {
        const int j = t / N, k = t - j * N;
        S.us[t] += alpha * S.dz[NWV * k + NX + j];
    }
    __syncthreads();
}

// FP64 certificate: cost, physical violation, KKT residual (stationarity
// with the multiplier estimates at beta); scratch doubles in the workspace
struct BCert {
    double cost, viol, stat;
    bool finite;
};

__device__ BCert bcertify(BCtx& C, float beta_f) {
    BSmem& S = C.S;
    const int N = C.N, Np1 = C.Np1;
    BInst<double> P;
    load_inst(*C.D, P);
    const double beta = beta_f;
    double* g64 = reinterpret_cast<double*>(C.rec);  // [17 N + 5] then [5 (N + 1)]
    double* g64b = g64 + (NWV * N + NX);
    double cost = 0.0, viol = 0.0;
    bool finite = true;
    for (int k = C.tid; k < N; k += kBimThreads) {
        double x[NX], u[NU], dx[NX];
        for (int i = 0; i < NX; ++i) {
            const double a0 = (double)S.xh[i * Np1 + k] + (double)S.xl[i * Np1 + k];
            const double a1 = (double)S.xh[i * Np1 + k + 1] + (double)S.xl[i * Np1 + k + 1];
            x[i] = a0;
            dx[i] = a1 - a0;
        }
        for (int j = 0; j < NU; ++j) u[j] = (double)S.us[j * N + k];
        const int mi = S.mi[k];
        BStage<double> St;
        stage_ctx(P, mi & 1023, x, u, St);
        double g[NL];
        for (int j = 0; j < NL; ++j) g[j] = 0.0;
        for (int j = 0; j < NU; ++j) {
            g[NX + j] += 2.0 * rweight(P, j) * u[j];
            cost += rweight(P, j) * u[j] * u[j];
        }
        const float* lam = S.lam + 3 + NR * k;
        for (int r = 0; r < NR; ++r) {
            double c, J[NL], sc;
            bool on, iq;
            brow<double, true>(r, P, St, (mi >> 10) & 1, (mi >> 11) & 1, x, u, dx, c, J, on, iq, sc);
            if (!on) continue;
            const double t = (double)lam[r] + beta * c;
            const double y = iq ? fmax(t, 0.0) : t;
            const double vr = iq ? fmax(c, 0.0) : fabs(c);
            viol = fmax(viol, vr / sc);
            if (!isfinite(c)) finite = false;
            for (int j = 0; j < NL; ++j) g[j] += y * J[j];
        }
        for (int j = 0; j < NWV; ++j) g64[NWV * k + j] = g[j];
        for (int i = 0; i < NX; ++i) g64b[NX * (k + 1) + i] = g[NWV + i];
    }
    __syncthreads();
    double stat = 0.0;
    for (int k = C.tid; k <= N; k += kBimThreads) {
        for (int i = 0; i < NX; ++i) {
            double gv = (k < N) ? g64[NWV * k + i] : 0.0;
            if (k > 0) gv += g64b[NX * k + i];
            if (k == N && i < 3) {
                const double e = (double)S.xh[i * Np1 + N] + (double)S.xl[i * Np1 + N] - P.goal[i];
                gv += 2.0 * P.wT * e;
                cost += P.wT * e * e;
            }
            if (k == 0 && i < 3) {
                const double c = (double)S.xh[i * Np1] + (double)S.xl[i * Np1] - P.start[i];
                gv += (double)S.lam[i] + beta * c;
                viol = fmax(viol, fabs(c));
            }
            stat = fmax(stat, fabs(gv));
            if (!isfinite(gv)) finite = false;
        }
        if (k < N)
            for (int j = 0; j < NU; ++j) stat = fmax(stat, fabs(g64[NWV * k + NX + j]));
    }
    // block reductions (double, through the workspace scratch)
    for (int o = 16; o > 0; o >>= 1) {
        cost += __shfl_xor_sync(kFullB, cost, o);
        viol = fmax(viol, __shfl_xor_sync(kFullB, viol, o));
        stat = fmax(stat, __shfl_xor_sync(kFullB, stat, o));
    }
    const bool fin = __all_sync(kFullB, finite);
    __syncthreads();
    double* red = g64b + NX * (N + 1);
    if (C.lane == 0) {
        red[C.warp] = cost;
        red[4 + C.warp] = viol;
        red[8 + C.warp] = stat;
        red[12 + C.warp] = fin ? 1.0 : 0.0;
    }
    __syncthreads();
    BCert ct;
    ct.cost = red[0] + red[1] + red[2] + red[3];
    ct.viol = fmax(fmax(red[4], red[5]), fmax(red[6], red[7]));
    ct.stat = fmax(fmax(red[8], red[9]), fmax(red[10], red[11]));
    ct.finite = red[12] > 0 && red[13] > 0 && red[14] > 0 && red[15] > 0 && isfinite(ct.cost);
    __syncthreads();
    return ct;
}

__global__ void __launch_bounds__(kBimThreads, 4) bimanual_kernel(EvalArgs A) {
    extern __shared__ float bsm[];
    BCtx C;
    C.tid = threadIdx.x;
    C.warp = threadIdx.x >> 5;
    C.lane = threadIdx.x & 31;
    C.S = bcarve(bsm, A.Nmax);
    C.rec = A.ws + (size_t)blockIdx.x * A.ws_per_warp;
    BSmem& S = C.S;
    const SolverParams& sp = A.sp;
    const int64_t n_tos = A.d_n ? min(*A.d_n, A.n) : A.n;
    __shared__ unsigned int s_t;
    for (;;) {
        if (C.tid == 0) s_t = atomicAdd(A.queue, 1u);
        __syncthreads();
        const unsigned int t = s_t;
        __syncthreads();
        if ((int64_t)t >= n_tos) break;
        const int64_t ti = A.perm ? (int64_t)A.perm[t] : (int64_t)t;
        const comet_mode_seq sq = A.seqs[ti];
        bool bad = sq.instance < 0 || sq.instance >= A.n_inst;
        const DevInstance* D = bad ? A.inst : A.inst + sq.instance;
        const int len = sq.len;
        bad = bad || len < 1 || len > D->Lmax || len > COMET_MAX_SEGMENTS;
        if (!bad)
            for (int i = 0; i < len; ++i) bad = bad || sq.modes[i] >= D->n_modes;
        if (bad) {
            if (C.tid == 0) {
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
        C.D = D;
        load_inst(*D, C.P);
        C.len = len;
        C.N = D->K * len;
        C.Np1 = C.N + 1;
        const int N = C.N, Np1 = C.Np1, Nm1 = A.Nmax + 1;
        const BInst<float>& P = C.P;
        // initial iterate
        const float* warm = A.warm ? A.warm + ti * A.stride : nullptr;
        for (int q = C.tid; q < NX * Np1; q += kBimThreads) {
            const int i = q / Np1, k = q - i * Np1;
            float x;
            if (warm) {
                x = warm[i * Nm1 + k];
            } else if (i < 3) {
                const float al = (float)k / (float)N;
                x = (1.f - al) * P.start[i] + al * P.goal[i];
            } else {
                x = 0.f;
            }
            S.xh[q] = x;
            S.xl[q] = 0.f;
        }
        for (int q = C.tid; q < NU * N; q += kBimThreads) {
            const int j = q / N, k = q - j * N;
            S.us[q] = warm ? warm[NX * Nm1 + j * A.Nmax + k] : ((j == ULN - 5) ? P.mg : 0.f);
        }
        for (int q = C.tid; q < 3 + NR * N; q += kBimThreads) S.lam[q] = 0.f;
        for (int q = C.tid; q < NWV * N + NX; q += kBimThreads) S.dz[q] = S.gr[q] = 0.f;
        for (int k = C.tid; k < N; k += kBimThreads) {
            const int seg = (int)(((long long)k * len) / N);
            const int m = sq.modes[seg];
            int mL = 0, mR = 0;
            if (k + 1 < N) {
                const int m1 = sq.modes[(int)(((long long)(k + 1) * len) / N)];
                const int hL0 = (m / 13) % 13, hL1 = (m1 / 13) % 13, hR0 = m % 13, hR1 = m1 % 13;
                const int fL0 = hL0 ? (hL0 - 1) / 3 : -1, fL1 = hL1 ? (hL1 - 1) / 3 : -1;
                const int fR0 = hR0 ? (hR0 - 1) / 3 : -1, fR1 = hR1 ? (hR1 - 1) / 3 : -1;
                mL = fL0 != fL1;
                mR = fR0 != fR1;
            }
            S.mi[k] = m | (mL << 10) | (mR << 11);
        }
        __syncthreads();

        float beta = sp.beta0, rho = sp.rho0, eta = INFINITY;
        int inner = 0, it = 0, status = COMET_TO_MAX_ITER;
        bool nonfinite = false;
        for (it = 0; it < sp.max_iters; ++it) {
            // (assemble, sweep) trips through one call site of each phase
            // (one inlined copy in the hot loop): the measures and model at
            // the iterate, the dual update at beta_old after a solved
            // subproblem, and reassembly at rising damping after a failed
            // sweep.  Every decision is taken on CTA-wide reductions, so all
            // threads follow the same trips.
            enum { kMeasure, kUpdate, kRetry };
            int trip = kMeasure, retries = 0;
            bool fac = false, done = false;
            float beta_old = beta;
            for (;;) {
                const BMeasures m = bphase_a(C, beta, rho, true, trip == kUpdate, beta_old);
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
                fac = bphase_b(C, beta, rho);
                if (fac || retries >= sp.max_retries) break;
                ++retries;
                rho = fminf(sp.rho_max, rho * 10.f);
                trip = kRetry;
            }
            if (done) break;
            ++inner;
            if (!fac) continue;
            bphase_gains(C);
            const float Dv = bphase_c(C);
            const float alpha = bphase_d(C, beta, Dv, sp);
            if (alpha > 0.f) {
                bphase_e(C, alpha);
                rho = fmaxf(sp.rho_min, rho / 10.f);
            } else {
                rho = fminf(sp.rho_max, rho * 10.f);
            }
        }
        const BCert ct = bcertify(C, beta);
        if (!ct.finite) nonfinite = true;
        if (nonfinite) status = COMET_TO_NONFINITE;
        if (status == COMET_TO_CONVERGED && !(ct.viol <= sp.eps_feas)) status = COMET_TO_INFEASIBLE;
        if (C.tid == 0) {
            A.out_status[ti] = status;
            A.out_cost[ti] = (float)ct.cost;
            if (A.out_viol) A.out_viol[ti] = (float)ct.viol;
            if (A.out_merit) A.out_merit[ti] = (float)(ct.cost + sp.merit_mu * fmax(ct.viol - sp.eps_feas, 0.0));
            if (A.out_iters) A.out_iters[ti] = it;
            if (A.out_stat) A.out_stat[ti] = (float)ct.stat;
        }
        if (A.out_traj) {
            float* out = A.out_traj + ti * A.stride;
            for (int q = C.tid; q < NX * Nm1; q += kBimThreads) {
                const int i = q / Nm1, k = q - i * Nm1;
                out[q] = (k <= N) ? S.xh[i * Np1 + k] + S.xl[i * Np1 + k] : 0.f;
            }
            for (int q = C.tid; q < NU * A.Nmax; q += kBimThreads) {
                const int j = q / A.Nmax, k = q - j * A.Nmax;
                out[NX * Nm1 + q] = (k < N) ? S.us[j * N + k] : 0.f;
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t bim_smem_bytes(int Nmax) { return bsmem_floats(Nmax) * sizeof(float); }

int bim_blocks_per_sm(int Nmax) {
    const size_t smem = bim_smem_bytes(Nmax);
    if (cudaFuncSetAttribute(bimanual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bimanual_kernel, kBimThreads, smem) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_bimanual(const EvalArgs& a, int n_ctas, cudaStream_t s) {
    const size_t smem = bim_smem_bytes(a.Nmax);
    bimanual_kernel<<<n_ctas, kBimThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace comet
