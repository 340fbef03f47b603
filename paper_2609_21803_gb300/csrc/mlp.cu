// mlp.cu -- the learned proposal (comet_proposal.h): a 4-layer GELU MLP on
// the BF16 tensor cores that predicts an order's log merit (Eq.
// search_merit) and the controls of its solved trajectory (Eq. mode_nlp),
// trained on the GPU on evaluator results and used to order, prune and
// warm-start the orders of an expansion round (Algorithm 1).
//
// Every GEMM runs on the hand-written tcgen05 kernel (mlp_gemm.cu) with a
// fused epilogue; the element-wise parts (features, targets, loss gradient,
// bias gradients, AdamW, mini-batch gather, warm-start rollout) are plain
// CUDA kernels.  A training step is captured once as a CUDA graph and
// replayed; its step counter lives in device memory.

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "comet.h"
#include "comet_internal.h"
#include "comet_proposal.h"
#include "expand_internal.h"
#include "mlp_internal.h"
#include "problem_internal.h"

namespace {

constexpr int kLayers = 4;
constexpr int kInstFeat = 12;  // per-instance features ahead of the one-hot slots
constexpr int kBimSlot = 30;   // bimanual slot: ground 3 + left hand 13 + right hand 13 + blank
constexpr float kGrav = 9.81f;

// bimanual controls (xd, zd, thd, fn_L, ft_L, sd_L, fn_R, ft_R, sd_R, lam_n,
// lam_t, p_c): the forces, which the proposal predicts in units of m g
__host__ __device__ inline bool bim_force(int j) { return j == 3 || j == 4 || j == 6 || j == 7 || j == 9 || j == 10; }

}  // namespace

struct comet_proposal {
    comet_problem* p = nullptr;
    comet_proposal_desc desc;
    int in_dim = 0, width = 0, out_dim = 0, l_max = 0, n_max = 0, n_modes = 0, n_inst = 0;
    // task layout: bimanual (factored one-hot, 12 controls on 5 states) or pushing
    int bim = 0, nx = 4, n_ctrl = 3, slot_w = 13;
    int64_t n_params = 0;
    int64_t w_off[kLayers], b_off[kLayers];
    int din[kLayers], dout[kLayers];
    float* master = nullptr;  // [n_params]
    float* grad = nullptr;
    float* m1 = nullptr;
    float* m2 = nullptr;
    uint16_t* wq[kLayers] = {};   // bf16 W_l [dout][din]
    uint16_t* wqt[kLayers] = {};  // bf16 W_l^T [din][dout]
    float* feat_inst = nullptr;   // [n_inst][kInstFeat]
    int64_t* d_step = nullptr;    // AdamW step count t
    float* d_loss = nullptr;
    int* d_err = nullptr;
    // activations of one batch (rows_cap rows; transposed copies ld_t)
    int64_t rows_cap = 0, ld_t = 0;
    uint16_t* X = nullptr;
    uint16_t* Xt = nullptr;
    float* Z[3] = {};
    uint16_t* H[3] = {};
    uint16_t* Ht[3] = {};
    float* Y = nullptr;
    uint16_t* G[kLayers] = {};
    uint16_t* Gt[kLayers] = {};
    float* T = nullptr;
    float* Om = nullptr;
    // training set
    int64_t ds_cap = 0, ds_n = 0;
    uint16_t* ds_X = nullptr;
    float* ds_T = nullptr;
    float* ds_Om = nullptr;
    // prune scratch
    int64_t pr_cap = 0;
    comet_mode_seq* pr_seqs = nullptr;
    unsigned long long* pr_codes = nullptr;
    float* pr_merit = nullptr;
    comet::TopKey* pr_top_a = nullptr;
    comet::TopKey* pr_top_b = nullptr;
    std::vector<void*> allocs;
};

namespace {

comet_status qfail(comet_status st, const char* msg) {
    comet::set_error(msg);
    return st;
}

comet_status qcuda(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return qfail(e == cudaErrorMemoryAllocation ? COMET_ERR_OOM : COMET_ERR_CUDA, buf);
}

#define QTRY(call, what)                               \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return qcuda(e_, what); \
    } while (0)

bool qdev(const void* ptr) {
    cudaPointerAttributes at;
    if (!ptr || cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int64_t pad_to(int64_t n, int64_t m) { return (n + m - 1) / m * m; }

template <typename T>
cudaError_t qalloc(comet_proposal* q, T** ptr, size_t count) {
    void* v = nullptr;
    const cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    q->allocs.push_back(v);
    *ptr = static_cast<T*>(v);
    return cudaSuccess;
}

void qfree(comet_proposal* q, void* ptr) {
    if (!ptr) return;
    auto it = std::find(q->allocs.begin(), q->allocs.end(), ptr);
    if (it != q->allocs.end()) q->allocs.erase(it);
    cudaFree(ptr);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_value(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    // SplitMix64 finaliser (Steele, Lea and Flood 2014)
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

struct LayerTab {
    int64_t w_off[kLayers], b_off[kLayers];
    int din[kLayers], dout[kLayers];
    uint16_t* wq[kLayers];
    uint16_t* wqt[kLayers];
};

LayerTab layer_tab(const comet_proposal* q) {
    LayerTab t;
    for (int l = 0; l < kLayers; ++l) {
        t.w_off[l] = q->w_off[l];
        t.b_off[l] = q->b_off[l];
        t.din[l] = q->din[l];
        t.dout[l] = q->dout[l];
        t.wq[l] = q->wq[l];
        t.wqt[l] = q->wqt[l];
    }
    return t;
}

// weight i of the flat vector -> (layer, row, col); false for a bias
__device__ __forceinline__ bool weight_of(const LayerTab& t, int64_t i, int& l, int& r, int& c) {
#pragma unroll
    for (int j = 0; j < kLayers; ++j) {
        const int64_t o = i - t.w_off[j];
        if (o >= 0 && o < (int64_t)t.dout[j] * t.din[j]) {
            l = j;
            r = (int)(o / t.din[j]);
            c = (int)(o - (int64_t)r * t.din[j]);
            return true;
        }
    }
    return false;
}

// U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from a counter-based hash of
// (seed, index); zero biases
__global__ void init_params_kernel(float* p, int64_t n, LayerTab t, unsigned long long seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int l, r, c;
        float v = 0.f;
        if (weight_of(t, i, l, r, c)) {
            const unsigned long long h = mix64(seed * 0x9e3779b97f4a7c15ull + (unsigned long long)i);
            const float u = (float)(h >> 40) * (1.0f / 16777216.0f);  // [0, 1)
            v = (2.f * u - 1.f) * rsqrtf((float)t.din[l]);
        }
        p[i] = v;
    }
}

// BF16 copies W_l and W_l^T of the master weights
__global__ void quantize_kernel(const float* p, int64_t n, LayerTab t) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int l, r, c;
        if (weight_of(t, i, l, r, c)) {
            const uint16_t b = bf16_bits(p[i]);
            t.wq[l][(int64_t)r * t.din[l] + c] = b;
            t.wqt[l][(int64_t)c * t.dout[l] + r] = b;
        }
    }
}

// AdamW with bias-corrected moments and decoupled weight decay at step t =
// *d_step (incremented by the loss kernel of the same step)
__global__ void adamw_kernel(float* p, const float* g, float* m, float* v, int64_t n, LayerTab t,
                             const int64_t* d_step, float lr, float b1, float b2, float eps, float wd) {
    const float st = (float)(*d_step);
    const float bc1 = 1.f - powf(b1, st), bc2 = 1.f - powf(b2, st);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * ((mi / bc1) / (sqrtf(vi / bc2) + eps) + wd * p[i]);
        p[i] = pi;
        int l, r, c;
        if (weight_of(t, i, l, r, c)) {
            const uint16_t b = bf16_bits(pi);
            t.wq[l][(int64_t)r * t.din[l] + c] = b;
            t.wqt[l][(int64_t)c * t.dout[l] + r] = b;
        }
    }
}

// features of order i (see comet_proposal.h); rows i >= n (device count)
// and orders of another instance range give zero rows
__global__ void features_kernel(const comet_mode_seq* seqs, int64_t n_rows, const int64_t* d_n, const float* fi,
                                int n_inst, int l_max, int n_modes, int in_dim, uint16_t* X, uint16_t* Xt,
                                int64_t ld_t, int bim) {
    const int slot_w = bim ? kBimSlot : n_modes + 1;
    const int64_t nn = d_n ? min(*d_n, n_rows) : n_rows;
    const int64_t total = n_rows * in_dim;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / in_dim;
        const int c = (int)(t - i * in_dim);
        float x = 0.f;
        if (i < nn) {
            const comet_mode_seq s = seqs[i];
            if (s.instance >= 0 && s.instance < n_inst && s.len >= 1 && s.len <= l_max) {
                if (c < kInstFeat) {
                    x = fi[s.instance * kInstFeat + c];
                } else if (c < kInstFeat + slot_w * l_max) {
                    const int slot = (c - kInstFeat) / slot_w, e = (c - kInstFeat) % slot_w;
                    if (bim) {
                        // mode m = 169 g + 13 h_L + h_R: one-hots of g, h_L, h_R
                        const int m = slot < s.len ? (int)s.modes[slot] : -1;
                        x = (m < 0) ? (e == kBimSlot - 1 ? 1.f : 0.f)
                                    : ((e == m / 169 || e == 3 + (m / 13) % 13 || e == 16 + m % 13) ? 1.f : 0.f);
                    } else {
                        const int want = slot < s.len ? (int)s.modes[slot] : n_modes;
                        x = (e == want) ? 1.f : 0.f;
                    }
                }
            }
        }
        const uint16_t b = bf16_bits(x);
        X[i * in_dim + c] = b;
        if (Xt) Xt[(int64_t)c * ld_t + i] = b;
    }
}

// training targets and weights of evaluator results (comet_proposal.h)
__global__ void targets_kernel(const comet_mode_seq* seqs, int64_t n, const float* cost, const float* viol,
                               const int32_t* status, const float* traj, int64_t stride, const int* Kseg,
                               int n_inst, int n_max, int out_dim, float merit_mu, float eps_feas, float lambda_w,
                               float* T, float* Om, int nx, int n_ctrl, int bim, const comet::DevInstance* inst) {
    const int64_t total = n * out_dim;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / out_dim;
        const int c = (int)(t - i * out_dim);
        const comet_mode_seq s = seqs[i];
        const int st = status[i];
        const bool valid_inst = s.instance >= 0 && s.instance < n_inst;
        float tv = 0.f, w = 0.f;
        if (c == 0) {
            float m = cost[i] + merit_mu * fmaxf(viol[i] - eps_feas, 0.f);
            if (st != COMET_TO_NONFINITE && isfinite(m) && valid_inst) {
                tv = logf(fmaxf(m, 1e-12f));
                w = 1.f;
            }
        } else if (c <= n_ctrl * n_max && valid_inst && st == COMET_TO_CONVERGED) {
            const int comp = (c - 1) / n_max, k = (c - 1) % n_max;
            const int N = Kseg[s.instance] * s.len;
            if (k < N) {
                tv = traj[i * stride + nx * (int64_t)(n_max + 1) + (int64_t)comp * n_max + k];
                if (bim && bim_force(comp)) tv /= inst[s.instance].mass * kGrav;
                w = lambda_w / ((float)n_ctrl * (float)N);
            }
        }
        T[t] = tv;
        Om[t] = w;
    }
}

// mini-batch gather: row b of the batch is sample hash(seed, step, b) mod S
__global__ void gather_kernel(const uint16_t* dX, const float* dT, const float* dOm, int64_t S, int batch,
                              const int64_t* d_step, unsigned long long seed, int in_dim, int out_dim, uint16_t* X,
                              uint16_t* Xt, int64_t ld_t, float* T, float* Om) {
    const unsigned long long step = (unsigned long long)(*d_step);
    const int64_t per = (int64_t)in_dim + out_dim;
    const int64_t total = (int64_t)batch * per;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / per;
        const int c = (int)(t - b * per);
        const unsigned long long h = mix64(seed ^ mix64(step * 0x100000001b3ull + (unsigned long long)b));
        const int64_t j = (int64_t)(h % (unsigned long long)S);
        if (c < in_dim) {
            const uint16_t v = dX[j * in_dim + c];
            X[b * in_dim + c] = v;
            Xt[(int64_t)c * ld_t + b] = v;
        } else {
            const int o = c - in_dim;
            T[b * out_dim + o] = dT[j * out_dim + o];
            Om[b * out_dim + o] = dOm[j * out_dim + o];
        }
    }
}

// dL/dY = (2/B) Omega (Y - T) -> G (bf16) and its transpose; the loss sum
// is accumulated into *loss and the step counter advanced
__global__ void loss_grad_kernel(const float* Y, const float* T, const float* Om, int64_t M, int out_dim, uint16_t* G,
                                 uint16_t* Gt, int64_t ld_t, float* loss, int64_t* d_step) {
    __shared__ float red[32];
    const float inv_b = 1.f / (float)M;
    float acc = 0.f;
    const int64_t total = M * out_dim;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / out_dim;
        const int c = (int)(t - r * out_dim);
        const float d = Y[t] - T[t], w = Om[t];
        acc += w * d * d;
        const uint16_t g = bf16_bits(2.f * w * d * inv_b);
        G[t] = g;
        Gt[(int64_t)c * ld_t + r] = g;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) atomicAdd(loss, v * inv_b);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_step += 1;
}

// db[n] = sum_m G[m][n], from the transposed copy (one block per n)
__global__ void bias_grad_kernel(const uint16_t* Gt, int64_t ld_t, int64_t M, float* db) {
    __shared__ float red[32];
    const uint16_t* row = Gt + (int64_t)blockIdx.x * ld_t;
    float acc = 0.f;
    for (int64_t m = threadIdx.x; m < M; m += blockDim.x) acc += bf16_value(row[m]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) db[blockIdx.x] = v;
    }
}

// merit = exp(y_0) and the warm start of order i from the predicted
// controls: Euler rollout of the pusher-slider model from the start pose
// (s_0 = 0, s reset to 0 after a face change), or the cold-start poses
__global__ void predict_post_kernel(const float* Y, int out_dim, const comet_mode_seq* seqs, const int* row_of,
                                    int64_t n_rows, const int64_t* d_n, const comet::DevInstance* inst, int n_inst,
                                    int n_max, int warm_mode, float* merit, float* warm, int64_t stride, int bim) {
    const int64_t nn = d_n ? min(*d_n, n_rows) : n_rows;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = row_of ? (int64_t)row_of[i] : i;
        const float* y = Y + r * out_dim;
        if (merit) merit[i] = expf(y[0]);
        if (!warm) continue;
        float* w = warm + i * stride;
        const comet_mode_seq s = seqs[i];
        if (s.instance < 0 || s.instance >= n_inst || s.len < 1) {
            for (int64_t t = 0; t < stride; ++t) w[t] = 0.f;
            continue;
        }
        const comet::DevInstance& P = inst[s.instance];
        const int L = s.len, N = P.K * L, Nm1 = n_max + 1;
        if (bim) {
            // bimanual: the cold start's poses (hand offsets 0) and the
            // predicted controls, forces back from units of m g
            const float mg = P.mass * kGrav;
            for (int k = 0; k <= n_max; ++k) {
                const float al = (float)k / (float)N;
                for (int c = 0; c < 5; ++c)
                    w[c * Nm1 + k] = (k <= N && c < 3) ? (1.f - al) * P.start[c] + al * P.goal[c] : 0.f;
            }
            for (int c = 0; c < 12; ++c)
                for (int k = 0; k < n_max; ++k)
                    w[5 * Nm1 + c * n_max + k] = (k < N) ? y[1 + c * n_max + k] * (bim_force(c) ? mg : 1.f) : 0.f;
            continue;
        }
        float x[4] = {P.start[0], P.start[1], P.start[2], 0.f};
        for (int k = 0; k <= N; ++k) {
            if (warm_mode == 1 && k > 0) {
                const float al = (float)k / (float)N;
                for (int c = 0; c < 3; ++c) x[c] = (1.f - al) * P.start[c] + al * P.goal[c];
                x[3] = 0.f;
            }
            for (int c = 0; c < 4; ++c) w[c * Nm1 + k] = x[c];
            if (k == N) break;
            const float fn = y[1 + k], ft = y[1 + n_max + k], sd = y[1 + 2 * n_max + k];
            for (int c = 0; c < 3; ++c) {
                const float u = y[1 + c * n_max + k];
                w[4 * Nm1 + c * n_max + k] = u;
            }
            if (warm_mode == 0) {
                const int seg = (int)(((long long)k * L) / N);
                const int face = s.modes[seg] / 3;
                const float nx = (face == 0) ? 1.f : ((face == 2) ? -1.f : 0.f);
                const float ny = (face == 1) ? 1.f : ((face == 3) ? -1.f : 0.f);
                const float tx = -ny, ty = nx;
                float st, ct;
                sincosf(x[2], &st, &ct);
                const float vx = P.kappa * (fn * nx + ft * tx), vy = P.kappa * (fn * ny + ft * ty);
                const float om = P.kappa * (-P.a[face] * ft - x[3] * fn) * P.inv_c2;
                bool reset = false;
                if (k + 1 < N) {
                    const int seg1 = (int)(((long long)(k + 1) * L) / N);
                    reset = (s.modes[seg1] / 3) != face;
                }
                x[0] += P.dt * (ct * vx - st * vy);
                x[1] += P.dt * (st * vx + ct * vy);
                x[2] += P.dt * om;
                x[3] = reset ? 0.f : x[3] + P.dt * sd;
            }
        }
        for (int k = N + 1; k <= n_max; ++k)
            for (int c = 0; c < 4; ++c) w[c * Nm1 + k] = 0.f;
        for (int c = 0; c < 3; ++c)
            for (int k = N; k < n_max; ++k) w[4 * Nm1 + c * n_max + k] = 0.f;
    }
}

__global__ void encode_kernel(const comet_mode_seq* seqs, int64_t n_rows, const int64_t* d_n, int n_modes,
                              unsigned long long* codes) {
    const int64_t nn = d_n ? min(*d_n, n_rows) : n_rows;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const comet_mode_seq s = seqs[i];
        const unsigned long long base = (unsigned long long)(n_modes + 1);
        unsigned long long code = s.len, p = base;
        for (int j = 0; j < s.len; ++j) {
            code += (unsigned long long)(s.modes[j] + 1) * p;
            p *= base;
        }
        codes[i] = code;
    }
}

__global__ void log_merit_kernel(const float* Y, int out_dim, int64_t n_rows, const int64_t* d_n, float* m) {
    const int64_t nn = d_n ? min(*d_n, n_rows) : n_rows;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x)
        m[i] = Y[i * out_dim];
}

// the kept candidates, best first: F.next[i] = candidate top[i].idx
__global__ void keep_kernel(const comet::TopKey* top, const comet_mode_seq* cand, int64_t* n_next, int keep,
                            comet_mode_seq* next, int* row_of) {
    const int64_t n = *n_next;
    const int kept = (int)min((int64_t)keep, n);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kept; i += gridDim.x * blockDim.x) {
        const int r = (int)top[i].idx;
        next[i] = cand[r];
        row_of[i] = r;
    }
}

__global__ void set_count_kernel(int64_t* n_next, int keep) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *n_next = min(*n_next, (int64_t)keep);
}

// Xt[c][b] = X[b][c]
__global__ void transpose_kernel(const uint16_t* X, int64_t n, int in_dim, uint16_t* Xt, int64_t ld) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * in_dim;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / in_dim;
        const int c = (int)(t - b * in_dim);
        Xt[(int64_t)c * ld + b] = X[t];
    }
}

int grid_for(int64_t work, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, 152 * 16));
}

// ------------------------------------------------------------ host side

cudaError_t ensure_rows(comet_proposal* q, int64_t rows) {
    if (rows <= q->rows_cap) return cudaSuccess;
    const int64_t cap = pad_to(std::max<int64_t>(rows, 128), 128);
    auto rel = [&](auto*& ptr) {
        qfree(q, ptr);
        ptr = nullptr;
    };
    rel(q->X);
    rel(q->Xt);
    rel(q->Y);
    rel(q->T);
    rel(q->Om);
    for (int l = 0; l < 3; ++l) {
        rel(q->Z[l]);
        rel(q->H[l]);
        rel(q->Ht[l]);
    }
    for (int l = 0; l < kLayers; ++l) {
        rel(q->G[l]);
        rel(q->Gt[l]);
    }
    q->rows_cap = 0;
    cudaError_t e;
    const int W = q->width, I = q->in_dim, O = q->out_dim;
    if ((e = qalloc(q, &q->X, (size_t)cap * I)) != cudaSuccess) return e;
    if ((e = qalloc(q, &q->Xt, (size_t)cap * I)) != cudaSuccess) return e;
    if ((e = qalloc(q, &q->Y, (size_t)cap * O)) != cudaSuccess) return e;
    if ((e = qalloc(q, &q->T, (size_t)cap * O)) != cudaSuccess) return e;
    if ((e = qalloc(q, &q->Om, (size_t)cap * O)) != cudaSuccess) return e;
    for (int l = 0; l < 3; ++l) {
        if ((e = qalloc(q, &q->Z[l], (size_t)cap * W)) != cudaSuccess) return e;
        if ((e = qalloc(q, &q->H[l], (size_t)cap * W)) != cudaSuccess) return e;
        if ((e = qalloc(q, &q->Ht[l], (size_t)cap * W)) != cudaSuccess) return e;
    }
    for (int l = 0; l < kLayers; ++l) {
        const int d = (l == kLayers - 1) ? O : W;
        if ((e = qalloc(q, &q->G[l], (size_t)cap * d)) != cudaSuccess) return e;
        if ((e = qalloc(q, &q->Gt[l], (size_t)cap * d)) != cudaSuccess) return e;
    }
    q->rows_cap = cap;
    q->ld_t = cap;
    return cudaSuccess;
}

cudaError_t forward(comet_proposal* q, int64_t M, bool train, cudaStream_t s) {
    using namespace comet::mlp;
    const int W = q->width;
    // inference: the four layers in one persistent kernel (the layered GEMMs
    // remain for training, which keeps Z and the transposed activations)
    if (!train && (q->in_dim == 64 || q->in_dim == 128) && W == 256 && q->out_dim <= 256) {
        const uint16_t* w[4] = {q->wq[0], q->wq[1], q->wq[2], q->wq[3]};
        const float* b[4] = {q->master + q->b_off[0], q->master + q->b_off[1], q->master + q->b_off[2],
                             q->master + q->b_off[3]};
        return mlp_forward_fused(q->X, M, q->in_dim, w, q->out_dim, b, q->Y, q->out_dim, q->d_err, q->p->num_sms, s);
    }
    for (int l = 0; l < kLayers; ++l) {
        Epilogue ep;
        memset(&ep, 0, sizeof(ep));
        ep.err = q->d_err;
        ep.bias = q->master + q->b_off[l];
        const Mat A = (l == 0) ? Mat{q->X, M, q->in_dim, q->in_dim} : Mat{q->H[l - 1], M, W, W};
        const Mat B{q->wq[l], q->dout[l], q->din[l], q->din[l]};
        if (l < kLayers - 1) {
            ep.kind = kEpiBiasGelu;
            ep.out_f32 = q->Z[l];
            ep.ld_out = W;
            ep.h = q->H[l];
            ep.ld_h = W;
            ep.h_t = train ? q->Ht[l] : nullptr;
            ep.ld_ht = q->ld_t;
        } else {
            ep.kind = kEpiStore;
            ep.out_f32 = q->Y;
            ep.ld_out = q->out_dim;
        }
        const cudaError_t e = gemm_bf16(A, B, M, q->dout[l], q->din[l], 1, ep, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// backward + AdamW of the batch in q->X / Xt / T / Om (M rows)
cudaError_t backward_update(comet_proposal* q, int64_t M, const comet_adamw_opts& o, cudaStream_t s) {
    using namespace comet::mlp;
    cudaError_t e;
    if ((e = cudaMemsetAsync(q->grad, 0, sizeof(float) * q->n_params, s)) != cudaSuccess) return e;
    loss_grad_kernel<<<grid_for(M * q->out_dim), 256, 0, s>>>(q->Y, q->T, q->Om, M, q->out_dim, q->G[kLayers - 1],
                                                               q->Gt[kLayers - 1], q->ld_t, q->d_loss, q->d_step);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int W = q->width;
    const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(16, M / 256));
    for (int l = kLayers - 1; l >= 0; --l) {
        // dW_l = G_l^T H_{l-1}: both operands from the transposed copies
        Epilogue ew;
        memset(&ew, 0, sizeof(ew));
        ew.kind = kEpiAtomicAdd;
        ew.out_f32 = q->grad + q->w_off[l];
        ew.ld_out = q->din[l];
        ew.err = q->d_err;
        const Mat A{q->Gt[l], q->dout[l], M, q->ld_t};
        const Mat B{(l > 0) ? q->Ht[l - 1] : q->Xt, q->din[l], M, q->ld_t};
        if ((e = gemm_bf16(A, B, q->dout[l], q->din[l], (int)M, splits, ew, s)) != cudaSuccess) return e;
        bias_grad_kernel<<<q->dout[l], 256, 0, s>>>(q->Gt[l], q->ld_t, M, q->grad + q->b_off[l]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (l == 0) break;
        // G_{l-1} = (G_l W_l) * GELU'(Z_{l-1})
        Epilogue eg;
        memset(&eg, 0, sizeof(eg));
        eg.kind = kEpiGeluGrad;
        eg.z_in = q->Z[l - 1];
        eg.ld_z = W;
        eg.h = q->G[l - 1];
        eg.ld_h = W;
        eg.h_t = q->Gt[l - 1];
        eg.ld_ht = q->ld_t;
        eg.err = q->d_err;
        const Mat Ag{q->G[l], M, q->dout[l], q->dout[l]};
        const Mat Bg{q->wqt[l], q->din[l], q->dout[l], q->dout[l]};
        if ((e = gemm_bf16(Ag, Bg, M, q->din[l], q->dout[l], 1, eg, s)) != cudaSuccess) return e;
    }
    adamw_kernel<<<grid_for(q->n_params), 256, 0, s>>>(q->master, q->grad, q->m1, q->m2, q->n_params, layer_tab(q),
                                                       q->d_step, (float)o.lr, (float)o.beta1, (float)o.beta2,
                                                       (float)o.eps, (float)o.weight_decay);
    return cudaGetLastError();
}

comet_status check_err(comet_proposal* q, cudaStream_t s) {
    int err = 0;
    QTRY(cudaMemcpyAsync(&err, q->d_err, sizeof(int), cudaMemcpyDeviceToHost, s), "read error flag");
    QTRY(cudaStreamSynchronize(s), "synchronise");
    if (err) return qfail(COMET_ERR_TIMEOUT, "tensor-core GEMM: a bounded wait ran out");
    return COMET_OK;
}

// copy n * bytes_per from src (host or device) to a device buffer
cudaError_t to_device(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
}

cudaError_t ensure_prune(comet_proposal* q, int64_t cap) {
    // the top-k passes write at most chunks x keep <= chunks x kChunk keys
    const int64_t chunks = (cap + comet::kChunk - 1) / comet::kChunk;
    if (cap <= q->pr_cap) return cudaSuccess;
    qfree(q, q->pr_seqs);
    qfree(q, q->pr_codes);
    qfree(q, q->pr_merit);
    qfree(q, q->pr_top_a);
    qfree(q, q->pr_top_b);
    q->pr_cap = 0;
    cudaError_t e;
    if ((e = qalloc(q, &q->pr_seqs, cap)) != cudaSuccess) return e;
    if ((e = qalloc(q, &q->pr_codes, cap)) != cudaSuccess) return e;
    if ((e = qalloc(q, &q->pr_merit, cap)) != cudaSuccess) return e;
    const int64_t tn = std::max<int64_t>(chunks * comet::kChunk, comet::kChunk);
    if ((e = qalloc(q, &q->pr_top_a, tn)) != cudaSuccess) return e;
    if ((e = qalloc(q, &q->pr_top_b, tn)) != cudaSuccess) return e;
    q->pr_cap = cap;
    return cudaSuccess;
}

}  // namespace

namespace comet {

// Order and prune a frontier's next batch on the device (comet_proposal_prune
// and the learned planner); capturable once the buffers are reserved.
comet_status proposal_prune_device(comet_proposal* q, comet_frontier* f, int keep, float* warm, int* row_scratch,
                                   cudaStream_t s) {
    FrontierDev& F = f->d;
    const int64_t cap = f->batch;
    features_kernel<<<grid_for(cap * q->in_dim), 256, 0, s>>>(F.next, cap, F.n_next, q->feat_inst, q->n_inst,
                                                              q->l_max, q->n_modes, q->in_dim, q->X, nullptr, 0, q->bim);
    QTRY(cudaGetLastError(), "features");
    QTRY(forward(q, cap, false, s), "forward");
    encode_kernel<<<grid_for(cap), 256, 0, s>>>(F.next, cap, F.n_next, q->n_modes, q->pr_codes);
    log_merit_kernel<<<grid_for(cap), 256, 0, s>>>(q->Y, q->out_dim, cap, F.n_next, q->pr_merit);
    QTRY(cudaGetLastError(), "scores");
    QTRY(cudaMemcpyAsync(q->pr_seqs, F.next, sizeof(comet_mode_seq) * cap, cudaMemcpyDeviceToDevice, s), "copy");
    FrontierDev R;
    memset(&R, 0, sizeof(R));
    R.codes = q->pr_codes;
    R.merit = q->pr_merit;
    R.nV = reinterpret_cast<unsigned long long*>(F.n_next);
    R.capacity = cap;
    R.top_a = q->pr_top_a;
    R.top_b = q->pr_top_b;
    cudaError_t e = cudaSuccess;
    const TopKey* top = launch_topk(R, keep, s, &e);
    if (!top) return qcuda(e, "rank");
    keep_kernel<<<grid_for(keep), 256, 0, s>>>(top, q->pr_seqs, F.n_next, keep, F.next, row_scratch);
    set_count_kernel<<<1, 32, 0, s>>>(F.n_next, keep);
    QTRY(cudaGetLastError(), "keep");
    if (warm) {
        predict_post_kernel<<<grid_for(keep, 128), 128, 0, s>>>(q->Y, q->out_dim, F.next, row_scratch, keep, F.n_next,
                                                                q->p->d_inst, q->n_inst, q->n_max,
                                                                q->desc.warm_mode, nullptr, warm, q->p->stride,
                                                                q->bim);
        QTRY(cudaGetLastError(), "warm starts");
    }
    return COMET_OK;
}

comet_status proposal_reserve_prune(comet_proposal* q, int64_t cap, int keep) {
    if (keep < 1 || keep > kChunk) return qfail(COMET_ERR_INVALID_ARG, "keep must be in [1, 4096]");
    QTRY(ensure_rows(q, cap), "proposal activations");
    QTRY(ensure_prune(q, cap), "prune buffers");
    return COMET_OK;
}

comet_problem* proposal_problem(const comet_proposal* q) { return q ? q->p : nullptr; }

// warm starts of the seed orders (device), rows in order
comet_status proposal_predict_device(comet_proposal* q, const comet_mode_seq* seqs, int64_t n, float* merit,
                                     float* warm, cudaStream_t s) {
    QTRY(ensure_rows(q, n), "proposal activations");
    features_kernel<<<grid_for(n * q->in_dim), 256, 0, s>>>(seqs, n, nullptr, q->feat_inst, q->n_inst, q->l_max,
                                                            q->n_modes, q->in_dim, q->X, nullptr, 0, q->bim);
    QTRY(cudaGetLastError(), "features");
    QTRY(forward(q, n, false, s), "forward");
    predict_post_kernel<<<grid_for(n, 128), 128, 0, s>>>(q->Y, q->out_dim, seqs, nullptr, n, nullptr, q->p->d_inst,
                                                         q->n_inst, q->n_max, q->desc.warm_mode, merit, warm,
                                                         q->p->stride, q->bim);
    QTRY(cudaGetLastError(), "predict");
    return COMET_OK;
}

}  // namespace comet

extern "C" {

void comet_default_proposal_desc(comet_proposal_desc* d) {
    if (!d) return;
    memset(d, 0, sizeof(*d));
    d->width = 256;
    d->rows_cap = 4096;
    d->dataset_cap = 0;
    d->seed = 1;
    d->lambda_w = 1.0;
    d->warm_mode = 1;
}

void comet_default_adamw_opts(comet_adamw_opts* o) {
    if (!o) return;
    o->lr = 1e-3;
    o->beta1 = 0.9;
    o->beta2 = 0.999;
    o->eps = 1e-8;
    o->weight_decay = 0.0;
}

comet_status comet_proposal_create(comet_problem* p, const comet_proposal_desc* d_in, comet_proposal** out) {
    if (!p || !out) return qfail(COMET_ERR_INVALID_ARG, "problem and out are required");
    *out = nullptr;
    comet_proposal_desc d;
    if (d_in)
        d = *d_in;
    else
        comet_default_proposal_desc(&d);
    if (d.width < 16 || d.width > 256 || d.width % 16 || d.rows_cap < 1 || d.dataset_cap < 0 ||
        (d.warm_mode != 0 && d.warm_mode != 1) || !(d.lambda_w >= 0))
        return qfail(COMET_ERR_INVALID_ARG, "bad proposal descriptor (width a multiple of 16 in [16, 256])");
    if (!comet::mlp::tensor_maps_available())
        return qfail(COMET_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    {
        cudaError_t ge = comet::mlp::gemm_prepare();
        if (ge == cudaSuccess) ge = comet::mlp::fused_prepare();
        if (ge != cudaSuccess) return qcuda(ge, "GEMM kernel attributes");
    }
    int l_max = 0, n_modes = 0;
    for (const auto& i : p->inst) {
        l_max = std::max(l_max, (int)i.max_segments);
        n_modes = std::max(n_modes, (int)i.n_modes);
    }
    comet_proposal* q = new comet_proposal();
    q->p = p;
    q->desc = d;
    q->l_max = l_max;
    q->n_modes = n_modes;
    q->n_max = p->Nmax;
    q->n_inst = (int)p->inst.size();
    q->bim = p->task == COMET_TASK_BIMANUAL ? 1 : 0;
    q->nx = q->bim ? 5 : 4;
    q->n_ctrl = q->bim ? 12 : 3;
    q->slot_w = q->bim ? kBimSlot : n_modes + 1;
    q->in_dim = (int)pad_to(kInstFeat + (int64_t)q->slot_w * l_max, 64);
    q->width = d.width;
    q->out_dim = (int)pad_to(1 + (int64_t)q->n_ctrl * p->Nmax, 16);
    const int dims[kLayers + 1] = {q->in_dim, q->width, q->width, q->width, q->out_dim};
    int64_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
        q->din[l] = dims[l];
        q->dout[l] = dims[l + 1];
        q->w_off[l] = off;
        off += (int64_t)dims[l] * dims[l + 1];
        q->b_off[l] = off;
        off += dims[l + 1];
    }
    q->n_params = off;
    auto cleanup = [&](comet_status st) {
        comet_proposal_destroy(q);
        return st;
    };
    cudaError_t e = cudaSuccess;
    cudaStream_t s = p->stream;
    if ((e = qalloc(q, &q->master, off)) != cudaSuccess || (e = qalloc(q, &q->grad, off)) != cudaSuccess ||
        (e = qalloc(q, &q->m1, off)) != cudaSuccess || (e = qalloc(q, &q->m2, off)) != cudaSuccess ||
        (e = qalloc(q, &q->feat_inst, (size_t)q->n_inst * kInstFeat)) != cudaSuccess ||
        (e = qalloc(q, &q->d_step, 1)) != cudaSuccess || (e = qalloc(q, &q->d_loss, 1)) != cudaSuccess ||
        (e = qalloc(q, &q->d_err, 1)) != cudaSuccess)
        return cleanup(qcuda(e, "proposal allocation"));
    for (int l = 0; l < kLayers; ++l)
        if ((e = qalloc(q, &q->wq[l], (size_t)q->din[l] * q->dout[l])) != cudaSuccess ||
            (e = qalloc(q, &q->wqt[l], (size_t)q->din[l] * q->dout[l])) != cudaSuccess)
            return cleanup(qcuda(e, "proposal allocation"));
    if ((e = ensure_rows(q, d.rows_cap)) != cudaSuccess) return cleanup(qcuda(e, "proposal activations"));
    if (d.dataset_cap > 0) {
        q->ds_cap = d.dataset_cap;
        if ((e = qalloc(q, &q->ds_X, (size_t)d.dataset_cap * q->in_dim)) != cudaSuccess ||
            (e = qalloc(q, &q->ds_T, (size_t)d.dataset_cap * q->out_dim)) != cudaSuccess ||
            (e = qalloc(q, &q->ds_Om, (size_t)d.dataset_cap * q->out_dim)) != cudaSuccess)
            return cleanup(qcuda(e, "proposal training set"));
    }
    std::vector<float> fi((size_t)q->n_inst * kInstFeat, 0.f);
    for (int i = 0; i < q->n_inst; ++i) {
        const comet_instance_desc& D = p->inst[i];
        float* f = fi.data() + (size_t)i * kInstFeat;
        for (int c = 0; c < 3; ++c) {
            f[c] = (float)D.start[c];
            f[3 + c] = (float)D.goal[c];
        }
        f[6] = (float)(10.0 * D.side_x);
        f[7] = (float)(10.0 * D.side_y);
        if (q->bim) {
            // the box in the vertical plane: 3 (g - s) for x and z (gravity
            // fixes the frame), dtheta, and the mass
            f[8] = (float)(3.0 * (D.goal[0] - D.start[0]));
            f[9] = (float)(3.0 * (D.goal[1] - D.start[1]));
            f[10] = (float)(D.goal[2] - D.start[2]);
            f[11] = (float)D.mass;
            continue;
        }
        // the goal in the start frame: 3 R(-theta_s)(g - s), dtheta
        const double dx = D.goal[0] - D.start[0], dy = D.goal[1] - D.start[1];
        const double c = cos(D.start[2]), sn = sin(D.start[2]);
        f[8] = (float)(3.0 * (c * dx + sn * dy));
        f[9] = (float)(3.0 * (-sn * dx + c * dy));
        f[10] = (float)(D.goal[2] - D.start[2]);
    }
    if ((e = cudaMemcpyAsync(q->feat_inst, fi.data(), sizeof(float) * fi.size(), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return cleanup(qcuda(e, "proposal init"));
    init_params_kernel<<<grid_for(off), 256, 0, s>>>(q->master, off, layer_tab(q), (unsigned long long)d.seed);
    quantize_kernel<<<grid_for(off), 256, 0, s>>>(q->master, off, layer_tab(q));
    if ((e = cudaGetLastError()) != cudaSuccess) return cleanup(qcuda(e, "proposal init"));
    cudaMemsetAsync(q->m1, 0, sizeof(float) * off, s);
    cudaMemsetAsync(q->m2, 0, sizeof(float) * off, s);
    cudaMemsetAsync(q->grad, 0, sizeof(float) * off, s);
    cudaMemsetAsync(q->d_step, 0, sizeof(int64_t), s);
    cudaMemsetAsync(q->d_err, 0, sizeof(int), s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cleanup(qcuda(e, "proposal init"));
    *out = q;
    return COMET_OK;
}

comet_status comet_proposal_destroy(comet_proposal* q) {
    if (!q) return COMET_OK;
    if (q->p) cudaStreamSynchronize(q->p->stream);
    for (void* v : q->allocs) cudaFree(v);
    delete q;
    return COMET_OK;
}

comet_status comet_proposal_dims(const comet_proposal* q, int32_t* in_dim, int32_t* width, int32_t* out_dim,
                                 int64_t* n_params) {
    if (!q) return qfail(COMET_ERR_INVALID_ARG, "proposal is NULL");
    if (in_dim) *in_dim = q->in_dim;
    if (width) *width = q->width;
    if (out_dim) *out_dim = q->out_dim;
    if (n_params) *n_params = q->n_params;
    return COMET_OK;
}

comet_status comet_proposal_set_params(comet_proposal* q, const float* flat) {
    if (!q || !flat) return qfail(COMET_ERR_INVALID_ARG, "proposal and params are required");
    cudaStream_t s = q->p->stream;
    QTRY(to_device(q->master, flat, sizeof(float) * q->n_params, s), "copy params");
    quantize_kernel<<<grid_for(q->n_params), 256, 0, s>>>(q->master, q->n_params, layer_tab(q));
    QTRY(cudaGetLastError(), "quantize");
    QTRY(cudaMemsetAsync(q->m1, 0, sizeof(float) * q->n_params, s), "reset");
    QTRY(cudaMemsetAsync(q->m2, 0, sizeof(float) * q->n_params, s), "reset");
    QTRY(cudaMemsetAsync(q->d_step, 0, sizeof(int64_t), s), "reset");
    QTRY(cudaStreamSynchronize(s), "synchronise");
    return COMET_OK;
}

// checkpoint file: this header, then the parameters, the two AdamW moments
// (n_params floats each, little-endian IEEE single)
struct ProposalCkpt {
    char magic[8];
    int32_t version, in_dim, width, out_dim, bim, reserved;
    int64_t n_params, step;
};
constexpr char kCkptMagic[8] = {'C', 'O', 'M', 'E', 'T', 'P', 'R', '1'};

comet_status comet_proposal_save(comet_proposal* q, const char* path) {
    if (!q || !path) return qfail(COMET_ERR_INVALID_ARG, "proposal and path are required");
    cudaStream_t s = q->p->stream;
    const size_t n = (size_t)q->n_params;
    std::vector<float> buf(3 * n);
    ProposalCkpt h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kCkptMagic, sizeof(h.magic));
    h.version = 1;
    h.in_dim = q->in_dim;
    h.width = q->width;
    h.out_dim = q->out_dim;
    h.bim = q->bim;
    h.n_params = q->n_params;
    QTRY(cudaMemcpyAsync(buf.data(), q->master, sizeof(float) * n, cudaMemcpyDeviceToHost, s), "copy params");
    QTRY(cudaMemcpyAsync(buf.data() + n, q->m1, sizeof(float) * n, cudaMemcpyDeviceToHost, s), "copy moments");
    QTRY(cudaMemcpyAsync(buf.data() + 2 * n, q->m2, sizeof(float) * n, cudaMemcpyDeviceToHost, s), "copy moments");
    QTRY(cudaMemcpyAsync(&h.step, q->d_step, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "copy step count");
    QTRY(cudaStreamSynchronize(s), "synchronise");
    FILE* f = fopen(path, "wb");
    if (!f) return qfail(COMET_ERR_INVALID_ARG, "checkpoint: cannot open the file for writing");
    const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    if (fclose(f) != 0 || !ok) return qfail(COMET_ERR_INVALID_ARG, "checkpoint: write failed");
    return COMET_OK;
}

comet_status comet_proposal_load(comet_proposal* q, const char* path) {
    if (!q || !path) return qfail(COMET_ERR_INVALID_ARG, "proposal and path are required");
    FILE* f = fopen(path, "rb");
    if (!f) return qfail(COMET_ERR_INVALID_ARG, "checkpoint: cannot open the file");
    ProposalCkpt h;
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, kCkptMagic, sizeof(h.magic)) != 0 || h.version != 1) {
        fclose(f);
        return qfail(COMET_ERR_INVALID_ARG, "checkpoint: not a proposal checkpoint");
    }
    if (h.in_dim != q->in_dim || h.width != q->width || h.out_dim != q->out_dim || h.bim != q->bim ||
        h.n_params != q->n_params || h.step < 0) {
        fclose(f);
        return qfail(COMET_ERR_INVALID_ARG, "checkpoint: the network's layout differs from this proposal's");
    }
    const size_t n = (size_t)q->n_params;
    std::vector<float> buf(3 * n);
    const bool ok = fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    if (!ok) return qfail(COMET_ERR_INVALID_ARG, "checkpoint: the file is truncated");
    cudaStream_t s = q->p->stream;
    QTRY(cudaMemcpyAsync(q->master, buf.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s), "copy params");
    QTRY(cudaMemcpyAsync(q->m1, buf.data() + n, sizeof(float) * n, cudaMemcpyHostToDevice, s), "copy moments");
    QTRY(cudaMemcpyAsync(q->m2, buf.data() + 2 * n, sizeof(float) * n, cudaMemcpyHostToDevice, s), "copy moments");
    QTRY(cudaMemcpyAsync(q->d_step, &h.step, sizeof(int64_t), cudaMemcpyHostToDevice, s), "copy step count");
    quantize_kernel<<<grid_for(q->n_params), 256, 0, s>>>(q->master, q->n_params, layer_tab(q));
    QTRY(cudaGetLastError(), "quantize");
    QTRY(cudaStreamSynchronize(s), "synchronise");
    return COMET_OK;
}

comet_status comet_proposal_get_params(comet_proposal* q, float* flat, float* grad) {
    if (!q) return qfail(COMET_ERR_INVALID_ARG, "proposal is NULL");
    cudaStream_t s = q->p->stream;
    if (flat) QTRY(cudaMemcpyAsync(flat, q->master, sizeof(float) * q->n_params, cudaMemcpyDefault, s), "copy");
    if (grad) QTRY(cudaMemcpyAsync(grad, q->grad, sizeof(float) * q->n_params, cudaMemcpyDefault, s), "copy");
    QTRY(cudaStreamSynchronize(s), "synchronise");
    return COMET_OK;
}

comet_status comet_proposal_features(comet_proposal* q, const comet_mode_seq* seqs, int64_t n, uint16_t* out_x) {
    if (!q || (n > 0 && (!seqs || !out_x))) return qfail(COMET_ERR_INVALID_ARG, "arguments are required");
    if (n <= 0) return COMET_OK;
    if (!qdev(out_x)) return qfail(COMET_ERR_INVALID_ARG, "out_x must be device memory");
    cudaStream_t s = q->p->stream;
    const comet_mode_seq* d = seqs;
    void* tmp = nullptr;
    if (!qdev(seqs)) {
        for (int64_t i = 0; i < n; ++i)
            if (seqs[i].instance < 0 || seqs[i].instance >= q->n_inst || seqs[i].len < 1 || seqs[i].len > q->l_max)
                return qfail(COMET_ERR_INVALID_ARG, "malformed order");
        QTRY(cudaMalloc(&tmp, sizeof(comet_mode_seq) * n), "staging");
        QTRY(cudaMemcpyAsync(tmp, seqs, sizeof(comet_mode_seq) * n, cudaMemcpyHostToDevice, s), "copy orders");
        d = (const comet_mode_seq*)tmp;
    }
    features_kernel<<<grid_for(n * q->in_dim), 256, 0, s>>>(d, n, nullptr, q->feat_inst, q->n_inst, q->l_max,
                                                            q->n_modes, q->in_dim, out_x, nullptr, 0, q->bim);
    cudaError_t e = cudaGetLastError();
    if (tmp) {
        cudaStreamSynchronize(s);
        cudaFree(tmp);
    }
    if (e != cudaSuccess) return qcuda(e, "features");
    return COMET_OK;
}

comet_status comet_proposal_forward(comet_proposal* q, const uint16_t* x, int64_t n, float* out_y) {
    if (!q || (n > 0 && (!x || !out_y))) return qfail(COMET_ERR_INVALID_ARG, "arguments are required");
    if (n <= 0) return COMET_OK;
    cudaStream_t s = q->p->stream;
    QTRY(ensure_rows(q, n), "proposal activations");
    QTRY(to_device(q->X, x, sizeof(uint16_t) * n * q->in_dim, s), "copy x");
    QTRY(cudaMemsetAsync(q->d_err, 0, sizeof(int), s), "reset");
    QTRY(forward(q, n, false, s), "forward");
    QTRY(cudaMemcpyAsync(out_y, q->Y, sizeof(float) * n * q->out_dim, cudaMemcpyDefault, s), "copy y");
    return check_err(q, s);
}

comet_status comet_proposal_time_forward(comet_proposal* q, const uint16_t* x, int64_t n, int32_t reps,
                                         float* out_ms) {
    if (!q || !x || n < 1 || reps < 1 || !out_ms) return qfail(COMET_ERR_INVALID_ARG, "arguments are required");
    cudaStream_t s = q->p->stream;
    QTRY(ensure_rows(q, n), "proposal activations");
    QTRY(to_device(q->X, x, sizeof(uint16_t) * n * q->in_dim, s), "copy x");
    QTRY(cudaMemsetAsync(q->d_err, 0, sizeof(int), s), "reset");
    QTRY(forward(q, n, false, s), "forward");  // warm
    cudaEvent_t e0, e1;
    QTRY(cudaEventCreate(&e0), "event");
    QTRY(cudaEventCreate(&e1), "event");
    cudaError_t e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = forward(q, n, false, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return qcuda(e, "timed forward");
    *out_ms = ms / (float)reps;
    return check_err(q, s);
}

comet_status comet_proposal_train_batch(comet_proposal* q, const uint16_t* x, const float* target,
                                        const float* weight, int64_t n, const comet_adamw_opts* o_in,
                                        float* out_loss) {
    if (!q || n < 1 || !x || !target || !weight) return qfail(COMET_ERR_INVALID_ARG, "arguments are required");
    comet_adamw_opts o;
    if (o_in)
        o = *o_in;
    else
        comet_default_adamw_opts(&o);
    cudaStream_t s = q->p->stream;
    QTRY(ensure_rows(q, n), "proposal activations");
    QTRY(to_device(q->X, x, sizeof(uint16_t) * n * q->in_dim, s), "copy x");
    QTRY(to_device(q->T, target, sizeof(float) * n * q->out_dim, s), "copy target");
    QTRY(to_device(q->Om, weight, sizeof(float) * n * q->out_dim, s), "copy weight");
    // X^T for the first layer's weight gradient
    transpose_kernel<<<grid_for(n * q->in_dim), 256, 0, s>>>(q->X, n, q->in_dim, q->Xt, q->ld_t);
    QTRY(cudaGetLastError(), "transpose");
    QTRY(cudaMemsetAsync(q->d_err, 0, sizeof(int), s), "reset");
    QTRY(cudaMemsetAsync(q->d_loss, 0, sizeof(float), s), "reset");
    QTRY(forward(q, n, true, s), "forward");
    QTRY(backward_update(q, n, o, s), "backward");
    if (out_loss) QTRY(cudaMemcpyAsync(out_loss, q->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s), "loss");
    return check_err(q, s);
}

comet_status comet_proposal_add_samples(comet_proposal* q, const comet_mode_seq* seqs, int64_t n, const float* cost,
                                        const float* viol, const int32_t* status, const float* traj) {
    if (!q || n < 0 || (n > 0 && (!seqs || !cost || !viol || !status || !traj)))
        return qfail(COMET_ERR_INVALID_ARG, "arguments are required");
    if (n == 0) return COMET_OK;
    if (q->ds_n + n > q->ds_cap) return qfail(COMET_ERR_BUDGET, "training set is full");
    cudaStream_t s = q->p->stream;
    const int64_t stride = q->p->stride;
    const bool dev = qdev(seqs);
    if (dev != qdev(cost) || dev != qdev(viol) || dev != qdev(status) || dev != qdev(traj))
        return qfail(COMET_ERR_INVALID_ARG, "pass all device or all host buffers");
    void* tmp = nullptr;
    const comet_mode_seq* ds = seqs;
    const float *dc = cost, *dv = viol, *dt = traj;
    const int32_t* dst = status;
    if (!dev) {
        const size_t b_seq = sizeof(comet_mode_seq) * n, b_f = sizeof(float) * n, b_t = sizeof(float) * n * stride;
        QTRY(cudaMalloc(&tmp, b_seq + 3 * b_f + b_t + 1024), "staging");
        char* b = (char*)tmp;
        ds = (const comet_mode_seq*)b;
        dc = (const float*)(b + pad_to(b_seq, 256));
        dv = (const float*)(b + pad_to(b_seq, 256) + pad_to(b_f, 256));
        dst = (const int32_t*)(b + pad_to(b_seq, 256) + 2 * pad_to(b_f, 256));
        dt = (const float*)(b + pad_to(b_seq, 256) + 3 * pad_to(b_f, 256));
        cudaMemcpyAsync((void*)ds, seqs, b_seq, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync((void*)dc, cost, b_f, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync((void*)dv, viol, b_f, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync((void*)dst, status, b_f, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync((void*)dt, traj, b_t, cudaMemcpyHostToDevice, s);
    }
    // per-instance knots per segment
    std::vector<int> K(q->n_inst);
    for (int i = 0; i < q->n_inst; ++i) K[i] = q->p->inst[i].knots_per_segment;
    int* dK = nullptr;
    cudaError_t e = cudaMalloc(&dK, sizeof(int) * q->n_inst);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dK, K.data(), sizeof(int) * q->n_inst, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        features_kernel<<<grid_for(n * q->in_dim), 256, 0, s>>>(ds, n, nullptr, q->feat_inst, q->n_inst, q->l_max,
                                                                q->n_modes, q->in_dim,
                                                                q->ds_X + q->ds_n * q->in_dim, nullptr, 0, q->bim);
        targets_kernel<<<grid_for(n * q->out_dim), 256, 0, s>>>(
            ds, n, dc, dv, dst, dt, stride, dK, q->n_inst, q->n_max, q->out_dim, (float)q->p->opts.merit_mu,
            (float)q->p->opts.eps_feas, (float)q->desc.lambda_w, q->ds_T + q->ds_n * q->out_dim,
            q->ds_Om + q->ds_n * q->out_dim, q->nx, q->n_ctrl, q->bim, q->p->d_inst);
        e = cudaGetLastError();
    }
    cudaStreamSynchronize(s);
    cudaFree(dK);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return qcuda(e, "add samples");
    q->ds_n += n;
    return COMET_OK;
}

comet_status comet_proposal_dataset_size(comet_proposal* q, int64_t* n) {
    if (!q || !n) return qfail(COMET_ERR_INVALID_ARG, "arguments are required");
    *n = q->ds_n;
    return COMET_OK;
}

comet_status comet_proposal_dataset_rows(comet_proposal* q, int64_t first, int64_t n, uint16_t* out_x,
                                         float* out_t, float* out_w) {
    if (!q || first < 0 || n < 0 || first + n > q->ds_n) return qfail(COMET_ERR_INVALID_ARG, "rows out of range");
    cudaStream_t s = q->p->stream;
    if (n > 0 && out_x)
        QTRY(cudaMemcpyAsync(out_x, q->ds_X + first * q->in_dim, sizeof(uint16_t) * n * q->in_dim, cudaMemcpyDefault,
                             s),
             "copy");
    if (n > 0 && out_t)
        QTRY(cudaMemcpyAsync(out_t, q->ds_T + first * q->out_dim, sizeof(float) * n * q->out_dim, cudaMemcpyDefault,
                             s),
             "copy");
    if (n > 0 && out_w)
        QTRY(cudaMemcpyAsync(out_w, q->ds_Om + first * q->out_dim, sizeof(float) * n * q->out_dim,
                             cudaMemcpyDefault, s),
             "copy");
    QTRY(cudaStreamSynchronize(s), "synchronise");
    return COMET_OK;
}

comet_status comet_proposal_train(comet_proposal* q, int64_t steps, int32_t batch, const comet_adamw_opts* o_in,
                                  uint64_t seed, float* out_loss) {
    if (!q || steps < 0 || batch < 1) return qfail(COMET_ERR_INVALID_ARG, "bad arguments");
    if (q->ds_n < 1) return qfail(COMET_ERR_INVALID_ARG, "training set is empty");
    if (steps == 0) return COMET_OK;
    comet_adamw_opts o;
    if (o_in)
        o = *o_in;
    else
        comet_default_adamw_opts(&o);
    QTRY(ensure_rows(q, batch), "proposal activations");
    // private stream: a graph cannot be captured on the legacy stream
    cudaStream_t user = q->p->stream, s = nullptr;
    QTRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, user);
    cudaStreamWaitEvent(s, ev, 0);
    float* d_losses = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    comet_status st = COMET_OK;
    cudaError_t e = cudaMalloc(&d_losses, sizeof(float) * steps);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->d_err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t ce = cudaMemsetAsync(q->d_loss, 0, sizeof(float), s);
        if (ce == cudaSuccess) {
            gather_kernel<<<grid_for((int64_t)batch * (q->in_dim + q->out_dim)), 256, 0, s>>>(
                q->ds_X, q->ds_T, q->ds_Om, q->ds_n, batch, q->d_step, (unsigned long long)seed, q->in_dim,
                q->out_dim, q->X, q->Xt, q->ld_t, q->T, q->Om);
            ce = cudaGetLastError();
        }
        if (ce == cudaSuccess) ce = forward(q, batch, true, s);
        if (ce == cudaSuccess) ce = backward_update(q, batch, o, s);
        e = cudaStreamEndCapture(s, &graph);
        if (ce != cudaSuccess) e = ce;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    for (int64_t i = 0; i < steps && e == cudaSuccess; ++i) {
        e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_losses + i, q->d_loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess && out_loss)
        e = cudaMemcpyAsync(out_loss, d_losses, sizeof(float) * steps, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = qcuda(e, "train");
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaFree(d_losses);
    cudaEventRecord(ev, s);
    cudaStreamWaitEvent(user, ev, 0);
    cudaStreamSynchronize(s);
    cudaEventDestroy(ev);
    cudaStreamDestroy(s);
    if (st != COMET_OK) return st;
    return check_err(q, user);
}

comet_status comet_proposal_predict(comet_proposal* q, const comet_mode_seq* seqs, int64_t n, float* out_merit,
                                    float* out_warm) {
    if (!q || n < 0 || (n > 0 && !seqs)) return qfail(COMET_ERR_INVALID_ARG, "arguments are required");
    if (n == 0) return COMET_OK;
    cudaStream_t s = q->p->stream;
    const int64_t stride = q->p->stride;
    const bool host_seqs = !qdev(seqs);
    const bool host_m = out_merit && !qdev(out_merit);
    const bool host_w = out_warm && !qdev(out_warm);
    if (host_seqs)
        for (int64_t i = 0; i < n; ++i)
            if (seqs[i].instance < 0 || seqs[i].instance >= q->n_inst || seqs[i].len < 1 || seqs[i].len > q->l_max)
                return qfail(COMET_ERR_INVALID_ARG, "malformed order");
    void* tmp = nullptr;
    const size_t b_seq = pad_to(sizeof(comet_mode_seq) * n, 256), b_m = pad_to(sizeof(float) * n, 256);
    QTRY(cudaMalloc(&tmp, b_seq + b_m + sizeof(float) * n * stride + 256), "staging");
    char* b = (char*)tmp;
    const comet_mode_seq* ds = host_seqs ? (const comet_mode_seq*)b : seqs;
    float* dm = out_merit ? (host_m ? (float*)(b + b_seq) : out_merit) : nullptr;
    float* dw = out_warm ? (host_w ? (float*)(b + b_seq + b_m) : out_warm) : nullptr;
    cudaError_t e = cudaSuccess;
    if (host_seqs) e = cudaMemcpyAsync((void*)ds, seqs, sizeof(comet_mode_seq) * n, cudaMemcpyHostToDevice, s);
    QTRY(cudaMemsetAsync(q->d_err, 0, sizeof(int), s), "reset");
    comet_status st = COMET_OK;
    if (e == cudaSuccess) st = comet::proposal_predict_device(q, ds, n, dm, dw, s);
    if (st == COMET_OK && e == cudaSuccess && host_m)
        e = cudaMemcpyAsync(out_merit, dm, sizeof(float) * n, cudaMemcpyDeviceToHost, s);
    if (st == COMET_OK && e == cudaSuccess && host_w)
        e = cudaMemcpyAsync(out_warm, dw, sizeof(float) * n * stride, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    cudaFree(tmp);
    if (st != COMET_OK) return st;
    if (e != cudaSuccess) return qcuda(e, "predict");
    return check_err(q, s);
}

comet_status comet_proposal_prune(comet_proposal* q, comet_frontier* f, int32_t keep, float* out_warm) {
    if (!q || !f || f->p != q->p) return qfail(COMET_ERR_INVALID_ARG, "proposal / frontier mismatch");
    if (out_warm && !qdev(out_warm)) return qfail(COMET_ERR_INVALID_ARG, "out_warm must be device memory");
    comet_status st = comet::proposal_reserve_prune(q, f->batch, keep);
    if (st != COMET_OK) return st;
    cudaStream_t s = q->p->stream;
    int* rows = nullptr;
    QTRY(cudaMalloc(&rows, sizeof(int) * keep), "scratch");
    QTRY(cudaMemsetAsync(q->d_err, 0, sizeof(int), s), "reset");
    st = comet::proposal_prune_device(q, f, keep, out_warm, rows, s);
    cudaStreamSynchronize(s);
    cudaFree(rows);
    if (st != COMET_OK) return st;
    return check_err(q, s);
}

comet_status comet_gemm_bf16(const uint16_t* a, int64_t lda, const uint16_t* b, int64_t ldb, int64_t m, int32_t n,
                             int32_t k, const comet_gemm_epilogue* ep, void* cuda_stream) {
    using namespace comet::mlp;
    if (!a || !b || !ep || m < 0 || n < 0 || k < 1) return qfail(COMET_ERR_INVALID_ARG, "bad GEMM arguments");
    if (!tensor_maps_available()) return qfail(COMET_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    if (!qdev(a) || !qdev(b)) return qfail(COMET_ERR_INVALID_ARG, "GEMM operands must be device memory");
    if (ep->kind < 0 || ep->kind > 3) return qfail(COMET_ERR_INVALID_ARG, "unknown epilogue");
    if ((ep->kind == COMET_GEMM_STORE || ep->kind == COMET_GEMM_ATOMIC_ADD) && !ep->out_f32)
        return qfail(COMET_ERR_INVALID_ARG, "out_f32 is required");
    if ((ep->kind == COMET_GEMM_BIAS_GELU || ep->kind == COMET_GEMM_GELU_GRAD) && !ep->out_bf16 && !ep->out_bf16_t &&
        !ep->out_f32)
        return qfail(COMET_ERR_INVALID_ARG, "an output is required");
    if (ep->kind == COMET_GEMM_GELU_GRAD && !ep->z_in) return qfail(COMET_ERR_INVALID_ARG, "z_in is required");
    int* d_err = nullptr;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    QTRY(cudaMalloc(&d_err, sizeof(int)), "flag");
    cudaMemsetAsync(d_err, 0, sizeof(int), s);
    Epilogue e;
    e.kind = ep->kind;
    e.bias = ep->bias;
    e.out_f32 = ep->out_f32;
    e.ld_out = ep->ld_f32;
    e.h = ep->out_bf16;
    e.ld_h = ep->ld_bf16;
    e.h_t = ep->out_bf16_t;
    e.ld_ht = ep->ld_bf16_t;
    e.z_in = ep->z_in;
    e.ld_z = ep->ld_z;
    e.err = d_err;
    const Mat A{a, m, k, lda}, B{b, n, k, ldb};
    const cudaError_t ce = gemm_bf16(A, B, m, n, k, std::max(1, ep->k_splits), e, s);
    int err = 0;
    cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    cudaFree(d_err);
    if (ce != cudaSuccess) return qcuda(ce, "GEMM launch");
    if (err) return qfail(COMET_ERR_TIMEOUT, "tensor-core GEMM: a bounded wait ran out");
    return COMET_OK;
}

}  // extern "C"
