// BF16 GEMM on the 5th-generation tensor cores for the learned proposal.
//
//   D[M][N] = A[M][K] . B[N][K]^T   (bf16 operands, FP32 accumulation)
//
// One CTA computes a 128 x BN tile (BN <= 64) over its share of K:
//   * warp 0, one lane: TMA producer.  Tiles of 64 K-elements (128 bytes
//     per row, the 128-byte swizzle span) of A and B are copied into a
//     4-stage shared-memory ring; each stage's full barrier counts the bytes.
//   * warp 1, one lane: MMA issuer.  Four tcgen05.mma (kind::f16, K = 16)
//     per stage accumulate into TMEM (128 lanes x BN FP32 columns); a
//     tcgen05.commit frees the stage and, after the last, signals the
//     accumulator barrier.
//   * warp 2 allocates and frees the TMEM columns.
//   * all four warps: epilogue.  Warp w reads TMEM lanes 32w..32w+31 (rows
//     of the tile) 32 columns at a time with tcgen05.ld, turns each 32 x 32
//     block around in shared memory and applies the fused epilogue (bias,
//     GELU, GELU' gating, BF16 conversion, the transposed copy the
//     weight-gradient GEMM consumes, or split-K atomics) with coalesced
//     stores.
//
// Every mbarrier wait is bounded (about one second of clock cycles); when
// one runs out the CTA records the failure in the error flag, skips the rest
// of its work, waits (bounded) for the copies it issued and frees its TMEM.
#include "mlp_internal.h"

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

namespace comet {
namespace mlp {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;           // bf16 elements per 128-byte swizzle row
constexpr int kStages = 4;
constexpr int kThreads = 128;
constexpr int kMaxBN = 64;  // column tile: more CTAs for the small GEMMs of the MLP
constexpr long long kWaitCycles = 2000000000ll;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
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

// Bounded wait for the phase of the given parity; false if it ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored as rows
// of 128 bytes with the 128-byte swizzle (the layout TMA writes with
// CU_TENSOR_MAP_SWIZZLE_128B): 8-row groups 1024 bytes apart (stride byte
// offset), leading byte offset unused, descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint16_t to_bf16(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// GELU in the tanh form of Hendrycks and Gimpel,
//   0.5 x (1 + tanh(a (x + b x^3))), a = sqrt(2 / pi), b = 0.044715,
// with the hardware tanh approximation (relative error about 2^-11, below
// the BF16 rounding of the stored activations)
__device__ __forceinline__ float tanh_hw(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float kGeluA = 0.79788456080286536f;  // sqrt(2 / pi)
constexpr float kGeluB = 0.044715f;

__device__ __forceinline__ float gelu_f(float x) {
    const float t = tanh_hw(kGeluA * (x + kGeluB * x * x * x));
    return 0.5f * x * (1.f + t);
}

__device__ __forceinline__ float gelu_grad_f(float x) {
    const float t = tanh_hw(kGeluA * (x + kGeluB * x * x * x));
    return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * kGeluA * (1.f + 3.f * kGeluB * x * x);
}

struct __align__(8) Barriers {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t accum;
    uint32_t tmem_base;
    uint32_t failed;
};

__global__ void __launch_bounds__(kThreads, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, int M,
                     int N, int K, int k_chunk, int bn, int tmem_cols, Epilogue ep) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    const uint32_t a_bytes = BM * BK * 2;
    const uint32_t b_bytes = (uint32_t)bn * BK * 2;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    Barriers* bars = reinterpret_cast<Barriers*>(smem + kStages * stage_bytes);
    const uint32_t s_base = smem_u32(smem);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * bn;
    const int k_begin = blockIdx.z * k_chunk;
    const int k_len = min(k_chunk, K - k_begin);
    const int nkb = (k_len + BK - 1) / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&bars->full[s]), 1);
            mbar_init(smem_u32(&bars->empty[s]), 1);
        }
        mbar_init(smem_u32(&bars->accum), 1);
        bars->failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&bars->tmem_base)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars->tmem_base;

    if (warp == 0 && lane == 0) {
        // ---- producer
        int issued = 0;
        for (int i = 0; i < nkb; ++i) {
            const int s = i % kStages;
            const uint32_t ph = (uint32_t)(i / kStages) & 1u;
            if (i >= kStages && !mbar_wait(smem_u32(&bars->empty[s]), ph ^ 1u)) {
                atomicExch(&bars->failed, 1u);
                break;
            }
            if (*(volatile uint32_t*)&bars->failed) break;
            const uint32_t full = smem_u32(&bars->full[s]);
            mbar_expect_tx(full, stage_bytes);
            const int kx = k_begin + i * BK;
            tma_load_2d(s_base + s * stage_bytes, &map_a, kx, m0, full);
            tma_load_2d(s_base + s * stage_bytes + a_bytes, &map_b, kx, n0, full);
            ++issued;
        }
        if (*(volatile uint32_t*)&bars->failed) {
            // wait (bounded) for the copies still in flight before the CTA
            // can release its shared memory
            for (int i = (issued > kStages ? issued - kStages : 0); i < issued; ++i)
                mbar_wait(smem_u32(&bars->full[i % kStages]), (uint32_t)(i / kStages) & 1u);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = instr_desc(BM, bn);
        bool ok = true;
        for (int i = 0; i < nkb && ok; ++i) {
            const int s = i % kStages;
            const uint32_t ph = (uint32_t)(i / kStages) & 1u;
            if (!mbar_wait(smem_u32(&bars->full[s]), ph)) {
                atomicExch(&bars->failed, 1u);
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t a = s_base + s * stage_bytes, b = a + a_bytes;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(tmem, smem_desc(a + kk * 32), smem_desc(b + kk * 32), idesc, (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(smem_u32(&bars->empty[s]));
        }
        mma_commit(smem_u32(&bars->accum));
    }
    __syncwarp();

    // ---- epilogue: all warps
    const bool have = mbar_wait(smem_u32(&bars->accum), 0);
    if (!have) atomicExch(&bars->failed, 1u);
    tc_fence_after();
    __syncwarp();
    const bool run = __all_sync(0xffffffffu, have && !*(volatile uint32_t*)&bars->failed);
    // Each 32 x 32 block of the accumulator goes through shared memory (the
    // pipeline stages are free once the accumulator is complete), so that
    // row-major outputs are written with lanes along a row and the
    // transposed copy with lanes along a column: every store is coalesced.
    // Warp w stages in its own two 32 x 33 tiles (raw accumulator, result).
    if (run) {
        float* st1 = reinterpret_cast<float*>(smem) + warp * (2 * 32 * 33);
        float* st2 = st1 + 32 * 33;
        const int row0 = m0 + warp * 32;
        for (int c0 = 0; c0 < bn; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            const int nb = n0 + c0;
            if (nb >= N) continue;
#pragma unroll
            for (int j = 0; j < 32; ++j) st1[lane * 33 + j] = v[j];
            __syncwarp();
            // lanes along a row: column nb + lane
            const int col = nb + lane;
            const bool col_ok = col < N;
            const float bias = (ep.bias && col_ok) ? ep.bias[col] : 0.f;
            for (int r = 0; r < 32; ++r) {
                const int row = row0 + r;
                const bool ok = col_ok && row < M;
                const float a = st1[r * 33 + lane];
                float res = 0.f;
                if (ep.kind == kEpiStore) {
                    if (ok) ep.out_f32[(int64_t)row * ep.ld_out + col] = a + bias;
                } else if (ep.kind == kEpiAtomicAdd) {
                    if (ok) atomicAdd(ep.out_f32 + (int64_t)row * ep.ld_out + col, a);
                } else if (ep.kind == kEpiBiasGelu) {
                    const float z = a + bias;
                    if (ok && ep.out_f32) ep.out_f32[(int64_t)row * ep.ld_out + col] = z;
                    res = gelu_f(z);
                } else {  // kEpiGeluGrad
                    const float z = ok ? ep.z_in[(int64_t)row * ep.ld_z + col] : 0.f;
                    res = a * gelu_grad_f(z);
                }
                if (ep.kind == kEpiBiasGelu || ep.kind == kEpiGeluGrad) {
                    const uint16_t hb = to_bf16(res);
                    if (ok && ep.h) ep.h[(int64_t)row * ep.ld_h + col] = hb;
                    st2[r * 33 + lane] = __uint_as_float((uint32_t)hb);
                }
            }
            __syncwarp();
            if (ep.h_t && (ep.kind == kEpiBiasGelu || ep.kind == kEpiGeluGrad)) {
                // lanes along a column of the transposed copy: row row0 + lane
                const int row = row0 + lane;
                if (row < M) {
                    const int nv = min(32, N - nb);
                    for (int j = 0; j < nv; ++j)
                        ep.h_t[(int64_t)(nb + j) * ep.ld_ht + row] = (uint16_t)__float_as_uint(st2[lane * 33 + j]);
                }
            }
            __syncwarp();
        }
    }
    if (*(volatile uint32_t*)&bars->failed && threadIdx.x == 0 && ep.err) atomicExch(ep.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// ------------------------------------------------------------------------
// Fused forward pass of the 4-layer MLP (in_dim <= 128, width 256, out_dim
// <= 256): one persistent CTA per SM walks 128-row tiles; the four layers
// are chained through one 256-column TMEM accumulator and a 64 KB
// activation tile in shared memory, so a tile never leaves the SM between
// layers.  Warps 0..15: epilogue (warp w reads TMEM lanes 32 (w mod 4).. and
// columns 64 (w / 4)..), writing bias + GELU as BF16 into the activation
// tile in the 128-byte-swizzled K-major layout the next tcgen05.mma reads
// (16-byte chunk c of row r at chunk c ^ (r mod 8)); warp 16, one lane: TMA
// producer (the X tile, and the weights as 64-column K slices of 256 rows
// through a 3-stage ring); warp 17, one lane: MMA issuer.

constexpr int kFEpiWarps = 16;
constexpr int kFThreads = (kFEpiWarps + 2) * 32;
constexpr int kFEpilogue = kFEpiWarps * 32;  // threads of the epilogue warps
constexpr int kFRing = 3;
constexpr uint32_t kWStage = 256 * BK * 2;   // 32 KB: one K slice of a weight
constexpr uint32_t kXBlock = BM * BK * 2;    // 16 KB: one K slice of a tile

struct __align__(8) FusedBars {
    uint64_t x_full, x_free, acc_full, h_ready;
    uint64_t w_full[kFRing], w_empty[kFRing];
    uint32_t tmem_base, failed;
};

struct FusedParams {
    const float* bias[4];
    float* y;
    int64_t ld_y;
    int M, in_dim, out_dim;
    int* err;
};

__global__ void __launch_bounds__(kFThreads, 1)
    mlp_fused_forward_kernel(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_w0,
                             const __grid_constant__ CUtensorMap map_w1, const __grid_constant__ CUtensorMap map_w2,
                             const __grid_constant__ CUtensorMap map_w3, FusedParams fp) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    const int n_xkb = fp.in_dim / BK;                       // 1 or 2 K slices of X
    uint8_t* xs = smem;                                     // n_xkb x 16 KB
    uint8_t* hs = xs + 2 * kXBlock;                         // 4 x 16 KB activations
    uint8_t* ws = hs + 4 * kXBlock;                         // kFRing x 32 KB weights
    float* bs = reinterpret_cast<float*>(ws + kFRing * kWStage);  // 4 x 256 biases
    FusedBars* bars = reinterpret_cast<FusedBars*>(bs + 4 * 256);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (fp.M + BM - 1) / BM;
    const int kb_layer[4] = {n_xkb, 4, 4, 4};
    const CUtensorMap* wmap[4] = {&map_w0, &map_w1, &map_w2, &map_w3};

    for (int t = threadIdx.x; t < 4 * 256; t += kFThreads) {
        const int l = t >> 8, c = t & 255;
        bs[t] = (l < 3 || c < fp.out_dim) ? fp.bias[l][c] : 0.f;
    }
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bars->x_full), 1);
        mbar_init(smem_u32(&bars->x_free), 1);
        mbar_init(smem_u32(&bars->acc_full), 1);
        mbar_init(smem_u32(&bars->h_ready), kFEpilogue);
        for (int s = 0; s < kFRing; ++s) {
            mbar_init(smem_u32(&bars->w_full[s]), 1);
            mbar_init(smem_u32(&bars->w_empty[s]), 1);
        }
        bars->failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&bars->tmem_base)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    volatile uint32_t* failed = &bars->failed;

    if (warp == kFEpiWarps) {
        if (lane == 0) {
            // ---- producer
            uint32_t g = 0;  // weight slices issued
            int it = 0;
            for (int tile = blockIdx.x; tile < n_tiles && !*failed; tile += gridDim.x, ++it) {
                if (it > 0 && !mbar_wait(smem_u32(&bars->x_free), (uint32_t)(it - 1) & 1u)) {
                    atomicExch(&bars->failed, 1u);
                    break;
                }
                const uint32_t xb = smem_u32(&bars->x_full);
                mbar_expect_tx(xb, (uint32_t)n_xkb * kXBlock);
                for (int kb = 0; kb < n_xkb; ++kb)
                    tma_load_2d(smem_u32(xs) + kb * kXBlock, &map_x, kb * BK, tile * BM, xb);
                for (int l = 0; l < 4 && !*failed; ++l)
                    for (int kb = 0; kb < kb_layer[l]; ++kb, ++g) {
                        const int s = (int)(g % kFRing);
                        const uint32_t use = g / kFRing;
                        if (g >= (uint32_t)kFRing && !mbar_wait(smem_u32(&bars->w_empty[s]), (use & 1u) ^ 1u)) {
                            atomicExch(&bars->failed, 1u);
                            break;
                        }
                        const uint32_t fb = smem_u32(&bars->w_full[s]);
                        mbar_expect_tx(fb, kWStage);
                        tma_load_2d(smem_u32(ws) + s * kWStage, wmap[l], kb * BK, 0, fb);
                    }
            }
        }
    } else if (warp == kFEpiWarps + 1) {
        if (lane == 0) {
            // ---- MMA issuer
            const uint32_t idesc = instr_desc(BM, 256);
            uint32_t g = 0, L = 0;
            int it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++it) {
                if (!mbar_wait(smem_u32(&bars->x_full), (uint32_t)it & 1u)) {
                    ok = false;
                    break;
                }
                for (int l = 0; l < 4 && ok; ++l, ++L) {
                    // the accumulator is free and the activations of the
                    // previous layer are in place
                    if (L > 0 && !mbar_wait(smem_u32(&bars->h_ready), (L - 1) & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int kb = 0; kb < kb_layer[l] && ok; ++kb, ++g) {
                        const int s = (int)(g % kFRing);
                        if (!mbar_wait(smem_u32(&bars->w_full[s]), (g / kFRing) & 1u)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a = (l == 0 ? smem_u32(xs) : smem_u32(hs)) + kb * kXBlock;
                        const uint32_t b = smem_u32(ws) + s * kWStage;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            mma_bf16(tmem, smem_desc(a + kk * 32), smem_desc(b + kk * 32), idesc,
                                     (kb > 0 || kk > 0) ? 1u : 0u);
                        mma_commit(smem_u32(&bars->w_empty[s]));
                    }
                    mma_commit(smem_u32(&bars->acc_full));
                    if (l == 0) mma_commit(smem_u32(&bars->x_free));
                }
            }
            if (!ok) {
                // unblock the epilogue warps: they see the flag and stop (in
                // the normal case every accumulator phase is committed exactly
                // once, so that each epilogue wait sees its own phase)
                atomicExch(&bars->failed, 1u);
                mma_commit(smem_u32(&bars->acc_full));
            }
        }
    } else {
        // ---- epilogue warps: row r = 32 (warp mod 4) + lane of the tile,
        // a band of 256 / (kFEpiWarps / 4) columns
        constexpr int kBand = 256 / (kFEpiWarps / 4);
        const int quarter = warp & 3, part = warp >> 2;
        const int r = quarter * 32 + lane;
        uint32_t L = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
            bool stop = false;
            for (int l = 0; l < 4; ++l, ++L) {
                const bool have = mbar_wait(smem_u32(&bars->acc_full), L & 1u);
                if (!have) atomicExch(&bars->failed, 1u);
                if (__any_sync(0xffffffffu, !have || *failed)) {
                    stop = true;
                    break;
                }
                tc_fence_after();
                const int ncol = (l == 3) ? fp.out_dim : 256;
                for (int c0 = kBand * part; c0 < kBand * part + kBand; c0 += 32) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
                    if (c0 >= ncol) continue;
                    const float* bias = bs + 256 * l;
                    if (l < 3) {
                        // 32 BF16 = 64 bytes = four 16-byte chunks of row r of
                        // K slice c0 / 64, placed by the 128-byte swizzle
                        uint32_t pk[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float a0 = gelu_f(v[2 * j] + bias[c0 + 2 * j]);
                            const float a1 = gelu_f(v[2 * j + 1] + bias[c0 + 2 * j + 1]);
                            pk[j] = (uint32_t)to_bf16(a0) | ((uint32_t)to_bf16(a1) << 16);
                        }
                        uint8_t* blk = hs + (c0 / 64) * kXBlock + r * 128;
                        const int ch0 = ((c0 % 64) * 2) / 16;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int pc = (ch0 + q) ^ (r & 7);
                            *reinterpret_cast<uint4*>(blk + pc * 16) =
                                make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
                        }
                    } else {
                        // turn the 32 x 32 block around in this warp's 4 KB of
                        // the (now free) activation tile, XOR-swizzled, so that
                        // each store writes 32 consecutive floats of one row
                        float* tb = reinterpret_cast<float*>(hs) + warp * 1024;
#pragma unroll
                        for (int j = 0; j < 32; ++j) tb[lane * 32 + (j ^ lane)] = v[j] + bias[c0 + j];
                        __syncwarp();
                        const int row0 = tile * BM + quarter * 32, col = c0 + lane;
                        for (int rr = 0; rr < 32; ++rr) {
                            const int rw = row0 + rr;
                            if (rw < fp.M && col < ncol) fp.y[(int64_t)rw * fp.ld_y + col] = tb[rr * 32 + (lane ^ rr)];
                        }
                        __syncwarp();
                    }
                }
                // TMEM read and activations written: make the shared-memory
                // writes visible to the tensor cores, then release the layer
                tc_fence_before();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(smem_u32(&bars->h_ready));
            }
            if (stop) break;
        }
    }
    if (*failed && threadIdx.x == 0 && fp.err) atomicExch(fp.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
    }
}

size_t fused_smem_bytes() {
    return 1024 + 6 * (size_t)kXBlock + kFRing * (size_t)kWStage + 4 * 256 * sizeof(float) + sizeof(FusedBars) + 64;
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

void resolve_encode() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
}

// 2-D tensor map of the leading rows x cols block of a row-major bf16
// matrix, box = 64 columns x box_rows; reads past the block return zeros
bool make_map(CUtensorMap* map, const Mat& m, int64_t rows, int64_t cols, int box_rows) {
    resolve_encode();
    if (!g_encode) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)m.ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(m.ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// dynamic shared memory of a launch with column tile bn (at most two CTAs
// fit on an SM, holding 2 x 64 of its 512 TMEM columns)
size_t smem_request(int bn) {
    return 1024 + (size_t)kStages * (BM * BK * 2 + (size_t)bn * BK * 2) + sizeof(Barriers) + 64;
}

int g_raised[64] = {};
std::mutex g_raise_mu;

}  // namespace

cudaError_t gemm_prepare() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int need = (int)smem_request(kMaxBN);
    std::lock_guard<std::mutex> lk(g_raise_mu);
    if (dev < 64 && g_raised[dev] >= need) return cudaSuccess;
    e = cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    if (e == cudaSuccess && dev < 64) g_raised[dev] = need;
    return e;
}

bool tensor_maps_available() {
    resolve_encode();
    return g_encode != nullptr;
}

cudaError_t gemm_bf16(const Mat& A, const Mat& B, int64_t M, int N, int K, int k_splits, const Epilogue& ep,
                      cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (K <= 0 || k_splits < 1 || M > (int64_t)INT32_MAX) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(A.ptr) & 15u) || (reinterpret_cast<uintptr_t>(B.ptr) & 15u) || (A.ld & 7) ||
        (B.ld & 7) || A.cols < K || B.cols < K || A.rows < M || B.rows < N)
        return cudaErrorInvalidValue;
    if (k_splits > 1 && ep.kind != kEpiAtomicAdd) return cudaErrorInvalidValue;
    // column tile: N rounded up to 16, at most kMaxBN; TMEM columns: a power
    // of two >= 32 covering the tile
    const int n16 = (N + 15) / 16 * 16;
    const int bn = n16 <= kMaxBN ? n16 : kMaxBN;
    int tmem_cols = 32;
    while (tmem_cols < bn) tmem_cols <<= 1;
    int k_chunk = (K + k_splits - 1) / k_splits;
    k_chunk = (k_chunk + BK - 1) / BK * BK;
    const int splits = (K + k_chunk - 1) / k_chunk;
    CUtensorMap ma, mb;
    // the maps cover exactly M x K and N x K: padding rows and columns of the
    // buffers are never read (the copies fill them with zeros)
    if (!make_map(&ma, A, M, K, BM) || !make_map(&mb, B, N, K, bn)) return cudaErrorInvalidValue;
    const size_t smem_req = smem_request(bn);
    cudaError_t e = gemm_prepare();
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + bn - 1) / bn), (unsigned)splits);
    gemm_bf16_kernel<<<grid, kThreads, smem_req, s>>>(ma, mb, (int)M, N, K, k_chunk, bn, tmem_cols, ep);
    return cudaGetLastError();
}

cudaError_t mlp_forward_fused(const uint16_t* x, int64_t M, int in_dim, const uint16_t* const w[4], int out_dim,
                              const float* const bias[4], float* y, int64_t ld_y, int* err, int num_sms,
                              cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if ((in_dim != 64 && in_dim != 128) || out_dim < 16 || out_dim > 256 || out_dim % 16 || M > (int64_t)INT32_MAX)
        return cudaErrorInvalidValue;
    for (int l = 0; l < 4; ++l)
        if (reinterpret_cast<uintptr_t>(w[l]) & 15u) return cudaErrorInvalidValue;
    if (reinterpret_cast<uintptr_t>(x) & 15u) return cudaErrorInvalidValue;
    CUtensorMap mx, mw[4];
    const Mat X{x, M, in_dim, in_dim};
    const int din[4] = {in_dim, 256, 256, 256}, dout[4] = {256, 256, 256, out_dim};
    if (!make_map(&mx, X, M, in_dim, BM)) return cudaErrorInvalidValue;
    for (int l = 0; l < 4; ++l) {
        const Mat W{w[l], dout[l], din[l], din[l]};
        if (!make_map(&mw[l], W, dout[l], din[l], 256)) return cudaErrorInvalidValue;
    }
    const size_t smem = fused_smem_bytes();
    cudaError_t e = fused_prepare();
    if (e != cudaSuccess) return e;
    FusedParams fp;
    for (int l = 0; l < 4; ++l) fp.bias[l] = bias[l];
    fp.y = y;
    fp.ld_y = ld_y;
    fp.M = (int)M;
    fp.in_dim = in_dim;
    fp.out_dim = out_dim;
    fp.err = err;
    const int tiles = (int)((M + BM - 1) / BM);
    const int grid = tiles < num_sms ? tiles : num_sms;
    mlp_fused_forward_kernel<<<grid, kFThreads, smem, s>>>(mx, mw[0], mw[1], mw[2], mw[3], fp);
    return cudaGetLastError();
}

cudaError_t fused_prepare() {
    static int raised[64] = {};
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 64 && raised[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(mlp_fused_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fused_smem_bytes());
    if (e == cudaSuccess && dev < 64) raised[dev] = 1;
    return e;
}

}  // namespace mlp
}  // namespace comet
