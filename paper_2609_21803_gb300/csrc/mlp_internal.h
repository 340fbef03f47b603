// Internal interface of the learned proposal's kernels: the BF16 tensor-core
// GEMM (tcgen05 + TMA + TMEM) and its fused epilogues.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "comet.h"
#include "comet_proposal.h"

namespace comet {
namespace mlp {

// What the GEMM epilogue does with the FP32 accumulator tile D = A B^T
// (A [M][K], B [N][K], both bf16 row-major, i.e. K-major operands).
enum EpiKind : int {
    kEpiStore = 0,      // out_f32[m][n] = D + bias[n]
    kEpiBiasGelu = 1,   // Z = D + bias -> z_f32, H = gelu(Z) -> h (bf16) and h_t (bf16, transposed)
    kEpiGeluGrad = 2,   // G = D * gelu'(z_in) -> h (bf16) and h_t (bf16, transposed)
    kEpiAtomicAdd = 3,  // out_f32[m][n] += D (split-K partial sums)
};

struct Epilogue {
    int kind;
    const float* bias;      // [N] (kEpiStore, kEpiBiasGelu; nullable)
    float* out_f32;         // [M][ld_out] (kEpiStore, kEpiAtomicAdd), z (kEpiBiasGelu)
    int64_t ld_out;
    uint16_t* h;            // [M][ld_h] bf16 (kEpiBiasGelu, kEpiGeluGrad; nullable)
    int64_t ld_h;
    uint16_t* h_t;          // [N][ld_ht] bf16, transposed (nullable)
    int64_t ld_ht;
    const float* z_in;      // [M][ld_z] pre-activation (kEpiGeluGrad)
    int64_t ld_z;
    int* err;               // device flag: a bounded wait ran out (nullable)
};

// A row-major bf16 matrix [rows][cols] with leading dimension ld (elements);
// the GEMM reduces over cols.
struct Mat {
    const uint16_t* ptr;
    int64_t rows, cols, ld;
};

// D[M][N] = A[M][K] B[N][K]^T over K split into `k_splits` chunks (each a
// multiple of 64; with k_splits > 1 the epilogue must be kEpiAtomicAdd).
// Requirements: ptr 16-byte aligned, ld a multiple of 8, N <= 256 per
// column tile (larger N is tiled), K >= 1.  Returns a CUDA error code.
cudaError_t gemm_bf16(const Mat& A, const Mat& B, int64_t M, int N, int K, int k_splits, const Epilogue& ep,
                      cudaStream_t s);

// The tensor-map encoder from the driver (resolved once); false if absent.
bool tensor_maps_available();

// Fused forward pass of the 4-layer MLP (width 256): x [M][in_dim] BF16
// (in_dim 64 or 128), w[l] BF16 row-major [out][in] (K-major), biases FP32,
// y [M][ld_y] FP32 (out_dim <= 256, a multiple of 16).  One persistent CTA
// per SM (at most num_sms CTAs).
cudaError_t mlp_forward_fused(const uint16_t* x, int64_t M, int in_dim, const uint16_t* const w[4], int out_dim,
                              const float* const bias[4], float* y, int64_t ld_y, int* err, int num_sms,
                              cudaStream_t s);
cudaError_t fused_prepare();

// Raise the GEMM kernel's shared-memory limit to its largest configuration
// on the current device (once; not a stream operation, so later launches
// stay capturable).
cudaError_t gemm_prepare();

}  // namespace mlp

// The proposal's device-side steps used by the learned planner (mlp.cu).
comet_status proposal_reserve_prune(comet_proposal* q, int64_t cap, int keep);
comet_status proposal_prune_device(comet_proposal* q, comet_frontier* f, int keep, float* warm, int* row_scratch,
                                   cudaStream_t s);
comet_status proposal_predict_device(comet_proposal* q, const comet_mode_seq* seqs, int64_t n, float* merit,
                                     float* warm, cudaStream_t s);
// The problem a proposal was created for.
comet_problem* proposal_problem(const comet_proposal* q);

}  // namespace comet
