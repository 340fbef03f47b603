// expand_internal.h -- device layout of a frontier (the evaluated set V and
// the next batch) shared by expand.cu and frontier.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "comet.h"

namespace comet {

constexpr int kChunk = 4096;  // keys sorted per CTA in the top-k passes

struct TopKey {
    uint32_t mk;    // order-preserving key of M_hat
    uint32_t idx;   // position of the entry in the ranked array (first pass)
    uint64_t code;  // mode code (tie break)
};

struct FrontierDev {
    int instance, n_modes, lmax, slots;
    int64_t capacity;     // |V| maximum
    int64_t batch_cap;    // largest batch added at once
    unsigned long long* codes;  // [capacity]
    float* merit;               // [capacity]
    unsigned long long* nV;     // |V|
    unsigned long long* set;    // hash set of V's codes
    unsigned long long set_mask;
    TopKey* top_a;              // top-k pass buffers
    TopKey* top_b;
    unsigned long long* cand_code;  // [k_max * slots]
    int* flag;                      // [k_max * slots]
    unsigned long long* cand_keys;  // candidate table
    unsigned int* cand_ord;
    unsigned long long cand_mask;
    comet_mode_seq* next;           // [batch]
    int64_t* n_next;
    int* error;                     // 1 malformed order, 2 capacity exceeded
};

size_t topk_smem_bytes();
cudaError_t prepare_expand();
cudaError_t launch_frontier_add(const FrontierDev& F, const comet_mode_seq* seqs, int64_t n, const int64_t* d_n,
                                const float* cost, const float* viol, float eps_feas, float merit_mu, cudaStream_t s);
const TopKey* launch_topk(const FrontierDev& F, int k, cudaStream_t s, cudaError_t* err);
cudaError_t launch_expand(const FrontierDev& F, int k, int batch, int64_t budget, cudaStream_t s);

}  // namespace comet

struct comet_problem;

struct comet_frontier {
    comet_problem* p = nullptr;
    comet::FrontierDev d;
    int32_t batch = 0;
    int32_t k_max = 0;
    void* blob = nullptr;  // one allocation for all device arrays
};
