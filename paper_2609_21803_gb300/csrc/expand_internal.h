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
    // neighbourhood rule: edit radius (1, 2), grammar (0 = every order over
    // the instance's modes; 1 = the pushing grammar over stick-on-a-face and
    // free motion), alphabet size and one-edit slots per order
    int radius, grammar, n_alpha, slots1;
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

// one-edit slots of an order under a rule (fixed layout over l_max:
// substitutions l_max x n_alpha, insertions (l_max + 1) x n_alpha, deletions
// l_max) and all slots per parent (radius 2 adds slots1 x slots1)
inline int64_t edit_slots1(int lmax, int n_alpha) { return (int64_t)lmax * n_alpha * 2 + n_alpha + lmax; }
inline int64_t edit_slots(int lmax, int n_alpha, int radius) {
    const int64_t s1 = edit_slots1(lmax, n_alpha);
    return radius == 2 ? s1 + s1 * s1 : s1;
}
constexpr int kGrammarNone = 0, kGrammarPush = 1;
constexpr int kPushFree = 12;  // free motion in the 13-mode pushing alphabet

size_t topk_smem_bytes();
cudaError_t prepare_expand();
cudaError_t launch_frontier_restore(const FrontierDev& F, int64_t n, cudaStream_t s);
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
