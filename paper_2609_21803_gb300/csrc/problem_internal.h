// problem_internal.h -- the comet_problem object shared by the host-side
// translation units (api.cu, frontier.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "comet.h"
#include "comet_internal.h"

struct comet_problem {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<comet_instance_desc> inst;
    comet::DevInstance* d_inst = nullptr;
    comet_solver_opts opts;
    int Nmax = 0;
    int task = COMET_TASK_PUSHER_SLIDER;
    int64_t stride = 0;
    int num_sms = 0;
    int warps_per_block = 4;
    int blocks_per_sm = 0;
    int unroll = 1;  // stages per trip of the evaluator's stage loops
    int stall_staging = 0;  // test hook of comet_debug_stall_staging
    float* d_ws = nullptr;
    int64_t ws_warps = 0;
    // per-warp workspace of the timing-optimisation kernel
    float* d_tws = nullptr;
    int64_t tws_floats = 0;
    unsigned int* d_queue = nullptr;
    int* d_bad = nullptr;
    // per-TO diagnostics of the last call
    float* d_viol = nullptr;
    float* d_merit = nullptr;
    int32_t* d_iters = nullptr;
    float* d_stat = nullptr;
    int64_t stats_cap = 0;
    int64_t last_n = 0;
    // longest-first ordering of heterogeneous batches
    unsigned int* d_perm = nullptr;
    unsigned int* d_lpt = nullptr;
    int64_t perm_cap = 0;
    bool hetero = false;  // instances differ in K or allow several lengths
    // staging for host buffers
    void* d_stage = nullptr;
    size_t stage_bytes = 0;
};

namespace comet {
// Make sure the per-warp workspace and the per-TO diagnostics of p can hold
// a launch of n TOs (allocates on growth; never during stream capture).
comet_status reserve_eval(comet_problem* p, int64_t n);
// Launch the evaluator on p's stream over device arrays; if d_n is not
// null the TO count is read from device memory (up to n_max TOs).
comet_status launch_eval_device(comet_problem* p, const comet_mode_seq* d_seqs, int64_t n_max, const int64_t* d_n,
                                const float* d_warm, int32_t max_iters, float* d_cost, float* d_traj,
                                int32_t* d_status);
}  // namespace comet
