// autotune.cu -- launch shape of the persistent evaluator: TOs per CTA (one
// warp per TO, 1..4), resident CTAs per SM and the unrolling of the stage
// loops (1 or 2 stages per trip).  comet_autotune times the evaluator on a
// sample of the caller's orders under every candidate shape and keeps the
// fastest; the pick is cached per (device, N_max) for the process, and
// problems created later with the same key start from it.
//
// Every (TOs per CTA, CTAs per SM) shape solves each TO in one warp with the
// same arithmetic, so the results do not depend on it, only the time does;
// the unrolled build of the stage loops is compiled with other multiply-add
// contractions, so its FP32 rounding differs.

#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "comet.h"
#include "comet_internal.h"
#include "problem_internal.h"

namespace {

std::mutex g_mu;
struct Shape {
    int wpb, bps, unroll;
};
std::map<std::pair<int, int>, Shape> g_cache;  // (device, N_max) -> shape

comet_status tfail(comet_status st, const char* msg) {
    comet::set_error(msg);
    return st;
}

comet_status tcuda(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return tfail(e == cudaErrorMemoryAllocation ? COMET_ERR_OOM : COMET_ERR_CUDA, buf);
}

// occupancy limit of the evaluator for a shape (0 if it does not fit)
int occupancy(const comet_problem* p, int wpb) {
    return comet::eval_blocks_per_sm(wpb, comet::smem_per_warp_bytes(p->Nmax) * wpb);
}

}  // namespace

namespace comet {

// launch shape cached for this device and N_max, if any
bool cached_launch_shape(int device, int nmax, int* wpb, int* bps, int* unroll) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find({device, nmax});
    if (it == g_cache.end()) return false;
    *wpb = it->second.wpb;
    *bps = it->second.bps;
    *unroll = it->second.unroll;
    return true;
}

}  // namespace comet

extern "C" {

comet_status comet_get_launch_config(comet_problem* p, comet_launch_config* out) {
    if (!p || !out) return tfail(COMET_ERR_INVALID_ARG, "problem and out are required");
    out->warps_per_block = p->warps_per_block;
    out->blocks_per_sm = p->blocks_per_sm;
    out->max_blocks_per_sm = p->task == COMET_TASK_PUSHER_SLIDER ? occupancy(p, p->warps_per_block) : p->blocks_per_sm;
    out->unroll = p->unroll;
    return COMET_OK;
}

comet_status comet_set_launch_config(comet_problem* p, const comet_launch_config* c) {
    if (!p || !c) return tfail(COMET_ERR_INVALID_ARG, "problem and config are required");
    if (p->task != COMET_TASK_PUSHER_SLIDER)
        return tfail(COMET_ERR_INVALID_ARG, "the bimanual evaluator runs one CTA per TO; its shape is fixed");
    if (c->warps_per_block < 1 || c->warps_per_block > 4)
        return tfail(COMET_ERR_INVALID_ARG, "warps_per_block must be in 1..4");
    const int occ = occupancy(p, c->warps_per_block);
    if (occ < 1) return tfail(COMET_ERR_INVALID_ARG, "this shape does not fit on an SM");
    if (c->blocks_per_sm < 1 || c->blocks_per_sm > occ)
        return tfail(COMET_ERR_INVALID_ARG, "blocks_per_sm must be in 1..the occupancy limit");
    if (c->unroll < 0 || c->unroll > 2) return tfail(COMET_ERR_INVALID_ARG, "unroll must be 0, 1 or 2");
    if (p->stream) cudaStreamSynchronize(p->stream);
    p->warps_per_block = c->warps_per_block;
    p->blocks_per_sm = c->blocks_per_sm;
    p->unroll = c->unroll == 2 ? 2 : 1;
    return COMET_OK;
}

comet_status comet_autotune(comet_problem* p, const comet_mode_seq* sample, int64_t n, int32_t max_iters,
                            comet_launch_config* out, float* out_ms, int32_t* n_candidates) {
    if (!p || !sample || n < 1) return tfail(COMET_ERR_INVALID_ARG, "problem and a sample are required");
    if (p->task != COMET_TASK_PUSHER_SLIDER)
        return tfail(COMET_ERR_INVALID_ARG, "the bimanual evaluator runs one CTA per TO; its shape is fixed");
    cudaStream_t s = p->stream;
    // candidate shapes: 1..4 TOs per CTA, each at its occupancy limit and at
    // three quarters of it (fewer resident warps, less contention), each
    // with the stage loops unrolled once and twice
    std::vector<Shape> cand;
    for (int w = 1; w <= 4; ++w) {
        const int occ = occupancy(p, w);
        if (occ < 1) continue;
        const int q = std::max(1, (occ * 3) / 4);
        for (int un = 1; un <= 2; ++un) {
            cand.push_back({w, occ, un});
            if (q != occ) cand.push_back({w, q, un});
        }
    }
    if (cand.empty()) return tfail(COMET_ERR_INVALID_ARG, "no launch shape fits");
    // device copies of the sample and outputs
    cudaPointerAttributes at;
    const bool dev = cudaPointerGetAttributes(&at, sample) == cudaSuccess &&
                     (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (!dev)
        for (int64_t i = 0; i < n; ++i)
            if (sample[i].instance < 0 || sample[i].instance >= (int)p->inst.size() || sample[i].len < 1 ||
                sample[i].len > p->inst[sample[i].instance].max_segments)
                return tfail(COMET_ERR_INVALID_ARG, "malformed order in the sample");
    void* buf = nullptr;
    const size_t b_seq = (sizeof(comet_mode_seq) * n + 255) & ~(size_t)255;
    cudaError_t e = cudaMalloc(&buf, b_seq + (sizeof(float) + sizeof(int32_t)) * n + 512);
    if (e != cudaSuccess) return tcuda(e, "autotune buffers");
    comet_mode_seq* d_seq = dev ? const_cast<comet_mode_seq*>(sample) : (comet_mode_seq*)buf;
    float* d_cost = (float*)((char*)buf + b_seq);
    int32_t* d_status = (int32_t*)((char*)buf + b_seq + ((sizeof(float) * n + 255) & ~(size_t)255));
    if (!dev) e = cudaMemcpyAsync(d_seq, sample, sizeof(comet_mode_seq) * n, cudaMemcpyHostToDevice, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int w0 = p->warps_per_block, b0 = p->blocks_per_sm, u0 = p->unroll;
    float best_ms = 0.f;
    int best = -1;
    comet_status st = COMET_OK;
    for (size_t c = 0; c < cand.size() && e == cudaSuccess && st == COMET_OK; ++c) {
        p->warps_per_block = cand[c].wpb;
        p->blocks_per_sm = cand[c].bps;
        p->unroll = cand[c].unroll;
        st = comet::reserve_eval(p, n);
        if (st != COMET_OK) break;
        // one untimed launch (attributes, caches), then the timed one
        st = comet::launch_eval_device(p, d_seq, n, nullptr, nullptr, max_iters, d_cost, nullptr, d_status);
        if (st != COMET_OK) break;
        e = cudaEventRecord(e0, s);
        if (e != cudaSuccess) break;
        st = comet::launch_eval_device(p, d_seq, n, nullptr, nullptr, max_iters, d_cost, nullptr, d_status);
        if (st != COMET_OK) break;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (out_ms) out_ms[c] = ms;
        if (best < 0 || ms < best_ms) {
            best = (int)c;
            best_ms = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(buf);
    if (n_candidates) *n_candidates = (int32_t)cand.size();
    if (st != COMET_OK || e != cudaSuccess || best < 0) {
        p->warps_per_block = w0;
        p->blocks_per_sm = b0;
        p->unroll = u0;
        if (st != COMET_OK) return st;
        return tcuda(e, "autotune");
    }
    p->warps_per_block = cand[best].wpb;
    p->blocks_per_sm = cand[best].bps;
    p->unroll = cand[best].unroll;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[{p->device, p->Nmax}] = cand[best];
    }
    if (out) comet_get_launch_config(p, out);
    return COMET_OK;
}

}  // extern "C"
