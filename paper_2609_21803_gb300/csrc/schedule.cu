// schedule.cu -- longest-first ordering of a heterogeneous batch for the
// persistent evaluator (the size-binned work queue): TOs are binned by their
// interval count N = K * len and handed out in decreasing N, so the longest
// solves start first and the tail of the launch holds only short ones.
// Counting sort over the N values; counts and grids are fixed-size, so the
// ordering can be captured in a CUDA graph with a device-resident TO count.

#include <cuda_runtime.h>
#include <stdint.h>

#include "comet.h"
#include "comet_internal.h"

namespace comet {
namespace {

__device__ __forceinline__ int to_bin(const comet_mode_seq& q, const DevInstance* inst, int n_inst) {
    if (q.instance < 0 || q.instance >= n_inst || q.len < 1) return 0;
    const int N = inst[q.instance].K * (int)q.len;
    return N < kMaxN ? N : kMaxN;
}

__global__ void hist_kernel(const comet_mode_seq* seqs, int64_t n, const int64_t* d_n, const DevInstance* inst,
                            int n_inst, unsigned int* hist) {
    const int64_t nn = d_n ? min(*d_n, n) : n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[to_bin(seqs[i], inst, n_inst)], 1u);
}

// exclusive scan over bins in decreasing N: cursor[b] = number of TOs with a
// larger N (single CTA)
__global__ void scan_desc_kernel(const unsigned int* hist, unsigned int* cursor) {
    __shared__ unsigned int part[1024];
    const int per = (kMaxN + 1 + 1023) / 1024;
    // thread t owns bins [kMaxN - per*(t+1) + 1, kMaxN - per*t] (descending)
    unsigned int s = 0;
    for (int j = 0; j < per; ++j) {
        const int b = kMaxN - per * (int)threadIdx.x - j;
        if (b >= 0) s += hist[b];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const unsigned int v = (threadIdx.x >= (unsigned)d) ? part[threadIdx.x - d] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned int run = (threadIdx.x > 0) ? part[threadIdx.x - 1] : 0u;
    for (int j = 0; j < per; ++j) {
        const int b = kMaxN - per * (int)threadIdx.x - j;
        if (b >= 0) {
            cursor[b] = run;
            run += hist[b];
        }
    }
}

__global__ void scatter_kernel(const comet_mode_seq* seqs, int64_t n, const int64_t* d_n, const DevInstance* inst,
                               int n_inst, unsigned int* cursor, unsigned int* perm) {
    const int64_t nn = d_n ? min(*d_n, n) : n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned int pos = atomicAdd(&cursor[to_bin(seqs[i], inst, n_inst)], 1u);
        perm[pos] = (unsigned int)i;
    }
}

}  // namespace

size_t lpt_scratch_bytes() { return 2 * sizeof(unsigned int) * (kMaxN + 1); }

cudaError_t launch_lpt_order(const comet_mode_seq* seqs, int64_t n, const int64_t* d_n, const DevInstance* inst,
                             int n_inst, unsigned int* scratch, unsigned int* perm, cudaStream_t s) {
    unsigned int* hist = scratch;
    unsigned int* cursor = scratch + (kMaxN + 1);
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned int) * (kMaxN + 1), s);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const int blocks = (int)((n + threads - 1) / threads < 1024 ? (n + threads - 1) / threads : 1024);
    if (blocks < 1) return cudaSuccess;
    hist_kernel<<<blocks, threads, 0, s>>>(seqs, n, d_n, inst, n_inst, hist);
    scan_desc_kernel<<<1, 1024, 0, s>>>(hist, cursor);
    scatter_kernel<<<blocks, threads, 0, s>>>(seqs, n, d_n, inst, n_inst, cursor, perm);
    return cudaGetLastError();
}

}  // namespace comet
