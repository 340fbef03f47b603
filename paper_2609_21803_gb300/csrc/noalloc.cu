// noalloc.cu -- an evaluation entry point that allocates no memory.
//
// comet_eval_modes() keeps its scratch (per-warp stage records, the work
// counter, the instance table, per-TO diagnostics) in device memory that the
// problem allocates with cudaMalloc.  Some callers cannot allocate: code that
// runs inside a memory pool or arena that owns all device memory of the
// process, real-time loops where an allocation (and the device-wide
// synchronisation cudaMalloc / cudaFree may imply) is not allowed after
// start-up, or hosts that forbid the CUDA allocator altogether.  For them,
// comet_eval_modes_noalloc() runs the same evaluator kernel with its scratch
// in one fixed, file-scope device array instead.
//
// The array holds kNoallocScratchBytes (32 MiB) on every device that loads
// the library, until the process exits.  Its device address is looked up
// (cudaGetSymbolAddress, with the device current) on every call: the lookup
// is cheap, and an address cached across calls would go stale if the caller
// reset the device in between.  The first call on a device may load the
// library's device code there.  All calls share the array and it keeps the
// last call's contents: the work counter and the error flag are cleared by
// every call, and calls whose kernels overlap on the GPU (two streams, or two
// host threads) race on it.
//
// The instance table reaches the array through a one-block kernel that takes
// the table by value as its launch parameter, so the call never copies from
// host memory: it does not wait for the stream to drain and holds no pointer
// into the caller's stack.

#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>

#include "comet.h"
#include "comet_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = 32u << 20;
constexpr int kNoallocMaxInstances = 64;

// scratch layout: [header 256 B: work counter, error flag]
//                 [instance table: kNoallocMaxInstances DevInstance]
//                 [per-warp stage records]
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr size_t kHeaderBytes = 256;
constexpr size_t kInstBytes = ((sizeof(comet::DevInstance) * kNoallocMaxInstances + 255) / 256) * 256;
constexpr size_t kRecordBytes = kNoallocScratchBytes - kHeaderBytes - kInstBytes;

// the instance table as one launch parameter (under the 32,764-byte limit of
// kernel parameters)
struct InstTable {
    comet::DevInstance inst[kNoallocMaxInstances];
};
static_assert(sizeof(InstTable) <= 32764, "instance table too large for a kernel parameter");
static_assert(sizeof(comet::DevInstance) % 4 == 0, "the table is copied in 4-byte words");

__global__ void noalloc_table_kernel(const __grid_constant__ InstTable t, int n_words, uint32_t* dst) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&t);
    for (int i = threadIdx.x; i < n_words; i += blockDim.x) dst[i] = src[i];
}

comet_status noalloc_fail(comet_status st, const char* msg) {
    comet::set_error(msg);
    return st;
}

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" comet_status comet_eval_modes_noalloc(const comet_instance_desc* inst, int32_t n_instances,
                                                 const comet_solver_opts* opts, void* cuda_stream,
                                                 const comet_mode_seq* mode_seqs, int64_t n,
                                                 const float* warm_starts, float* out_cost, float* out_traj,
                                                 int32_t* out_status) {
    if (!inst || n_instances < 1) return noalloc_fail(COMET_ERR_INVALID_ARG, "need at least one instance");
    if (n_instances > kNoallocMaxInstances)
        return noalloc_fail(COMET_ERR_INVALID_ARG,
                            "comet_eval_modes_noalloc: more than 64 instances do not fit the fixed scratch");
    for (int32_t i = 0; i < n_instances; ++i)
        if (inst[i].task != COMET_TASK_PUSHER_SLIDER)
            return noalloc_fail(COMET_ERR_INVALID_ARG, "comet_eval_modes_noalloc: pushing instances only");
    if (n < 0) return noalloc_fail(COMET_ERR_INVALID_ARG, "n < 0");
    if (n > 0xffffffffLL) return noalloc_fail(COMET_ERR_INVALID_ARG, "n too large");
    int Nmax = 0;
    {
        const comet_status st = comet::check_instances(inst, n_instances, &Nmax);
        if (st != COMET_OK) return st;  // message already set
    }
    if (n == 0) return COMET_OK;
    if (!mode_seqs || !out_cost || !out_status)
        return noalloc_fail(COMET_ERR_INVALID_ARG, "mode_seqs, out_cost and out_status are required");
    // no staging buffers here: every array must already be in device memory
    if (!on_device(mode_seqs) || !on_device(out_cost) || !on_device(out_status) ||
        (warm_starts && !on_device(warm_starts)) || (out_traj && !on_device(out_traj)))
        return noalloc_fail(COMET_ERR_INVALID_ARG,
                            "comet_eval_modes_noalloc: all arrays must be device memory (nothing is staged)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0)
        return noalloc_fail(COMET_ERR_CUDA, "cudaGetDevice failed");
    // the device address of the array on the current device (the host-side
    // name g_noalloc_scratch is not a device address)
    unsigned char* base = nullptr;
    {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return noalloc_fail(COMET_ERR_CUDA, cudaGetErrorString(e));
        base = static_cast<unsigned char*>(ptr);
    }
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return noalloc_fail(COMET_ERR_CUDA, "device query failed");
    const int warps_per_block = 4;
    const int blocks_per_sm =
        comet::eval_blocks_per_sm(warps_per_block, comet::smem_per_warp_bytes(Nmax) * warps_per_block);
    if (blocks_per_sm < 1) return noalloc_fail(COMET_ERR_INVALID_ARG, "N_max needs too much shared memory");
    // warps limited by the occupancy, the TO count and the record space
    const int64_t per_warp = (int64_t)comet::kRec * Nmax * (int64_t)sizeof(float);
    const int64_t fit = (int64_t)kRecordBytes / per_warp;
    int64_t warps = std::min<int64_t>((int64_t)num_sms * blocks_per_sm * warps_per_block, n);
    warps = ((warps + warps_per_block - 1) / warps_per_block) * warps_per_block;
    warps = std::min<int64_t>(warps, (fit / warps_per_block) * warps_per_block);
    if (warps < warps_per_block)
        return noalloc_fail(COMET_ERR_INVALID_ARG,
                            "comet_eval_modes_noalloc: N_max too large for the 32 MiB scratch");

    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned int* queue = reinterpret_cast<unsigned int*>(base);
    int* bad = reinterpret_cast<int*>(base + 64);
    comet::DevInstance* d_inst = reinterpret_cast<comet::DevInstance*>(base + kHeaderBytes);
    float* ws = reinterpret_cast<float*>(base + kHeaderBytes + kInstBytes);
    InstTable table;
    memset(&table, 0, sizeof(table));
    for (int i = 0; i < n_instances; ++i) comet::make_dev_instance(inst[i], &table.inst[i]);
    comet_solver_opts o;
    comet::merge_opts(opts, &o);
    // the counter and flag start at zero; the instance table is rewritten
    // from the launch parameter (no host memory is read by the GPU)
    cudaError_t e = cudaMemsetAsync(base, 0, kHeaderBytes, s);
    if (e == cudaSuccess) {
        const int n_words = (int)(sizeof(comet::DevInstance) * n_instances / 4);
        noalloc_table_kernel<<<1, 256, 0, s>>>(table, n_words, reinterpret_cast<uint32_t*>(d_inst));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return noalloc_fail(COMET_ERR_CUDA, cudaGetErrorString(e));

    comet::EvalArgs a;
    memset(&a, 0, sizeof(a));
    a.inst = d_inst;
    a.n_inst = n_instances;
    a.seqs = mode_seqs;
    a.n = n;
    a.warm = warm_starts;
    a.stride = 7 * (int64_t)Nmax + 4;
    a.Nmax = Nmax;
    a.out_cost = out_cost;
    a.out_traj = out_traj;
    a.out_status = out_status;
    a.ws = ws;
    a.ws_per_warp = (int64_t)comet::kRec * Nmax;
    a.queue = queue;
    a.bad_input = bad;
    a.sp = comet::make_params(o, 0);
    for (int i = 0; i < n_instances; ++i) a.sp.free_motion |= inst[i].n_modes == 13;
    e = comet::launch_eval(a, (int)warps, warps_per_block, s);
    if (e != cudaSuccess) return noalloc_fail(COMET_ERR_CUDA, cudaGetErrorString(e));
    return COMET_OK;
}
