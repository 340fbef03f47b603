// frontier.cu -- host side of the greedy local mode expansion (Sec. III-B,
// Algorithm 1): frontier lifetime, adding evaluated orders to V, one
// expansion round, and the planner that runs Algorithm 1 on the device with
// each round captured once as a CUDA graph and replayed.

#include <cuda_runtime.h>
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

comet_status ffail(comet_status st, const char* msg) {
    comet::set_error(msg);
    return st;
}

comet_status fcuda(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return ffail(e == cudaErrorMemoryAllocation ? COMET_ERR_OOM : COMET_ERR_CUDA, buf);
}

#define FTRY(call, what)                                  \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return fcuda(e_, what);    \
    } while (0)

uint64_t pow2_at_least(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

bool dev_ptr(const void* ptr) {
    cudaPointerAttributes at;
    if (!ptr || cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

comet_status comet_frontier_create(comet_problem* p, int32_t instance, int64_t capacity, int32_t batch,
                                   int32_t k_max, comet_frontier** out) {
    return comet_frontier_create_ex(p, instance, capacity, batch, k_max, 1, COMET_GRAMMAR_NONE, out);
}

comet_status comet_frontier_create_ex(comet_problem* p, int32_t instance, int64_t capacity, int32_t batch,
                                      int32_t k_max, int32_t radius, int32_t grammar, comet_frontier** out) {
    if (!p || !out) return ffail(COMET_ERR_INVALID_ARG, "problem and out are required");
    *out = nullptr;
    if (instance < 0 || instance >= (int)p->inst.size()) return ffail(COMET_ERR_INVALID_ARG, "instance out of range");
    if (capacity < 1 || batch < 1 || k_max < 1 || k_max > comet::kChunk || batch > capacity)
        return ffail(COMET_ERR_INVALID_ARG, "need 1 <= batch <= capacity and 1 <= k_max <= 4096");
    const comet_instance_desc& d = p->inst[instance];
    if (radius != 1 && radius != 2) return ffail(COMET_ERR_INVALID_ARG, "the edit radius is 1 or 2");
    if (grammar != COMET_GRAMMAR_NONE && grammar != COMET_GRAMMAR_PUSH)
        return ffail(COMET_ERR_INVALID_ARG, "unknown grammar");
    if (grammar == COMET_GRAMMAR_PUSH && (d.task != COMET_TASK_PUSHER_SLIDER || d.n_modes != 13))
        return ffail(COMET_ERR_INVALID_ARG, "the pushing grammar needs a pushing instance with n_modes = 13");
    const int n_alpha = grammar == COMET_GRAMMAR_PUSH ? 5 : d.n_modes;
    const int64_t slots = comet::edit_slots(d.max_segments, n_alpha, radius);
    if ((int64_t)k_max * slots > ((int64_t)1 << 26))
        return ffail(COMET_ERR_INVALID_ARG, "k_max x neighbourhood slots above 2^26 (use radius 1 or a smaller beam)");
    {
        const cudaError_t pe = comet::prepare_expand();
        if (pe != cudaSuccess) return fcuda(pe, "expand kernels");
    }
    comet_frontier* f = new comet_frontier();
    f->p = p;
    f->batch = batch;
    f->k_max = k_max;
    comet::FrontierDev& F = f->d;
    memset(&F, 0, sizeof(F));
    F.instance = instance;
    F.n_modes = d.n_modes;
    F.lmax = d.max_segments;
    F.radius = radius;
    F.grammar = grammar;
    F.n_alpha = n_alpha;
    F.slots1 = (int)comet::edit_slots1(F.lmax, n_alpha);
    F.slots = (int)slots;
    F.capacity = capacity;
    F.batch_cap = std::max<int64_t>(batch, 1);
    const uint64_t set_cap = pow2_at_least((uint64_t)capacity * 2);
    const int64_t total = (int64_t)k_max * F.slots;
    const uint64_t cand_cap = pow2_at_least((uint64_t)total * 2);
    const int64_t chunks = (capacity + comet::kChunk - 1) / comet::kChunk;
    const int64_t top_n = std::max<int64_t>(chunks * k_max, comet::kChunk);
    // carve one allocation
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_codes = take(sizeof(unsigned long long) * capacity);
    const size_t o_merit = take(sizeof(float) * capacity);
    const size_t o_nV = take(sizeof(unsigned long long));
    const size_t o_set = take(sizeof(unsigned long long) * set_cap);
    const size_t o_ta = take(sizeof(comet::TopKey) * top_n);
    const size_t o_tb = take(sizeof(comet::TopKey) * top_n);
    const size_t o_cc = take(sizeof(unsigned long long) * total);
    const size_t o_fl = take(sizeof(int) * total);
    const size_t o_ck = take(sizeof(unsigned long long) * cand_cap);
    const size_t o_co = take(sizeof(unsigned int) * cand_cap);
    const size_t o_nx = take(sizeof(comet_mode_seq) * batch);
    const size_t o_nn = take(sizeof(int64_t));
    const size_t o_er = take(sizeof(int));
    cudaError_t e = cudaMalloc(&f->blob, off);
    if (e != cudaSuccess) {
        delete f;
        return fcuda(e, "frontier allocation");
    }
    char* b = (char*)f->blob;
    F.codes = (unsigned long long*)(b + o_codes);
    F.merit = (float*)(b + o_merit);
    F.nV = (unsigned long long*)(b + o_nV);
    F.set = (unsigned long long*)(b + o_set);
    F.set_mask = set_cap - 1;
    F.top_a = (comet::TopKey*)(b + o_ta);
    F.top_b = (comet::TopKey*)(b + o_tb);
    F.cand_code = (unsigned long long*)(b + o_cc);
    F.flag = (int*)(b + o_fl);
    F.cand_keys = (unsigned long long*)(b + o_ck);
    F.cand_ord = (unsigned int*)(b + o_co);
    F.cand_mask = cand_cap - 1;
    F.next = (comet_mode_seq*)(b + o_nx);
    F.n_next = (int64_t*)(b + o_nn);
    F.error = (int*)(b + o_er);
    e = cudaMemsetAsync(f->blob, 0, off, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        cudaFree(f->blob);
        delete f;
        return fcuda(e, "frontier init");
    }
    *out = f;
    return COMET_OK;
}

// checkpoint file: this header, then V's codes (u64) and merits (f32), then
// the pending batch (comet_mode_seq records)
struct FrontierCkpt {
    char magic[8];
    int32_t version, instance, n_modes, lmax, radius, grammar;
    int64_t capacity, n_evaluated, n_next;
};
constexpr char kFrontierMagic[8] = {'C', 'O', 'M', 'E', 'T', 'F', 'V', '1'};

comet_status comet_frontier_save(comet_frontier* f, const char* path) {
    if (!f || !path) return ffail(COMET_ERR_INVALID_ARG, "frontier and path are required");
    const comet::FrontierDev& F = f->d;
    cudaStream_t s = f->p->stream;
    unsigned long long nv = 0;
    int64_t nn = 0;
    cudaError_t e = cudaMemcpyAsync(&nv, F.nV, sizeof(nv), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nn, F.n_next, sizeof(nn), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fcuda(e, "checkpoint: read the sizes");
    const int64_t n = (int64_t)std::min<unsigned long long>(nv, (unsigned long long)F.capacity);
    nn = std::max<int64_t>(0, std::min<int64_t>(nn, f->batch));
    std::vector<unsigned long long> codes(n);
    std::vector<float> merit(n);
    std::vector<comet_mode_seq> next(nn);
    if (n) e = cudaMemcpyAsync(codes.data(), F.codes, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(merit.data(), F.merit, sizeof(float) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && nn)
        e = cudaMemcpyAsync(next.data(), F.next, sizeof(comet_mode_seq) * nn, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fcuda(e, "checkpoint: read the frontier");
    FrontierCkpt h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kFrontierMagic, sizeof(h.magic));
    h.version = 1;
    h.instance = F.instance;
    h.n_modes = F.n_modes;
    h.lmax = F.lmax;
    h.radius = F.radius;
    h.grammar = F.grammar;
    h.capacity = F.capacity;
    h.n_evaluated = n;
    h.n_next = nn;
    FILE* fp = fopen(path, "wb");
    if (!fp) return ffail(COMET_ERR_INVALID_ARG, "checkpoint: cannot open the file for writing");
    bool ok = fwrite(&h, sizeof(h), 1, fp) == 1;
    ok = ok && (n == 0 || (fwrite(codes.data(), sizeof(unsigned long long), n, fp) == (size_t)n &&
                           fwrite(merit.data(), sizeof(float), n, fp) == (size_t)n));
    ok = ok && (nn == 0 || fwrite(next.data(), sizeof(comet_mode_seq), nn, fp) == (size_t)nn);
    if (fclose(fp) != 0 || !ok) return ffail(COMET_ERR_INVALID_ARG, "checkpoint: write failed");
    return COMET_OK;
}

comet_status comet_frontier_load(comet_frontier* f, const char* path) {
    if (!f || !path) return ffail(COMET_ERR_INVALID_ARG, "frontier and path are required");
    comet::FrontierDev& F = f->d;
    FILE* fp = fopen(path, "rb");
    if (!fp) return ffail(COMET_ERR_INVALID_ARG, "checkpoint: cannot open the file");
    FrontierCkpt h;
    if (fread(&h, sizeof(h), 1, fp) != 1 || memcmp(h.magic, kFrontierMagic, sizeof(h.magic)) != 0 || h.version != 1) {
        fclose(fp);
        return ffail(COMET_ERR_INVALID_ARG, "checkpoint: not a frontier checkpoint");
    }
    if (h.instance != F.instance || h.n_modes != F.n_modes || h.lmax != F.lmax || h.radius != F.radius ||
        h.grammar != F.grammar || h.n_evaluated < 0 || h.n_evaluated > F.capacity || h.n_next < 0 ||
        h.n_next > f->batch) {
        fclose(fp);
        return ffail(COMET_ERR_INVALID_ARG, "checkpoint: another instance, alphabet, rule or a larger frontier");
    }
    const int64_t n = h.n_evaluated, nn = h.n_next;
    std::vector<unsigned long long> codes(n);
    std::vector<float> merit(n);
    std::vector<comet_mode_seq> next(nn);
    bool ok = n == 0 || (fread(codes.data(), sizeof(unsigned long long), n, fp) == (size_t)n &&
                         fread(merit.data(), sizeof(float), n, fp) == (size_t)n);
    ok = ok && (nn == 0 || fread(next.data(), sizeof(comet_mode_seq), nn, fp) == (size_t)nn);
    fclose(fp);
    if (!ok) return ffail(COMET_ERR_INVALID_ARG, "checkpoint: the file is truncated");
    for (int64_t i = 0; i < n; ++i)
        if (codes[i] == 0) return ffail(COMET_ERR_INVALID_ARG, "checkpoint: an invalid mode code");
    for (int64_t i = 0; i < nn; ++i) {
        bool bad = next[i].instance != F.instance || next[i].len < 1 || next[i].len > F.lmax;
        for (int j = 0; !bad && j < next[i].len; ++j) bad = next[i].modes[j] >= F.n_modes;
        if (bad) return ffail(COMET_ERR_INVALID_ARG, "checkpoint: a pending order outside this frontier's alphabet");
    }
    cudaStream_t s = f->p->stream;
    const unsigned long long nv = (unsigned long long)n;
    cudaError_t e = cudaMemsetAsync(F.set, 0, sizeof(unsigned long long) * (F.set_mask + 1), s);
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(F.codes, codes.data(), sizeof(unsigned long long) * n,
                                                   cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(F.merit, merit.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nn)
        e = cudaMemcpyAsync(F.next, next.data(), sizeof(comet_mode_seq) * nn, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(F.nV, &nv, sizeof(nv), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(F.n_next, &h.n_next, sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(F.error, 0, sizeof(int), s);
    if (e == cudaSuccess) e = comet::launch_frontier_restore(F, n, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fcuda(e, "checkpoint: restore the frontier");
    return COMET_OK;
}

comet_status comet_frontier_destroy(comet_frontier* f) {
    if (!f) return COMET_OK;
    if (f->p && f->p->stream) cudaStreamSynchronize(f->p->stream); else cudaDeviceSynchronize();
    cudaFree(f->blob);
    delete f;
    return COMET_OK;
}

comet_status comet_frontier_add(comet_frontier* f, const comet_mode_seq* seqs, int64_t n, const float* cost,
                                const float* viol) {
    if (!f) return ffail(COMET_ERR_INVALID_ARG, "frontier is NULL");
    if (n < 0) return ffail(COMET_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return COMET_OK;
    if (!seqs || !cost || !viol) return ffail(COMET_ERR_INVALID_ARG, "seqs, cost and viol are required");
    if (n > f->d.capacity) return ffail(COMET_ERR_BUDGET, "more orders than the frontier capacity");
    comet_problem* p = f->p;
    cudaStream_t s = p->stream;
    // stage host arrays (validated first) through one temporary device block
    const bool ds = dev_ptr(seqs), dc = dev_ptr(cost), dv = dev_ptr(viol);
    void* tmp = nullptr;
    const comet_mode_seq* d_seqs = seqs;
    const float* d_cost = cost;
    const float* d_viol = viol;
    if (!(ds && dc && dv)) {
        if (!ds)
            for (int64_t i = 0; i < n; ++i)
                if (seqs[i].instance != f->d.instance || seqs[i].len < 1 || seqs[i].len > f->d.lmax)
                    return ffail(COMET_ERR_INVALID_ARG, "an order does not belong to this frontier's instance");
        const size_t bs = sizeof(comet_mode_seq) * n, bf = sizeof(float) * n;
        FTRY(cudaMalloc(&tmp, bs + 2 * bf + 512), "staging");
        char* t = (char*)tmp;
        if (!ds) {
            FTRY(cudaMemcpyAsync(t, seqs, bs, cudaMemcpyHostToDevice, s), "copy orders");
            d_seqs = (const comet_mode_seq*)t;
        }
        if (!dc) {
            FTRY(cudaMemcpyAsync(t + bs + 256, cost, bf, cudaMemcpyHostToDevice, s), "copy cost");
            d_cost = (const float*)(t + bs + 256);
        }
        if (!dv) {
            FTRY(cudaMemcpyAsync(t + bs + bf + 512 - 256, viol, bf, cudaMemcpyHostToDevice, s), "copy viol");
            d_viol = (const float*)(t + bs + bf + 512 - 256);
        }
    }
    comet::FrontierDev F = f->d;
    F.batch_cap = n;
    const cudaError_t e = comet::launch_frontier_add(F, d_seqs, n, nullptr, d_cost, d_viol, (float)p->opts.eps_feas,
                                                     (float)p->opts.merit_mu, s);
    if (tmp) {
        cudaStreamSynchronize(s);
        cudaFree(tmp);
    }
    if (e != cudaSuccess) return fcuda(e, "frontier add");
    return COMET_OK;
}

comet_status comet_expand(comet_problem* p, comet_frontier* f, int32_t k) {
    if (!p || !f || f->p != p) return ffail(COMET_ERR_INVALID_ARG, "problem / frontier mismatch");
    if (k < 1 || k > f->k_max) return ffail(COMET_ERR_INVALID_ARG, "k out of [1, k_max]");
    const cudaError_t e = comet::launch_expand(f->d, k, f->batch, 0, p->stream);
    if (e != cudaSuccess) return fcuda(e, "expand");
    return COMET_OK;
}

comet_status comet_frontier_next(comet_frontier* f, const comet_mode_seq** seqs, int64_t* n) {
    if (!f || !seqs || !n) return ffail(COMET_ERR_INVALID_ARG, "arguments are required");
    cudaStream_t s = f->p->stream;
    int64_t nn = 0;
    FTRY(cudaMemcpyAsync(&nn, f->d.n_next, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "read count");
    FTRY(cudaStreamSynchronize(s), "synchronise");
    *seqs = f->d.next;
    *n = nn;
    return COMET_OK;
}

comet_status comet_frontier_copy_next(comet_frontier* f, comet_mode_seq* out, int64_t cap, int64_t* n) {
    if (!f || !n || (cap > 0 && !out)) return ffail(COMET_ERR_INVALID_ARG, "arguments are required");
    const comet_mode_seq* d = nullptr;
    int64_t nn = 0;
    const comet_status st = comet_frontier_next(f, &d, &nn);
    if (st != COMET_OK) return st;
    if (nn > cap) return ffail(COMET_ERR_BUDGET, "output buffer smaller than the next batch");
    if (nn > 0) {
        FTRY(cudaMemcpyAsync(out, d, sizeof(comet_mode_seq) * nn, cudaMemcpyDefault, f->p->stream), "copy batch");
        FTRY(cudaStreamSynchronize(f->p->stream), "synchronise");
    }
    *n = nn;
    return COMET_OK;
}

comet_status comet_frontier_size(comet_frontier* f, int64_t* n_evaluated, int32_t* error_flags) {
    if (!f || !n_evaluated) return ffail(COMET_ERR_INVALID_ARG, "arguments are required");
    cudaStream_t s = f->p->stream;
    unsigned long long nv = 0;
    int err = 0;
    FTRY(cudaMemcpyAsync(&nv, f->d.nV, sizeof(nv), cudaMemcpyDeviceToHost, s), "read size");
    FTRY(cudaMemcpyAsync(&err, f->d.error, sizeof(err), cudaMemcpyDeviceToHost, s), "read flags");
    FTRY(cudaStreamSynchronize(s), "synchronise");
    *n_evaluated = (int64_t)std::min<unsigned long long>(nv, (unsigned long long)f->d.capacity);
    if (error_flags) *error_flags = err;
    return COMET_OK;
}

comet_status comet_frontier_best(comet_frontier* f, int32_t k, uint64_t* out_codes, float* out_merit) {
    if (!f || !out_codes || k < 1 || k > f->k_max) return ffail(COMET_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = f->p->stream;
    // the top-k passes of an expansion round, without generating neighbours
    comet::FrontierDev F = f->d;
    cudaError_t e = cudaSuccess;
    const comet::TopKey* top = comet::launch_topk(F, k, s, &e);
    if (!top) return fcuda(e, "top-k");
    std::vector<comet::TopKey> h(k);
    FTRY(cudaMemcpyAsync(h.data(), top, sizeof(comet::TopKey) * k, cudaMemcpyDeviceToHost, s), "read top-k");
    FTRY(cudaStreamSynchronize(s), "synchronise");
    unsigned long long nv = 0;
    FTRY(cudaMemcpy(&nv, F.nV, sizeof(nv), cudaMemcpyDeviceToHost), "read size");
    for (int i = 0; i < k; ++i) {
        const bool valid = (unsigned long long)i < nv;
        out_codes[i] = valid ? h[i].code : 0;
        if (out_merit) {
            // invert the order-preserving key
            const uint32_t mk = h[i].mk;
            const uint32_t bits = (mk & 0x80000000u) ? (mk & 0x7fffffffu) : ~mk;
            float m;
            memcpy(&m, &bits, 4);
            out_merit[i] = valid ? m : __builtin_inff();
        }
    }
    return COMET_OK;
}

}  // extern "C"

// ------------------------------------------------------------- planner

namespace {

__global__ void decode_kernel(const uint64_t* codes, int64_t n, int instance, int n_modes, comet_mode_seq* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long code = codes[i];
    comet_mode_seq q;
    memset(&q, 0, sizeof(q));
    q.instance = instance;
    const unsigned long long base = (unsigned long long)(n_modes + 1);
    const int L = (int)(code % base);
    code /= base;
    q.len = (uint8_t)L;
    for (int j = 0; j < L && j < COMET_MAX_SEGMENTS; ++j) {
        q.modes[j] = (uint16_t)(code % base - 1);
        code /= base;
    }
    out[i] = q;
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { cudaFree(p); }
};

}  // namespace

static_assert(sizeof(comet_plan_opts) == 40, "comet_plan_opts layout (the binding mirrors it)");

extern "C" comet_status comet_default_plan_opts(comet_plan_opts* po) {
    if (!po) return ffail(COMET_ERR_INVALID_ARG, "opts is NULL");
    memset(po, 0, sizeof(*po));
    po->k = 64;
    po->batch = 4096;
    po->rounds = 3;
    po->budget = 0;
    po->k_ref = 256;
    po->ref_iters = 0;
    po->use_graph = 1;
    po->radius = 1;
    po->grammar = COMET_GRAMMAR_NONE;
    return COMET_OK;
}

namespace comet {

// Algorithm 1 on the device; with a proposal q every expansion round
// generates the whole neighbourhood of the beam, keeps the `batch` best
// candidates by predicted merit and warm-starts them, and the seed batch is
// warm-started too.
comet_status plan_impl(comet_problem* p, int32_t instance, const comet_mode_seq* seeds, int64_t n_seeds,
                       const comet_plan_opts* po_in, comet_proposal* q, comet_plan_result* out, float* out_traj) {
    if (!p || !seeds || !out || n_seeds < 1) return ffail(COMET_ERR_INVALID_ARG, "problem, seeds and out are required");
    comet_plan_opts po;
    if (po_in)
        po = *po_in;
    else
        comet_default_plan_opts(&po);
    if (po.k < 1 || po.batch < 1 || po.rounds < 0 || po.k_ref < 1 || po.k_ref > comet::kChunk)
        return ffail(COMET_ERR_INVALID_ARG, "bad planner options");
    // a graph cannot be captured on the legacy default stream: the planner
    // runs on a private stream ordered after the problem's stream and the
    // problem's stream waits for it at the end
    cudaStream_t user_stream = p->stream;
    cudaStream_t s = nullptr;
    FTRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "planner stream");
    {
        cudaEvent_t e0;
        FTRY(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming), "event");
        cudaEventRecord(e0, user_stream);
        cudaStreamWaitEvent(s, e0, 0);
        cudaEventDestroy(e0);
    }
    struct StreamSwap {
        comet_problem* p;
        cudaStream_t user, own;
        ~StreamSwap() {
            cudaEvent_t e1;
            if (cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) == cudaSuccess) {
                cudaEventRecord(e1, own);
                cudaStreamWaitEvent(user, e1, 0);
                cudaEventDestroy(e1);
            }
            cudaStreamSynchronize(own);
            p->stream = user;
            cudaStreamDestroy(own);
        }
    } swap{p, user_stream, s};
    p->stream = s;
    memset(out, 0, sizeof(*out));
    const int64_t n0 = po.budget > 0 ? std::min<int64_t>(n_seeds, po.budget) : n_seeds;
    const int64_t capacity =
        po.budget > 0 ? std::max<int64_t>(po.budget, n0) : n0 + (int64_t)po.rounds * po.batch;
    const int32_t batch = (int32_t)std::min<int64_t>(po.batch, capacity);
    if (q && batch > comet::kChunk) return ffail(COMET_ERR_INVALID_ARG, "a learned plan keeps at most 4096 per round");
    // with a proposal the frontier's next batch holds the whole neighbourhood
    // of the beam, which the proposal then prunes to `batch`
    const comet_instance_desc& di = p->inst[instance];
    const int64_t slots =
        comet::edit_slots(di.max_segments, po.grammar == COMET_GRAMMAR_PUSH ? 5 : di.n_modes, po.radius);
    const int64_t cand = q ? std::max<int64_t>((int64_t)po.k * slots, batch) : batch;
    if (cand > INT32_MAX) return ffail(COMET_ERR_INVALID_ARG, "neighbourhood too large");
    // the next batch holds the whole neighbourhood, so the frontier's
    // capacity covers it even where the evaluations stay far below it
    comet_frontier* f = nullptr;
    comet_status st = comet_frontier_create_ex(p, instance, std::max<int64_t>(capacity, cand), (int32_t)cand,
                                               std::max(po.k, po.k_ref), po.radius, po.grammar, &f);
    if (st != COMET_OK) return st;
    struct Guard {
        comet_frontier* f;
        ~Guard() { comet_frontier_destroy(f); }
    } guard{f};
    const int64_t n_eval_max = std::max<int64_t>({n0, (int64_t)batch, (int64_t)po.k_ref});
    st = comet::reserve_eval(p, n_eval_max);
    if (st != COMET_OK) return st;
    DevBuf warm_buf, rows_buf;
    float* d_warm = nullptr;
    int* d_rows = nullptr;
    if (q) {
        st = comet::proposal_reserve_prune(q, std::max<int64_t>(f->batch, n0), batch);
        if (st != COMET_OK) return st;
        FTRY(cudaMalloc(&warm_buf.p, sizeof(float) * p->stride * std::max<int64_t>(n0, batch)), "warm starts");
        FTRY(cudaMalloc(&rows_buf.p, sizeof(int) * batch), "rows");
        d_warm = (float*)warm_buf.p;
        d_rows = (int*)rows_buf.p;
    }
    DevBuf buf;
    const size_t b_seq = sizeof(comet_mode_seq) * n_eval_max;
    const size_t b_f = sizeof(float) * n_eval_max;
    FTRY(cudaMalloc(&buf.p, b_seq + 2 * b_f + sizeof(int32_t) * n_eval_max + sizeof(uint64_t) * po.k_ref + 1024),
         "planner buffers");
    char* bp = (char*)buf.p;
    comet_mode_seq* d_seqs = (comet_mode_seq*)bp;
    float* d_cost = (float*)(bp + b_seq + 256);
    int32_t* d_status = (int32_t*)(bp + b_seq + b_f + 512);
    uint64_t* d_codes = (uint64_t*)(bp + b_seq + b_f + sizeof(int32_t) * n_eval_max + 768);
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() {
            for (int i = 0; i < 4; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } evg{ev};
    for (auto& e : ev) FTRY(cudaEventCreate(&e), "events");
    FTRY(cudaEventRecord(ev[0], s), "event");
    // seed batch F_0: evaluate with t_exp and add to V
    FTRY(cudaMemcpyAsync(d_seqs, seeds, sizeof(comet_mode_seq) * n0, cudaMemcpyDefault, s), "copy seeds");
    if (q) {
        st = comet::proposal_predict_device(q, d_seqs, n0, nullptr, d_warm, s);
        if (st != COMET_OK) return st;
    }
    st = comet::launch_eval_device(p, d_seqs, n0, nullptr, d_warm, 0, d_cost, nullptr, d_status);
    if (st != COMET_OK) return st;
    comet::FrontierDev F = f->d;
    FTRY(comet::launch_frontier_add(F, d_seqs, n0, nullptr, d_cost, p->d_viol, (float)p->opts.eps_feas,
                                    (float)p->opts.merit_mu, s),
         "add seeds");
    // one round: expand, evaluate F_{s+1} (count read on the device), add
    auto round = [&]() -> comet_status {
        cudaError_t e = comet::launch_expand(F, po.k, q ? f->batch : batch, po.budget, s);
        if (e != cudaSuccess) return fcuda(e, "expand");
        if (q) {
            const comet_status r = comet::proposal_prune_device(q, f, batch, d_warm, d_rows, s);
            if (r != COMET_OK) return r;
        }
        comet_status r = comet::launch_eval_device(p, F.next, batch, F.n_next, d_warm, 0, d_cost, nullptr, d_status);
        if (r != COMET_OK) return r;
        comet::FrontierDev Fa = F;
        Fa.batch_cap = batch;
        e = comet::launch_frontier_add(Fa, F.next, batch, F.n_next, d_cost, p->d_viol, (float)p->opts.eps_feas,
                                       (float)p->opts.merit_mu, s);
        if (e != cudaSuccess) return fcuda(e, "add");
        return COMET_OK;
    };
    if (po.use_graph && po.rounds > 0) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        FTRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
        const comet_status rs = round();
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (rs != COMET_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rs;
        }
        if (e != cudaSuccess) return fcuda(e, "end capture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fcuda(e, "instantiate");
        for (int r = 0; r < po.rounds && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, s);
        cudaGraphExecDestroy(exec);
        if (e != cudaSuccess) return fcuda(e, "graph launch");
    } else {
        for (int r = 0; r < po.rounds; ++r) {
            st = round();
            if (st != COMET_OK) return st;
        }
    }
    FTRY(cudaEventRecord(ev[1], s), "event");
    // refinement (Algorithm 1, line 13): re-solve the K_ref best orders of V
    // with budget t_ref and return the best feasible refined one
    FTRY(cudaEventRecord(ev[2], s), "event");
    std::vector<uint64_t> codes(po.k_ref);
    st = comet_frontier_best(f, po.k_ref, codes.data(), nullptr);
    if (st != COMET_OK) return st;
    int64_t n_ref = 0;
    while (n_ref < po.k_ref && codes[n_ref] != 0) ++n_ref;
    int64_t n_v = 0;
    int32_t err = 0;
    st = comet_frontier_size(f, &n_v, &err);
    if (st != COMET_OK) return st;
    out->evaluations = n_v;
    out->rounds_run = po.rounds;
    out->best.len = 0;
    out->best_status = COMET_TO_MAX_ITER;
    if (n_ref > 0) {
        FTRY(cudaMemcpyAsync(d_codes, codes.data(), sizeof(uint64_t) * n_ref, cudaMemcpyHostToDevice, s), "codes");
        decode_kernel<<<(unsigned)((n_ref + 127) / 128), 128, 0, s>>>(d_codes, n_ref, instance,
                                                                       p->inst[instance].n_modes, d_seqs);
        FTRY(cudaGetLastError(), "decode");
        const int32_t t_ref = p->opts.ref_iters > 0 ? p->opts.ref_iters : 1500;
        st = comet::launch_eval_device(p, d_seqs, n_ref, nullptr, nullptr, po.ref_iters > 0 ? po.ref_iters : t_ref,
                                       d_cost, nullptr, d_status);
        if (st != COMET_OK) return st;
        FTRY(cudaEventRecord(ev[3], s), "event");
        std::vector<float> cost(n_ref), viol(n_ref);
        std::vector<int32_t> status(n_ref);
        std::vector<comet_mode_seq> sq(n_ref);
        FTRY(cudaMemcpyAsync(cost.data(), d_cost, sizeof(float) * n_ref, cudaMemcpyDeviceToHost, s), "copy");
        FTRY(cudaMemcpyAsync(viol.data(), p->d_viol, sizeof(float) * n_ref, cudaMemcpyDeviceToHost, s), "copy");
        FTRY(cudaMemcpyAsync(status.data(), d_status, sizeof(int32_t) * n_ref, cudaMemcpyDeviceToHost, s), "copy");
        FTRY(cudaMemcpyAsync(sq.data(), d_seqs, sizeof(comet_mode_seq) * n_ref, cudaMemcpyDeviceToHost, s), "copy");
        FTRY(cudaStreamSynchronize(s), "synchronise");
        int64_t best = -1;
        for (int64_t i = 0; i < n_ref; ++i) {
            const bool feas = status[i] == COMET_TO_CONVERGED && viol[i] <= (float)p->opts.eps_feas;
            if (feas && (best < 0 || cost[i] < cost[best])) best = i;
        }
        if (best >= 0) {
            out->best = sq[best];
            out->best_cost = cost[best];
            out->best_viol = viol[best];
            out->best_status = status[best];
            if (out_traj) {
                // solve the winner once more to return its trajectory
                float* d_traj = nullptr;
                FTRY(cudaMalloc(&d_traj, sizeof(float) * p->stride), "trajectory");
                st = comet::launch_eval_device(p, d_seqs + best, 1, nullptr, nullptr,
                                               po.ref_iters > 0 ? po.ref_iters : t_ref, d_cost, d_traj, d_status);
                cudaError_t e = cudaMemcpyAsync(out_traj, d_traj, sizeof(float) * p->stride, cudaMemcpyDefault, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                cudaFree(d_traj);
                if (st != COMET_OK) return st;
                if (e != cudaSuccess) return fcuda(e, "copy trajectory");
            }
        }
    } else {
        FTRY(cudaEventRecord(ev[3], s), "event");
    }
    FTRY(cudaEventSynchronize(ev[3]), "synchronise");
    cudaEventElapsedTime(&out->explore_ms, ev[0], ev[1]);
    cudaEventElapsedTime(&out->refine_ms, ev[2], ev[3]);
    if (err) return ffail(COMET_ERR_BUDGET, "the evaluated set overflowed its capacity");
    return COMET_OK;
}

}  // namespace comet

extern "C" comet_status comet_plan(comet_problem* p, int32_t instance, const comet_mode_seq* seeds, int64_t n_seeds,
                                   const comet_plan_opts* opts, comet_plan_result* out, float* out_traj) {
    return comet::plan_impl(p, instance, seeds, n_seeds, opts, nullptr, out, out_traj);
}

extern "C" comet_status comet_plan_learned(comet_problem* p, int32_t instance, const comet_mode_seq* seeds,
                                           int64_t n_seeds, const comet_plan_opts* opts, comet_proposal* q,
                                           comet_plan_result* out, float* out_traj) {
    if (!q) return ffail(COMET_ERR_INVALID_ARG, "proposal is required");
    if (comet::proposal_problem(q) != p) return ffail(COMET_ERR_INVALID_ARG, "the proposal belongs to another problem");
    return comet::plan_impl(p, instance, seeds, n_seeds, opts, q, out, out_traj);
}

// ------------------------------------------------- batched planner

namespace {

struct SlotSrc {
    const comet_mode_seq* next;
    const int64_t* n;
};

// next batches of all frontiers into fixed slots of `batch` orders; slots
// past a frontier's count get length 0 (the evaluator skips them)
__global__ void gather_next_kernel(const SlotSrc* src, int n_inst, int batch, comet_mode_seq* out) {
    const int64_t total = (int64_t)n_inst * batch;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / batch), j = (int)(t - (int64_t)i * batch);
        comet_mode_seq q;
        if (j < *src[i].n) {
            q = src[i].next[j];
        } else {
            memset(&q, 0, sizeof(q));
        }
        out[t] = q;
    }
}

// ranked entries of one frontier -> orders; ranks past |V| become empty
// slots (length 0), which the evaluator skips
__global__ void decode_top_kernel(const comet::TopKey* top, int k, const unsigned long long* nV, int instance,
                                  int n_modes, comet_mode_seq* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    comet_mode_seq q;
    memset(&q, 0, sizeof(q));
    q.instance = instance;
    if ((unsigned long long)i < *nV) {
        unsigned long long code = top[i].code;
        const unsigned long long base = (unsigned long long)(n_modes + 1);
        const int L = (int)(code % base);
        code /= base;
        q.len = (uint8_t)L;
        for (int j = 0; j < L && j < COMET_MAX_SEGMENTS; ++j) {
            q.modes[j] = (uint16_t)(code % base - 1);
            code /= base;
        }
    }
    out[i] = q;
}

}  // namespace

namespace {

// Algorithm 1 over several instances, rounds shared by all of them; with a
// proposal q each frontier's whole neighbourhood is ranked and pruned to
// `batch` by predicted merit and the kept orders (and the seeds) are
// warm-started from its predicted controls.
comet_status plan_batch_impl(comet_problem* p, int32_t n_inst, const int32_t* instances,
                             const comet_mode_seq* seeds, const int64_t* seed_offsets, const comet_plan_opts* po_in,
                             comet_proposal* q, comet_plan_result* out) {
    if (!p || n_inst < 1 || !instances || !seeds || !seed_offsets || !out)
        return ffail(COMET_ERR_INVALID_ARG, "problem, instances, seeds, offsets and out are required");
    if (q && comet::proposal_problem(q) != p)
        return ffail(COMET_ERR_INVALID_ARG, "the proposal belongs to another problem");
    comet_plan_opts po;
    if (po_in)
        po = *po_in;
    else
        comet_default_plan_opts(&po);
    if (po.k < 1 || po.batch < 1 || po.rounds < 0 || po.k_ref < 1 || po.k_ref > comet::kChunk)
        return ffail(COMET_ERR_INVALID_ARG, "bad planner options");
    if (q && po.batch > comet::kChunk) return ffail(COMET_ERR_INVALID_ARG, "a learned plan keeps at most 4096 per round");
    for (int i = 0; i < n_inst; ++i) {
        if (instances[i] < 0 || instances[i] >= (int)p->inst.size())
            return ffail(COMET_ERR_INVALID_ARG, "instance out of range");
        if (seed_offsets[i + 1] <= seed_offsets[i]) return ffail(COMET_ERR_INVALID_ARG, "every instance needs seeds");
    }
    if (seed_offsets[0] != 0) return ffail(COMET_ERR_INVALID_ARG, "seed_offsets[0] must be 0");
    const int64_t S = seed_offsets[n_inst];
    // private stream (a graph cannot be captured on the legacy stream)
    cudaStream_t user_stream = p->stream;
    cudaStream_t s = nullptr;
    FTRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "planner stream");
    {
        cudaEvent_t e0;
        FTRY(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming), "event");
        cudaEventRecord(e0, user_stream);
        cudaStreamWaitEvent(s, e0, 0);
        cudaEventDestroy(e0);
    }
    struct StreamSwap {
        comet_problem* p;
        cudaStream_t user, own;
        ~StreamSwap() {
            cudaEvent_t e1;
            if (cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) == cudaSuccess) {
                cudaEventRecord(e1, own);
                cudaStreamWaitEvent(user, e1, 0);
                cudaEventDestroy(e1);
            }
            cudaStreamSynchronize(own);
            p->stream = user;
            cudaStreamDestroy(own);
        }
    } swap{p, user_stream, s};
    p->stream = s;
    // one frontier per instance
    std::vector<comet_frontier*> fr(n_inst, nullptr);
    struct FGuard {
        std::vector<comet_frontier*>* f;
        ~FGuard() {
            for (auto* x : *f)
                if (x) comet_frontier_destroy(x);
        }
    } fguard{&fr};
    const int32_t batch = po.batch;
    for (int i = 0; i < n_inst; ++i) {
        const int64_t n0 = seed_offsets[i + 1] - seed_offsets[i];
        // V never holds more than the seeds and `rounds` batches, nor more
        // than the budget
        const int64_t reach = n0 + (int64_t)po.rounds * batch;
        const int64_t cap = po.budget > 0 ? std::max<int64_t>(std::min<int64_t>(po.budget, reach), n0) : reach;
        // with a proposal the next batch holds the beam's whole neighbourhood
        const comet_instance_desc& di = p->inst[instances[i]];
        const int64_t slots =
            comet::edit_slots(di.max_segments, po.grammar == COMET_GRAMMAR_PUSH ? 5 : di.n_modes, po.radius);
        const int64_t cand = q ? std::max<int64_t>((int64_t)po.k * slots, batch) : std::min<int64_t>(batch, cap);
        if (cand > INT32_MAX) return ffail(COMET_ERR_INVALID_ARG, "neighbourhood too large");
        // a frontier's next batch never exceeds its capacity
        const int64_t cap_i = std::max<int64_t>(cap, cand);
        const comet_status st = comet_frontier_create_ex(p, instances[i], cap_i, (int32_t)cand,
                                                         std::max(po.k, po.k_ref), po.radius, po.grammar, &fr[i]);
        if (st != COMET_OK) return st;
    }
    const int64_t n_round = (int64_t)n_inst * batch, n_ref_all = (int64_t)n_inst * po.k_ref;
    const int64_t n_eval_max = std::max<int64_t>({S, n_round, n_ref_all});
    comet_status st = comet::reserve_eval(p, n_eval_max);
    if (st != COMET_OK) return st;
    DevBuf buf;
    const size_t b_seq = ((sizeof(comet_mode_seq) * n_eval_max + 255) / 256) * 256;
    const size_t b_f = ((sizeof(float) * n_eval_max + 255) / 256) * 256;
    const size_t b_src = ((sizeof(SlotSrc) * n_inst + 255) / 256) * 256;
    FTRY(cudaMalloc(&buf.p, b_seq + 2 * b_f + b_src), "planner buffers");
    char* bp = (char*)buf.p;
    comet_mode_seq* d_seqs = (comet_mode_seq*)bp;
    float* d_cost = (float*)(bp + b_seq);
    int32_t* d_status = (int32_t*)(bp + b_seq + b_f);
    SlotSrc* d_src = (SlotSrc*)(bp + b_seq + 2 * b_f);
    DevBuf warm_buf, rows_buf;
    float* d_warm = nullptr;
    int* d_rows = nullptr;
    if (q) {
        int64_t cand_max = 0;
        for (int i = 0; i < n_inst; ++i) cand_max = std::max<int64_t>(cand_max, fr[i]->batch);
        st = comet::proposal_reserve_prune(q, std::max<int64_t>(cand_max, S), batch);
        if (st != COMET_OK) return st;
        FTRY(cudaMalloc(&warm_buf.p, sizeof(float) * (size_t)p->stride * (size_t)std::max<int64_t>(S, n_round)),
             "warm starts");
        FTRY(cudaMalloc(&rows_buf.p, sizeof(int) * (size_t)n_round), "rows");
        d_warm = (float*)warm_buf.p;
        d_rows = (int*)rows_buf.p;
    }
    {
        std::vector<SlotSrc> h(n_inst);
        for (int i = 0; i < n_inst; ++i) h[i] = SlotSrc{fr[i]->d.next, fr[i]->d.n_next};
        FTRY(cudaMemcpyAsync(d_src, h.data(), sizeof(SlotSrc) * n_inst, cudaMemcpyHostToDevice, s), "slots");
    }
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() {
            for (int i = 0; i < 4; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } evg{ev};
    for (auto& e : ev) FTRY(cudaEventCreate(&e), "events");
    const float eps = (float)p->opts.eps_feas, mmu = (float)p->opts.merit_mu;
    FTRY(cudaEventRecord(ev[0], s), "event");
    // seed batches of every instance in one launch
    FTRY(cudaMemcpyAsync(d_seqs, seeds, sizeof(comet_mode_seq) * S, cudaMemcpyDefault, s), "copy seeds");
    if (q) {
        st = comet::proposal_predict_device(q, d_seqs, S, nullptr, d_warm, s);
        if (st != COMET_OK) return st;
    }
    st = comet::launch_eval_device(p, d_seqs, S, nullptr, d_warm, 0, d_cost, nullptr, d_status);
    if (st != COMET_OK) return st;
    for (int i = 0; i < n_inst; ++i) {
        const int64_t o = seed_offsets[i], n = seed_offsets[i + 1] - o;
        FTRY(comet::launch_frontier_add(fr[i]->d, d_seqs + o, n, nullptr, d_cost + o, p->d_viol + o, eps, mmu, s),
             "add seeds");
    }
    // one round: every frontier expands, all next batches are evaluated in
    // one persistent launch, each frontier adds its slots
    auto round = [&]() -> comet_status {
        for (int i = 0; i < n_inst; ++i) {
            const cudaError_t e = comet::launch_expand(fr[i]->d, po.k, fr[i]->batch, po.budget, s);
            if (e != cudaSuccess) return fcuda(e, "expand");
            if (q) {
                // rank the whole neighbourhood, keep `batch` in order; the
                // warm starts land in the frontier's slots
                const comet_status r = comet::proposal_prune_device(
                    q, fr[i], batch, d_warm + (int64_t)i * batch * p->stride, d_rows + (int64_t)i * batch, s);
                if (r != COMET_OK) return r;
            }
        }
        gather_next_kernel<<<(unsigned)std::min<int64_t>((n_round + 255) / 256, 4096), 256, 0, s>>>(d_src, n_inst,
                                                                                                   batch, d_seqs);
        FTRY(cudaGetLastError(), "gather");
        comet_status r = comet::launch_eval_device(p, d_seqs, n_round, nullptr, d_warm, 0, d_cost, nullptr, d_status);
        if (r != COMET_OK) return r;
        for (int i = 0; i < n_inst; ++i) {
            comet::FrontierDev Fa = fr[i]->d;
            Fa.batch_cap = batch;
            const int64_t o = (int64_t)i * batch;
            const cudaError_t e = comet::launch_frontier_add(Fa, d_seqs + o, batch, fr[i]->d.n_next, d_cost + o,
                                                             p->d_viol + o, eps, mmu, s);
            if (e != cudaSuccess) return fcuda(e, "add");
        }
        return COMET_OK;
    };
    if (po.use_graph && po.rounds > 0) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        FTRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
        const comet_status rs = round();
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (rs != COMET_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rs;
        }
        if (e != cudaSuccess) return fcuda(e, "end capture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fcuda(e, "instantiate");
        for (int r = 0; r < po.rounds && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, s);
        cudaGraphExecDestroy(exec);
        if (e != cudaSuccess) return fcuda(e, "graph launch");
    } else {
        for (int r = 0; r < po.rounds; ++r) {
            st = round();
            if (st != COMET_OK) return st;
        }
    }
    FTRY(cudaEventRecord(ev[1], s), "event");
    // refinement: the K_ref best of every instance, ranked and decoded on the
    // device (ranks past |V_i| become empty slots), re-solved in one launch
    FTRY(cudaEventRecord(ev[2], s), "event");
    for (int i = 0; i < n_inst; ++i) {
        cudaError_t e = cudaSuccess;
        const comet::TopKey* top = comet::launch_topk(fr[i]->d, po.k_ref, s, &e);
        if (!top) return fcuda(e, "top-k");
        decode_top_kernel<<<(unsigned)((po.k_ref + 127) / 128), 128, 0, s>>>(
            top, po.k_ref, fr[i]->d.nV, instances[i], p->inst[instances[i]].n_modes, d_seqs + (int64_t)i * po.k_ref);
        FTRY(cudaGetLastError(), "decode");
    }
    const int32_t t_ref = po.ref_iters > 0 ? po.ref_iters : (p->opts.ref_iters > 0 ? p->opts.ref_iters : 1500);
    st = comet::launch_eval_device(p, d_seqs, n_ref_all, nullptr, nullptr, t_ref, d_cost, nullptr, d_status);
    if (st != COMET_OK) return st;
    FTRY(cudaEventRecord(ev[3], s), "event");
    std::vector<float> cost(n_ref_all), viol(n_ref_all);
    std::vector<int32_t> status(n_ref_all);
    std::vector<comet_mode_seq> sq(n_ref_all);
    FTRY(cudaMemcpyAsync(cost.data(), d_cost, sizeof(float) * n_ref_all, cudaMemcpyDeviceToHost, s), "copy");
    FTRY(cudaMemcpyAsync(viol.data(), p->d_viol, sizeof(float) * n_ref_all, cudaMemcpyDeviceToHost, s), "copy");
    FTRY(cudaMemcpyAsync(status.data(), d_status, sizeof(int32_t) * n_ref_all, cudaMemcpyDeviceToHost, s), "copy");
    FTRY(cudaMemcpyAsync(sq.data(), d_seqs, sizeof(comet_mode_seq) * n_ref_all, cudaMemcpyDeviceToHost, s), "copy");
    FTRY(cudaStreamSynchronize(s), "synchronise");
    std::vector<int64_t> n_ev(n_inst, 0);
    for (int i = 0; i < n_inst; ++i) {
        int32_t err = 0;
        st = comet_frontier_size(fr[i], &n_ev[i], &err);
        if (st != COMET_OK) return st;
        if (err) return ffail(COMET_ERR_BUDGET, "an evaluated set overflowed its capacity");
    }
    float explore_ms = 0.f, refine_ms = 0.f;
    cudaEventElapsedTime(&explore_ms, ev[0], ev[1]);
    cudaEventElapsedTime(&refine_ms, ev[2], ev[3]);
    for (int i = 0; i < n_inst; ++i) {
        comet_plan_result& r = out[i];
        memset(&r, 0, sizeof(r));
        r.best_status = COMET_TO_MAX_ITER;
        r.rounds_run = po.rounds;
        r.evaluations = n_ev[i];
        r.explore_ms = explore_ms;
        r.refine_ms = refine_ms;
        int64_t best = -1;
        for (int64_t j = 0; j < po.k_ref; ++j) {
            const int64_t t = (int64_t)i * po.k_ref + j;
            const bool feas = status[t] == COMET_TO_CONVERGED && viol[t] <= (float)p->opts.eps_feas;
            if (feas && (best < 0 || cost[t] < cost[best])) best = t;
        }
        if (best >= 0) {
            r.best = sq[best];
            r.best_cost = cost[best];
            r.best_viol = viol[best];
            r.best_status = status[best];
        }
    }
    return COMET_OK;
}

}  // namespace

extern "C" comet_status comet_plan_batch(comet_problem* p, int32_t n_inst, const int32_t* instances,
                                         const comet_mode_seq* seeds, const int64_t* seed_offsets,
                                         const comet_plan_opts* opts, comet_plan_result* out) {
    return plan_batch_impl(p, n_inst, instances, seeds, seed_offsets, opts, nullptr, out);
}

extern "C" comet_status comet_plan_batch_learned(comet_problem* p, int32_t n_inst, const int32_t* instances,
                                                 const comet_mode_seq* seeds, const int64_t* seed_offsets,
                                                 const comet_plan_opts* opts, comet_proposal* q,
                                                 comet_plan_result* out) {
    if (!q) return ffail(COMET_ERR_INVALID_ARG, "proposal is required");
    return plan_batch_impl(p, n_inst, instances, seeds, seed_offsets, opts, q, out);
}

// ------------------------------------------------ uniform sampling of orders

namespace {

// what the sampler needs of an instance's order space
struct SampleSpec {
    int instance, n_modes, lmax, grammar;
    unsigned long long total;             // number of orders
    unsigned long long per_len[COMET_MAX_SEGMENTS];  // orders of each length 1..lmax
    unsigned long long comp[COMET_MAX_SEGMENTS][5];  // grammar: completions after mode (alphabet index)
};

__device__ __forceinline__ unsigned long long splitmix_draw(unsigned long long seed, unsigned long long i) {
    // SplitMix64 (Steele, Lea and Flood 2014): state seed + (i + 1) golden gamma
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int push_alpha(int a) { return a < 4 ? 3 * a : 12; }

__device__ __forceinline__ bool push_ok(int a, int b) {
    if (a == b) return false;
    if (a == 12 || b == 12) return true;
    const int d = (a / 3 - b / 3 + 4) & 3;
    return d == 1 || d == 3;
}

// order number idx of the (length, lexicographic) enumeration
__global__ void sample_kernel(SampleSpec sp, unsigned long long seed, int64_t first, int64_t n, comet_mode_seq* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long idx = splitmix_draw(seed, (unsigned long long)(first + i)) % sp.total;
    comet_mode_seq q;
    memset(&q, 0, sizeof(q));
    q.instance = sp.instance;
    int L = 1;
    while (L < sp.lmax && idx >= sp.per_len[L - 1]) idx -= sp.per_len[L - 1], ++L;
    q.len = (uint8_t)L;
    if (sp.grammar == 0) {
        for (int pos = L - 1; pos >= 0; --pos) {
            q.modes[pos] = (uint16_t)(idx % (unsigned long long)sp.n_modes);
            idx /= (unsigned long long)sp.n_modes;
        }
    } else {
        int last = 12;  // orders start in free motion
        q.modes[0] = 12;
        for (int pos = 1; pos < L; ++pos) {
            const int rem = L - 1 - pos;
            for (int a = 0; a < 5; ++a) {
                const int b = push_alpha(a);
                if (!push_ok(last, b)) continue;
                const unsigned long long c = sp.comp[rem][a];
                if (idx < c) {
                    q.modes[pos] = (uint16_t)b;
                    last = b;
                    break;
                }
                idx -= c;
            }
        }
    }
    out[i] = q;
}

}  // namespace

extern "C" comet_status comet_sample_orders(comet_problem* p, int32_t instance, uint64_t seed, int64_t first,
                                            int64_t n, int32_t grammar, comet_mode_seq* out) {
    if (!p || !out || n < 0 || first < 0) return ffail(COMET_ERR_INVALID_ARG, "problem, out and n >= 0 are required");
    if (instance < 0 || instance >= (int)p->inst.size()) return ffail(COMET_ERR_INVALID_ARG, "instance out of range");
    const comet_instance_desc& d = p->inst[instance];
    if (grammar != COMET_GRAMMAR_NONE && grammar != COMET_GRAMMAR_PUSH)
        return ffail(COMET_ERR_INVALID_ARG, "unknown grammar");
    if (grammar == COMET_GRAMMAR_PUSH && (d.task != COMET_TASK_PUSHER_SLIDER || d.n_modes != 13))
        return ffail(COMET_ERR_INVALID_ARG, "the pushing grammar needs a pushing instance with n_modes = 13");
    if (n == 0) return COMET_OK;
    SampleSpec sp;
    memset(&sp, 0, sizeof(sp));
    sp.instance = instance;
    sp.n_modes = d.n_modes;
    sp.lmax = d.max_segments;
    sp.grammar = grammar;
    // order counts per length (they fit in 64 bits: the mode codes do)
    const int alpha[5] = {0, 3, 6, 9, 12};
    auto ok = [](int a, int b) {
        if (a == b) return false;
        if (a == 12 || b == 12) return true;
        const int dd = ((a / 3 - b / 3) % 4 + 4) % 4;
        return dd == 1 || dd == 3;
    };
    if (grammar == COMET_GRAMMAR_PUSH) {
        for (int a = 0; a < 5; ++a) sp.comp[0][a] = 1;
        for (int r = 1; r < sp.lmax; ++r)
            for (int a = 0; a < 5; ++a) {
                unsigned long long c = 0;
                for (int b = 0; b < 5; ++b)
                    if (ok(alpha[a], alpha[b])) c += sp.comp[r - 1][b];
                sp.comp[r][a] = c;
            }
        for (int L = 1; L <= sp.lmax; ++L) sp.per_len[L - 1] = sp.comp[L - 1][4];  // starting in free motion
    } else {
        unsigned long long c = 1;
        for (int L = 1; L <= sp.lmax; ++L) {
            c *= (unsigned long long)sp.n_modes;
            sp.per_len[L - 1] = c;
        }
    }
    for (int L = 1; L <= sp.lmax; ++L) sp.total += sp.per_len[L - 1];
    cudaStream_t s = p->stream;
    const bool dev = dev_ptr(out);
    DevBuf buf;
    comet_mode_seq* d_out = out;
    if (!dev) {
        FTRY(cudaMalloc(&buf.p, sizeof(comet_mode_seq) * n), "sample buffer");
        d_out = (comet_mode_seq*)buf.p;
    }
    sample_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sp, seed, first, n, d_out);
    FTRY(cudaGetLastError(), "sample kernel");
    if (!dev) {
        FTRY(cudaMemcpyAsync(out, d_out, sizeof(comet_mode_seq) * n, cudaMemcpyDeviceToHost, s), "copy samples");
        FTRY(cudaStreamSynchronize(s), "synchronise");
    }
    return COMET_OK;
}
