// expand.cu -- device side of the greedy local mode expansion (Sec. III-B,
// Algorithm 1): the evaluated set V as a code list plus an open-addressing
// hash set, top-k of V by (M_hat, code), one-edit neighbourhoods of the top
// k in enumeration order, deduplication against V and within the round, and
// compaction of the first B unseen orders into the next batch F_{s+1}.
//
// Every count lives in device memory and every launch has a fixed grid, so
// a whole expansion round can be captured in a CUDA graph.

#include <cuda_runtime.h>
#include <stdint.h>

#include "comet.h"
#include "comet_internal.h"
#include "expand_internal.h"

namespace comet {
namespace {

constexpr unsigned long long kEmpty = 0ull;  // code 0 is never a valid order (length >= 1)

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    // SplitMix64 finaliser (Steele, Lea and Flood 2014) as the hash
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

// order-preserving map of a float to an unsigned key (NaN -> largest)
__device__ __forceinline__ uint32_t float_key(float f) {
    if (f != f) return 0xffffffffu;
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ bool key_less(const TopKey& a, const TopKey& b) {
    return a.mk < b.mk || (a.mk == b.mk && a.code < b.code);
}

__device__ unsigned long long encode_seq(const comet_mode_seq& s, int n_modes) {
    const unsigned long long base = (unsigned long long)(n_modes + 1);
    unsigned long long code = s.len, p = base;
    for (int i = 0; i < s.len; ++i) {
        code += (unsigned long long)(s.modes[i] + 1) * p;
        p *= base;
    }
    return code;
}

__device__ int decode_code(unsigned long long code, int n_modes, uint16_t* modes) {
    const unsigned long long base = (unsigned long long)(n_modes + 1);
    const int L = (int)(code % base);
    code /= base;
    for (int i = 0; i < L; ++i) {
        modes[i] = (uint16_t)(code % base - 1);
        code /= base;
    }
    return L;
}

// insert; returns true if the code was not present
__device__ bool set_insert(unsigned long long* set, unsigned long long mask, unsigned long long code) {
    unsigned long long h = mix64(code) & mask;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        const unsigned long long prev = atomicCAS(&set[h], kEmpty, code);
        if (prev == kEmpty) return true;
        if (prev == code) return false;
        h = (h + 1) & mask;
    }
    return false;  // table full (capacity is twice the maximum count, so unreachable)
}

__device__ bool set_contains(const unsigned long long* set, unsigned long long mask, unsigned long long code) {
    unsigned long long h = mix64(code) & mask;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        const unsigned long long v = set[h];
        if (v == code) return true;
        if (v == kEmpty) return false;
        h = (h + 1) & mask;
    }
    return false;
}

// candidate table: code -> smallest ordinal proposing it
__device__ void cand_insert(unsigned long long* keys, unsigned int* ords, unsigned long long mask,
                            unsigned long long code, unsigned int ord) {
    unsigned long long h = mix64(code) & mask;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        const unsigned long long prev = atomicCAS(&keys[h], kEmpty, code);
        if (prev == kEmpty || prev == code) {
            atomicMin(&ords[h], ord);
            return;
        }
        h = (h + 1) & mask;
    }
}

__device__ unsigned int cand_min(const unsigned long long* keys, const unsigned int* ords, unsigned long long mask,
                                 unsigned long long code) {
    unsigned long long h = mix64(code) & mask;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        if (keys[h] == code) return ords[h];
        if (keys[h] == kEmpty) break;
        h = (h + 1) & mask;
    }
    return 0xffffffffu;
}

// ------------------------------------------------------------- add to V

__global__ void add_kernel(FrontierDev F, const comet_mode_seq* seqs, int64_t n, const int64_t* d_n, const float* cost,
                           const float* viol, float eps_feas, float merit_mu) {
    const int64_t nn = d_n ? *d_n : n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const comet_mode_seq s = seqs[i];
        if (s.instance != F.instance || s.len < 1 || s.len > F.lmax) {
            atomicExch(F.error, 1);
            continue;
        }
        const unsigned long long code = encode_seq(s, F.n_modes);
        if (!set_insert(F.set, F.set_mask, code)) continue;  // already evaluated
        const unsigned long long slot = atomicAdd(F.nV, 1ull);
        if (slot >= (unsigned long long)F.capacity) {
            atomicExch(F.error, 2);
            continue;
        }
        const float c = cost[i], v = viol[i];
        // Eq. search_merit; a non-finite score ranks last
        float m = c + merit_mu * fmaxf(v - eps_feas, 0.f);
        if (!(m == m) || isinf(m)) m = __int_as_float(0x7f800000);
        F.codes[slot] = code;
        F.merit[slot] = m;
    }
}

// ---------------------------------------------------------------- top-k
// Each CTA sorts a chunk of kChunk keys (bitonic, shared memory) and writes
// its k smallest, in order, to out[block * k ...].

__global__ void topk_chunk_kernel(const TopKey* in_keys, const unsigned long long* codes, const float* merit,
                                  const unsigned long long* n_in_dev, int64_t n_in_fixed, int k, TopKey* out) {
    extern __shared__ TopKey sk[];
    // |V| may have run past the capacity (flagged on add): never read beyond it
    const int64_t n_in = n_in_dev ? min((int64_t)*n_in_dev, n_in_fixed) : n_in_fixed;
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    for (int t = threadIdx.x; t < kChunk; t += blockDim.x) {
        const int64_t i = base + t;
        TopKey key;
        if (i < n_in) {
            if (in_keys) {
                key = in_keys[i];
            } else {
                key.mk = float_key(merit[i]);
                key.idx = (uint32_t)i;
                key.code = codes[i];
            }
        } else {
            key.mk = 0xffffffffu;
            key.idx = 0xffffffffu;
            key.code = ~0ull;
        }
        sk[t] = key;
    }
    __syncthreads();
    for (int size = 2; size <= kChunk; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < kChunk / 2; t += blockDim.x) {
                const int lo = 2 * stride * (t / stride) + (t % stride);
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);
                TopKey a = sk[lo], b = sk[hi];
                if (key_less(b, a) == up) {
                    sk[lo] = b;
                    sk[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < k; t += blockDim.x) out[(int64_t)blockIdx.x * k + t] = sk[t];
}

// --------------------------------------------------------- neighbourhood


// Mode of alphabet position a: every mode (grammar 0), or for the pushing
// grammar stick on face a (mode 3 a, a < 4) and free motion (a = 4).
__device__ __forceinline__ int alpha_mode(const FrontierDev& F, int a) {
    return F.grammar == kGrammarPush ? (a < 4 ? 3 * a : kPushFree) : a;
}

// Pushing grammar (Sec. III-A; the reading fixed by the paper's printed
// counts): the order starts in free motion, no two consecutive segments
// share a mode, every mode is stick-on-a-face or free, and a direct
// contact-to-contact switch joins adjacent faces of the cyclic face list.
__device__ bool admissible(const FrontierDev& F, const uint16_t* s, int L) {
    if (F.grammar != kGrammarPush) return true;
    if (L < 1 || s[0] != kPushFree) return false;
    for (int i = 0; i < L; ++i)
        if (s[i] != kPushFree && (s[i] % 3 != 0 || s[i] >= 12)) return false;
    for (int i = 0; i + 1 < L; ++i) {
        const int a = s[i], b = s[i + 1];
        if (a == b) return false;
        if (a != kPushFree && b != kPushFree) {
            const int d = (a / 3 - b / 3 + 4) & 3;
            if (d != 1 && d != 3) return false;
        }
    }
    return true;
}

// One-edit neighbour of seq (length L) at slot j of the fixed layout:
// substitutions (position < l_max, alphabet position; the current mode is
// skipped), insertions (position <= l_max, alphabet position), deletions
// (position < l_max).  Slots that do not apply to this L are empty.  Within
// an order the slots run in the enumeration order of the neighbourhood.
// Returns the new length, or 0 for an empty slot.
__device__ int neighbour(const FrontierDev& F, const uint16_t* s, int L, int j, uint16_t* out) {
    const int nA = F.n_alpha, lmax = F.lmax;
    if (j < lmax * nA) {
        const int pos = j / nA, m = alpha_mode(F, j % nA);
        if (pos >= L || m == s[pos]) return 0;
        for (int i = 0; i < L; ++i) out[i] = s[i];
        out[pos] = (uint16_t)m;
        return L;
    }
    j -= lmax * nA;
    if (j < (lmax + 1) * nA) {
        const int pos = j / nA, m = alpha_mode(F, j % nA);
        if (L + 1 > lmax || pos > L) return 0;
        for (int i = 0, o = 0; i <= L; ++i) {
            if (i == pos) out[o++] = (uint16_t)m;
            if (i < L) out[o++] = s[i];
        }
        return L + 1;
    }
    j -= (lmax + 1) * nA;
    if (j < lmax && L - 1 >= 1 && j < L) {
        for (int i = 0, o = 0; i < L; ++i)
            if (i != j) out[o++] = s[i];
        return L - 1;
    }
    return 0;
}

// N_r(m) slot j (Sec. III-B): j < slots1 is a one-edit neighbour; with
// radius 2, j = slots1 + j1 slots1 + j2 is neighbour j2 of neighbour j1 (so
// the one-edit orders come first, then the two-edit ones grouped by their
// intermediate).  Every order on the way must be admissible; the parent
// itself is not a neighbour.  Returns the length, or 0.
__device__ int neighbour_r(const FrontierDev& F, const uint16_t* s, int L, int j, uint16_t* out) {
    if (j < F.slots1) {
        const int Ln = neighbour(F, s, L, j, out);
        return (Ln > 0 && admissible(F, out, Ln)) ? Ln : 0;
    }
    j -= F.slots1;
    uint16_t mid[COMET_MAX_SEGMENTS];
    const int Lm = neighbour(F, s, L, j / F.slots1, mid);
    if (Lm == 0 || !admissible(F, mid, Lm)) return 0;
    const int Ln = neighbour(F, mid, Lm, j % F.slots1, out);
    if (Ln == 0 || !admissible(F, out, Ln)) return 0;
    if (Ln == L) {
        bool same = true;
        for (int i = 0; i < L; ++i) same = same && out[i] == s[i];
        if (same) return 0;
    }
    return Ln;
}

__global__ void neighbour_kernel(FrontierDev F, const TopKey* top, int k, int64_t slots) {
    const int64_t total = (int64_t)k * slots;
    const unsigned long long nV = min(*F.nV, (unsigned long long)F.capacity);
    const int kk = (int)min((unsigned long long)k, nV);
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(o / slots);
        const int j = (int)(o - (int64_t)r * slots);
        unsigned long long code = kEmpty;
        if (r < kk) {
            uint16_t s[COMET_MAX_SEGMENTS], nb[COMET_MAX_SEGMENTS];
            const int L = decode_code(top[r].code, F.n_modes, s);
            const int Ln = neighbour_r(F, s, L, j, nb);
            if (Ln > 0) {
                comet_mode_seq q;
                q.len = (uint8_t)Ln;
                for (int i = 0; i < Ln; ++i) q.modes[i] = nb[i];
                code = encode_seq(q, F.n_modes);
                if (set_contains(F.set, F.set_mask, code))
                    code = kEmpty;  // already in V
                else
                    cand_insert(F.cand_keys, F.cand_ord, F.cand_mask, code, (unsigned int)o);
            }
        }
        F.cand_code[o] = code;
    }
}

// winners (first proposal of each unseen code) -> flags
__global__ void winner_kernel(FrontierDev F, int64_t total) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long code = F.cand_code[o];
        int flag = 0;
        if (code != kEmpty) flag = cand_min(F.cand_keys, F.cand_ord, F.cand_mask, code) == (unsigned int)o;
        F.flag[o] = flag;
    }
}

// single-CTA exclusive scan over the flags in ordinal order; the first
// `batch` winners (capped by the remaining evaluation budget) become F_{s+1}
__global__ void compact_kernel(FrontierDev F, int64_t total, int batch, int64_t budget) {
    __shared__ int warp_sums[32];
    __shared__ int carry;
    const unsigned long long nV = min(*F.nV, (unsigned long long)F.capacity);
    int64_t cap = batch;
    if (budget > 0) cap = min(cap, budget - (int64_t)nV);
    if (cap < 0) cap = 0;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < total; base += blockDim.x) {
        const int64_t o = base + threadIdx.x;
        const int f = (o < total) ? F.flag[o] : 0;
        // block-wide inclusive scan of f
        int v = f;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int d = 1; d < 32; d <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += x;
        }
        if (lane == 31) warp_sums[w] = v;
        __syncthreads();
        if (w == 0) {
            int s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
            for (int d = 1; d < 32; d <<= 1) {
                const int x = __shfl_up_sync(0xffffffffu, s, d);
                if (lane >= d) s += x;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const int excl = carry + (w > 0 ? warp_sums[w - 1] : 0) + v - f;
        if (f && excl < cap) {
            comet_mode_seq q;
            const unsigned long long code = F.cand_code[o];
            uint16_t m[COMET_MAX_SEGMENTS];
            const int L = decode_code(code, F.n_modes, m);
            q.instance = F.instance;
            q.len = (uint8_t)L;
            for (int i = 0; i < COMET_MAX_SEGMENTS; ++i) q.modes[i] = (i < L) ? m[i] : 0;
            q.pad[0] = q.pad[1] = q.pad[2] = 0;
            F.next[excl] = q;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + f;
        __syncthreads();
    }
    if (threadIdx.x == 0) *F.n_next = min((int64_t)carry, cap);
}

}  // namespace

size_t topk_smem_bytes() { return sizeof(TopKey) * kChunk; }

// V's codes back into the (cleared) hash set after a checkpoint restored
// codes[0..n) and merit[0..n)
__global__ void restore_kernel(FrontierDev F, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        set_insert(F.set, F.set_mask, F.codes[i]);
}

cudaError_t launch_frontier_restore(const FrontierDev& F, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, 4096);
    restore_kernel<<<blocks, threads, 0, s>>>(F, n);
    return cudaGetLastError();
}

cudaError_t launch_frontier_add(const FrontierDev& F, const comet_mode_seq* seqs, int64_t n, const int64_t* d_n,
                                const float* cost, const float* viol, float eps_feas, float merit_mu, cudaStream_t s) {
    const int64_t work = d_n ? F.batch_cap : n;
    if (work <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((work + threads - 1) / threads, 4096);
    add_kernel<<<blocks, threads, 0, s>>>(F, seqs, n, d_n, cost, viol, eps_feas, merit_mu);
    return cudaGetLastError();
}

cudaError_t prepare_expand() {
    // shared-memory attribute of the top-k kernel, once per device (not a
    // stream operation: called at frontier creation, outside any capture)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static bool done[64] = {};
    if (dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(topk_chunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)topk_smem_bytes());
    if (e == cudaSuccess && dev < 64) done[dev] = true;
    return e;
}

const TopKey* launch_topk(const FrontierDev& F, int k, cudaStream_t s, cudaError_t* err) {
    cudaError_t e = prepare_expand();
    *err = e;
    if (e != cudaSuccess) return nullptr;
    // chunk passes until one chunk remains; the first pass reads V directly
    int64_t n_in = F.capacity;
    const TopKey* in = nullptr;
    TopKey* bufs[2] = {F.top_a, F.top_b};
    int which = 0;
    bool first = true;
    for (;;) {
        const int64_t chunks = (n_in + kChunk - 1) / kChunk;
        topk_chunk_kernel<<<(unsigned)chunks, 1024, topk_smem_bytes(), s>>>(
            in, F.codes, F.merit, first ? F.nV : nullptr, n_in, k, bufs[which]);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            *err = e;
            return nullptr;
        }
        first = false;
        in = bufs[which];
        n_in = chunks * k;
        which ^= 1;
        if (chunks == 1) break;
    }
    return in;
}

cudaError_t launch_expand(const FrontierDev& F, int k, int batch, int64_t budget, cudaStream_t s) {
    cudaError_t e;
    const TopKey* top = launch_topk(F, k, s, &e);
    if (!top) return e;

    const int64_t slots = F.slots;
    const int64_t total = (int64_t)k * slots;
    e = cudaMemsetAsync(F.cand_keys, 0, sizeof(unsigned long long) * (F.cand_mask + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(F.cand_ord, 0xff, sizeof(unsigned int) * (F.cand_mask + 1), s);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((total + threads - 1) / threads, 4096);
    neighbour_kernel<<<blocks, threads, 0, s>>>(F, top, k, slots);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    winner_kernel<<<blocks, threads, 0, s>>>(F, total);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    compact_kernel<<<1, 1024, 0, s>>>(F, total, batch, budget);
    return cudaGetLastError();
}

}  // namespace comet
