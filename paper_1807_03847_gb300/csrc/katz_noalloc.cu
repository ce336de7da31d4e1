// katz_certify_topk_noalloc: certify a top-k ranking from per-node bounds
// without allocating anything.
//
// Some callers cannot let a library call cudaMalloc or cudaFree.  A serving
// process that hands all device memory to its own caching allocator at start
// (PyTorch's, for one) has none left for a library, and must keep every byte
// accounted for in its pool.  A latency-bound loop cannot afford cudaFree,
// which waits for the whole device to go idle and so stalls every other
// stream.  A plug-in host may forbid device allocation by the code it loads.
// For such callers this entry point takes the bounds and the output buffers
// from the caller and keeps its working memory in one file-scope __device__
// array of fixed size, present on every device that loads the library.
//
// Its work is the selection and checking half of an iteration of the
// library's main loop (a radix select of the k largest lower bounds, a
// one-CTA sort of them, and the separation count), run over all n nodes.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/katz.h"

namespace {

constexpr int NA_BINS = 65536;          // 16-bit digits
constexpr int NA_CAP = KATZ_MAX_K;      // candidates sorted in one CTA
constexpr int NA_THREADS = 1024;
constexpr int NA_MAX_DEVICES = 64;

struct NoAllocScratch {
    unsigned int hist[NA_BINS];
    unsigned long long cand_count;
    unsigned long long cross;
    unsigned long long above;      // keys known to lie above the current bucket
    unsigned long long k_rem;      // rank of the k-th key inside the current bucket
    unsigned long long pre_hi;     // selected digits so far (96-bit key: hi 64, lo 32)
    unsigned int pre_lo;
    int done;                      // threshold found
    int pairs_bad;
    int pad;
    unsigned long long thr_hi;     // candidates: key >= (thr_hi, thr_lo)
    unsigned int thr_lo;
    double theta;                  // k-th lower bound
    int theta_id;
    unsigned long long theta_key;
    double cand_l[NA_CAP];
    double cand_u[NA_CAP];
    int cand_id[NA_CAP];
};

// The working memory of every call on this device (at most 420 KiB).  Calls
// that overlap on the GPU (different streams) race on it.
__device__ __align__(256) NoAllocScratch g_noalloc;

std::mutex g_addr_mu;
NoAllocScratch* g_addr[NA_MAX_DEVICES] = {};
int g_sms[NA_MAX_DEVICES] = {};  // multiprocessors of each device (grid size of the O(n) passes)

typedef unsigned __int128 u128;

// 64-bit key whose unsigned order is the order of the doubles (negative
// values included), then the complemented id: one 96-bit key per node whose
// descending order is (lower bound desc, id asc)
__device__ __forceinline__ unsigned long long order_bits(double l) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(l);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ u128 key_of(double l, int v) {
    return ((u128)order_bits(l) << 32) | (u128)(0xffffffffu ^ (unsigned)v);
}

__global__ void na_reset(NoAllocScratch* S, long long k) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NA_BINS; q += gridDim.x * blockDim.x) S->hist[q] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S->cand_count = 0;
        S->cross = 0;
        S->above = 0;
        S->k_rem = (unsigned long long)k;
        S->pre_hi = 0;
        S->pre_lo = 0;
        S->done = 0;
        S->pairs_bad = 0;
    }
}

// histogram of digit `pass` (bits 95-16*pass .. 80-16*pass) of the keys that
// share the digits chosen so far; the lanes of a warp that hit the same bin
// (bounds of one magnitude share their top digits) add once
__global__ void na_hist(NoAllocScratch* S, const double* __restrict__ lower, long long n, int pass) {
    if (S->done) return;
    const int shift = 80 - 16 * pass;
    const u128 pre = ((u128)S->pre_hi << 32) | S->pre_lo;
    const int lane = threadIdx.x & 31;
    // base is the same for every thread of a block, so the loop is warp-uniform
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += (long long)gridDim.x * blockDim.x) {
        const long long v = base + threadIdx.x;
        unsigned bin = 0x10000u;  // none
        if (v < n) {
            const u128 key = key_of(lower[v], (int)v);
            if (pass == 0 || (key >> (shift + 16)) == (pre >> (shift + 16))) bin = (unsigned)(key >> shift) & 0xffffu;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        if (bin < 0x10000u && lane == __ffs(peers) - 1) atomicAdd(&S->hist[bin], (unsigned)__popc(peers));
    }
}

// pick the bucket that holds the k-th key; stop once all keys from that
// bucket up fit the candidate buffer
__global__ void na_find(NoAllocScratch* S, int pass) {
    __shared__ unsigned long long part[NA_THREADS];
    __shared__ int sel;
    __shared__ unsigned long long cum_sel;
    if (S->done) return;
    const int tid = threadIdx.x;
    constexpr int per = NA_BINS / NA_THREADS;
    // thread tid owns bins [NA_BINS-1 - tid*per - (per-1), NA_BINS-1 - tid*per], visited from the top
    unsigned long long s = 0;
    for (int q = 0; q < per; ++q) s += S->hist[NA_BINS - 1 - tid * per - q];
    part[tid] = s;
    if (tid == 0) sel = -1;
    __syncthreads();
    for (int off = 1; off < NA_THREADS; off <<= 1) {
        const unsigned long long a = tid >= off ? part[tid - off] : 0ull;
        __syncthreads();
        part[tid] += a;
        __syncthreads();
    }
    const unsigned long long k = S->k_rem;
    unsigned long long cum = tid ? part[tid - 1] : 0ull;
    if (cum < k && part[tid] >= k) {
        for (int q = 0; q < per; ++q) {
            const int b = NA_BINS - 1 - tid * per - q;
            const unsigned long long h = S->hist[b];
            if (cum + h >= k) {
                sel = b;
                cum_sel = cum;
                break;
            }
            cum += h;
        }
    }
    __syncthreads();
    const int b = sel;
    const unsigned long long hb = b >= 0 ? S->hist[b] : 0ull;
    __syncthreads();
    for (int q = tid; q < NA_BINS; q += NA_THREADS) S->hist[q] = 0;  // ready for the next pass
    if (tid == 0 && b >= 0) {
        const int shift = 80 - 16 * pass;
        const u128 pre = (((u128)S->pre_hi << 32) | S->pre_lo) | ((u128)(unsigned)b << shift);
        const unsigned long long above = S->above + cum_sel;
        if (above + hb <= (unsigned long long)NA_CAP || pass == 5) {
            S->done = 1;
            S->thr_hi = (unsigned long long)(pre >> 32);
            S->thr_lo = (unsigned int)pre;
        } else {
            S->above = above;
            S->k_rem = k - cum_sel;
            S->pre_hi = (unsigned long long)(pre >> 32);
            S->pre_lo = (unsigned int)pre;
        }
    }
}

__global__ void na_compact(NoAllocScratch* S, const double* __restrict__ lower, const double* __restrict__ upper,
                           long long n) {
    const u128 thr = ((u128)S->thr_hi << 32) | S->thr_lo;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        if (key_of(lower[v], (int)v) >= thr) {
            const unsigned long long pos = atomicAdd(&S->cand_count, 1ull);
            if (pos < (unsigned long long)NA_CAP) {
                S->cand_l[pos] = lower[v];
                S->cand_u[pos] = upper[v];
                S->cand_id[pos] = (int)v;
            }
        }
    }
}

struct Ent {
    unsigned long long key;
    int id;
    int src;
};

__device__ __forceinline__ bool before(const Ent& a, const Ent& b) {
    return a.key > b.key || (a.key == b.key && a.id < b.id);
}

// sort the candidates by (lower desc, id asc); the first k are the ranking,
// the k-th gives theta; adjacent top-k pairs must be eps-separated
__global__ void na_sort(NoAllocScratch* S, long long k, double eps, int32_t* ids_out) {
    extern __shared__ Ent e[];
    const int tid = threadIdx.x;
    const int cnt = (int)min((unsigned long long)NA_CAP, S->cand_count);
    int P = 1;
    while (P < cnt) P <<= 1;
    for (int q = tid; q < P; q += NA_THREADS)
        e[q] = q < cnt ? Ent{order_bits(S->cand_l[q]), S->cand_id[q], q} : Ent{0ull, 0x7fffffff, -1};
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int q = tid; q < (P >> 1); q += NA_THREADS) {
                const int pos = 2 * q - (q & (stride - 1));
                const Ent a = e[pos], b = e[pos + stride];
                const bool up = (pos & size) == 0;
                if (up ? before(b, a) : before(a, b)) {
                    e[pos] = b;
                    e[pos + stride] = a;
                }
            }
            __syncthreads();
        }
    }
    const int kk = (int)min((long long)cnt, k);
    for (int q = tid; q < kk; q += NA_THREADS) {
        ids_out[q] = e[q].id;
        if (q > 0 && __dsub_rn(S->cand_u[e[q].src], eps) >= S->cand_l[e[q - 1].src]) S->pairs_bad = 1;
    }
    if (tid == 0 && kk > 0) {
        S->theta = S->cand_l[e[kk - 1].src];
        S->theta_id = e[kk - 1].id;
        S->theta_key = e[kk - 1].key;
    }
}

// every node outside the top-k must be eps-separated from the k-th
__global__ void na_cross(NoAllocScratch* S, const double* __restrict__ lower, const double* __restrict__ upper,
                         long long n, double eps) {
    const double th = S->theta;
    const u128 th_key = ((u128)S->theta_key << 32) | (u128)(0xffffffffu ^ (unsigned)S->theta_id);
    unsigned long long c = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const bool in_top = key_of(lower[v], (int)v) >= th_key;
        if (!in_top && __dsub_rn(upper[v], eps) >= th) ++c;
    }
    for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&S->cross, c);
}

__global__ void na_finish(NoAllocScratch* S, int32_t* certified_out) {
    *certified_out = (S->cross == 0 && !S->pairs_bad) ? 1 : 0;
}

// Address of the scratch array on the current device and the device's
// multiprocessor count, resolved once per device.
katz_status scratch_on_current_device(NoAllocScratch** out, int* sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return KATZ_ECUDA;
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        int count = 0;
        if (cudaGetSymbolAddress(&p, g_noalloc) != cudaSuccess) return KATZ_ECUDA;
        if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || count < 1)
            return KATZ_ECUDA;
        if (cudaFuncSetAttribute(na_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 NA_CAP * (int)sizeof(Ent)) != cudaSuccess)
            return KATZ_ECUDA;
        g_sms[dev] = count;
        g_addr[dev] = (NoAllocScratch*)p;
    }
    *out = g_addr[dev];
    *sms = g_sms[dev];
    return KATZ_OK;
}

}  // namespace

extern "C" katz_status katz_certify_topk_noalloc(const double* lower, const double* upper, int64_t n, int64_t k,
                                                 double eps, int32_t* ids_out, int32_t* certified_out,
                                                 void* cuda_stream) {
    if (!lower || !upper || !ids_out || !certified_out) return KATZ_EINVAL;
    if (n < 1 || n > 0x7ffffffeLL || k < 1 || k > n || k > KATZ_MAX_K || !(eps > 0.0)) return KATZ_EINVAL;
    static_assert(sizeof(NoAllocScratch) <= 420 * 1024, "the stated size of the array");
    // an error left by the caller's earlier work stays the caller's: it is
    // neither cleared here nor reported as a failure of this call's launches
    if (cudaPeekAtLastError() != cudaSuccess) return KATZ_ECUDA;
    NoAllocScratch* S = nullptr;
    int sms = 0;
    katz_status st = scratch_on_current_device(&S, &sms);
    if (st != KATZ_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const long long cap = 8LL * sms;  // eight 256-thread blocks per multiprocessor, grid-stride beyond
    const int grid = (int)((n + 255) / 256 < cap ? (n + 255) / 256 : cap);
    na_reset<<<64, 1024, 0, s>>>(S, (long long)k);
    for (int pass = 0; pass < 6; ++pass) {
        na_hist<<<grid, 256, 0, s>>>(S, lower, (long long)n, pass);
        na_find<<<1, NA_THREADS, 0, s>>>(S, pass);
    }
    na_compact<<<grid, 256, 0, s>>>(S, lower, upper, (long long)n);
    na_sort<<<1, NA_THREADS, NA_CAP * sizeof(Ent), s>>>(S, (long long)k, eps, ids_out);
    na_cross<<<grid, 256, 0, s>>>(S, lower, upper, (long long)n, eps);
    na_finish<<<1, 1, 0, s>>>(S, certified_out);
    return cudaGetLastError() == cudaSuccess ? KATZ_OK : KATZ_ECUDA;
}
