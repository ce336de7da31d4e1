// Device kernels of the static bound iteration (Algorithm 1).
//
// One iteration r (all on one stream, no host round trip):
//   spmv         (katz_spmv.cu) s_r, c_r, bounds, candidates
//   select_topk  theta_r = k-th largest l_r over M (ties by id): one CTA sorts
//                the candidates in shared memory; replaces partialSort.
//   count        deactivates nodes of M outside the top-k with
//                u_r - eps < theta_r and counts those that stay.
//   finalize     converged(): |M| > k -> false, else adjacent-pair check of
//                the sorted top-k; sets the loop condition.
#include <cooperative_groups.h>
#include <stdint.h>

#include "katz_common.cuh"

namespace katz {

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T ld_nc(const T* p) { return __ldg(p); }

template <typename T>
__device__ __forceinline__ T scale(double alpha, T sum);
template <>
__device__ __forceinline__ double scale<double>(double alpha, double sum) { return __dmul_rn(alpha, sum); }

template <typename T>
__device__ __forceinline__ T add(T a, T b);
template <>
__device__ __forceinline__ double add<double>(double a, double b) { return __dadd_rn(a, b); }

template <typename Off>
__global__ void validate_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t n,
                                int64_t nnz, unsigned long long* bad, int64_t* degmax) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long nb = 0;
    long long dm = 0;
    for (int64_t v = tid; v < n; v += stride) {
        const int64_t a = rowptr[v], b = rowptr[v + 1];
        if (b < a) ++nb;
        dm = max(dm, (long long)(b - a));
    }
    if (tid == 0 && ((int64_t)rowptr[0] != 0 || (int64_t)rowptr[n] != nnz)) ++nb;
    if (col) {  // NULL: the column entries are checked where they are first used
        for (int64_t j = tid; j < nnz; j += stride) {
            const int32_t x = col[j];
            if (x < 0 || (int64_t)x >= n) ++nb;
        }
    }
    for (int off = 16; off; off >>= 1) {
        nb += __shfl_xor_sync(FULL, nb, off);
        dm = max(dm, __shfl_xor_sync(FULL, dm, off));
    }
    if ((threadIdx.x & 31) == 0) {
        if (nb) atomicAdd(bad, nb);
        if (dm) atomicMax((unsigned long long*)degmax, (unsigned long long)dm);
    }
}

template <typename T>
__global__ void init_walk_kernel(T* walk, double* c, double* c32, double* lb, double* ub, uint8_t* active,
                                 IterParams p) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = tid; v < p.n; v += stride) {
        walk[v] = (T)1;  // s_0 = omega_0 = 1 (Alg. 1)
        c[v] = 0.0;      // c_0 = 0
        if (c32) c32[v] = 0.0;
        if (lb) {
            lb[v] = 0.0;
            ub[v] = 1.0 / 0.0;
        }
        active[v] = 1;   // M = V
    }
    for (int64_t s = tid; s < p.slots; s += stride) walk[(size_t)s * p.stride + p.n] = (T)0;  // sentinel
}

// ---------------------------------------------------------------------------
// theta_0: the k-th largest l_1.  l_1 is an increasing function of the degree
// (s_1 = alpha deg), so it is l_1 evaluated at the k-th largest degree.
// ---------------------------------------------------------------------------
template <typename Off>
__global__ void deg_hist_kernel(const Off* __restrict__ rowptr, int64_t n, int64_t top, uint32_t* hist) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;
        const long long d = v < n ? min((long long)(rowptr[v + 1] - rowptr[v]), (long long)top) : -1;
        const unsigned mask = __match_any_sync(FULL, d);
        if (d >= 0 && lane == __ffs(mask) - 1) atomicAdd(&hist[d], (uint32_t)__popc(mask));
    }
}

// theta_0 from the k-th largest degree: level 1 is always FP64, s_1 = alpha
// * deg, c64 = 0 + s_1, c32 = 0, and l_1 grows with the degree
template <typename T>
__device__ __forceinline__ void set_theta0(long long found, const IterParams& p, Ctrl* ctrl) {
    const T s1 = scale<T>(p.alpha, (T)found);
    const double sd = (double)s1;
    double l, u;
    node_bounds(add<double>(0.0, sd), 0.0, sd, p, bstate(ctrl, p), l, u);
    ctrl->theta_prev = l;
}

template <typename T>
__global__ void kth_degree_kernel(const uint32_t* __restrict__ hist, int64_t D, IterParams p, Ctrl* ctrl) {
    __shared__ unsigned long long part[SELECT_THREADS];
    __shared__ long long found;
    const int tid = threadIdx.x;
    const int64_t bins = D + 1;
    const int64_t chunk = (bins + SELECT_THREADS - 1) / SELECT_THREADS;
    // thread tid owns bins [D - (tid+1)*chunk + 1, D - tid*chunk], scanned from the top
    const int64_t top = D - (int64_t)tid * chunk;
    unsigned long long s = 0;
    for (int64_t b = top; b > top - chunk && b >= 0; --b) s += hist[b];
    part[tid] = s;
    if (tid == 0) found = 0;
    __syncthreads();
    for (int off = 1; off < SELECT_THREADS; off <<= 1) {
        unsigned long long add_v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += add_v;
        __syncthreads();
    }
    const unsigned long long before = tid ? part[tid - 1] : 0;
    if (before < (unsigned long long)p.k && part[tid] >= (unsigned long long)p.k) {
        unsigned long long cum = before;
        for (int64_t b = top; b > top - chunk && b >= 0; --b) {
            cum += hist[b];
            if (cum >= (unsigned long long)p.k) { found = b; break; }
        }
    }
    __syncthreads();
    if (tid == 0) set_theta0<T>(found, p, ctrl);
}

// theta_0 while the degree classes of the relabelling are exact: the k-th
// largest degree is the kk-th largest among the rows [a, b) of one class,
// whose degrees lie in (lo, lo + 2^bits]; a radix select of the offset
// d - lo - 1 over 11-bit digits from the top, each digit one shared-memory
// histogram of those rows.
template <typename Off, typename T>
__global__ void __launch_bounds__(SELECT_THREADS)
kth_degree_class_kernel(const Off* __restrict__ rowptr, int64_t a, int64_t b, int64_t lo, int bits, int64_t kk,
                        IterParams p, Ctrl* ctrl) {
    constexpr int DIGIT = 11;
    __shared__ unsigned int hist[1 << DIGIT];
    __shared__ int s_digit;
    __shared__ long long s_k;
    const int tid = threadIdx.x, lane = tid & 31;
    long long prefix = 0, k = kk;
    for (int hi = bits; hi > 0;) {
        const int w = min(DIGIT, hi), sh = hi - w, nb = 1 << w;
        for (int q = tid; q < nb; q += SELECT_THREADS) hist[q] = 0;
        if (tid == 0) {  // a valid fallback (the smallest value the digit can take)
            s_digit = 0;
            s_k = 1;
        }
        __syncthreads();
        for (int64_t u = a + tid; u < b; u += SELECT_THREADS) {
            const long long o = (long long)rowptr[u + 1] - (long long)rowptr[u] - lo - 1;
            if (o >= 0 && (o >> hi) == (prefix >> hi)) atomicAdd(&hist[(o >> sh) & (nb - 1)], 1u);
        }
        __syncthreads();
        if (tid < 32) {  // lane l sums the bins [top - per, top), counted from the highest bin down
            const int per = (nb + 31) / 32, top = nb - lane * per;
            unsigned long long sum = 0;
            for (int q = top - 1; q >= max(0, top - per); --q) sum += hist[q];
            unsigned long long incl = sum;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long y = __shfl_up_sync(FULL, incl, off);
                if (lane >= off) incl += y;
            }
            const unsigned long long excl = incl - sum;
            if (excl < (unsigned long long)k && incl >= (unsigned long long)k) {
                unsigned long long cum = excl;
                for (int q = top - 1; q >= max(0, top - per); --q) {
                    if (cum + hist[q] >= (unsigned long long)k) {
                        s_digit = q;
                        s_k = k - (long long)cum;
                        break;
                    }
                    cum += hist[q];
                }
            }
        }
        __syncthreads();
        prefix |= (long long)s_digit << sh;
        k = s_k;
        hi = sh;
        __syncthreads();  // hist, s_digit and s_k are rewritten by the next digit
    }
    if (tid == 0) set_theta0<T>(lo + 1 + prefix, p, ctrl);
}

// ---------------------------------------------------------------------------
// select: sort the candidates by (l desc, id asc) in shared memory; the k-th
// entry is theta_r and the first k entries are the current top-k.
// ---------------------------------------------------------------------------
struct SelEntry {
    unsigned long long key;  // bit pattern of l (monotone for l >= 0)
    int32_t id;
    int32_t src;             // index into the candidate arrays
};

__device__ __forceinline__ bool sel_before(const SelEntry& a, const SelEntry& b) {
    return a.key > b.key || (a.key == b.key && a.id < b.id);
}

// A bitonic sort of E * SELECT_THREADS entries by sel_before, entry
// e = j * SELECT_THREADS + tid held in register j of thread tid.  A compare
// at distance d pairs e with e ^ d: for d < 32 the partner is in the same
// warp (shuffles), for d >= SELECT_THREADS in the same thread, and only the
// distances in between go through shared memory (one barrier on each side).
// The first cnt entries of sel are sorted (the rest padding that sorts
// last); the first kk go out as the top-k and entry kk-1 gives theta.
__device__ __forceinline__ SelEntry shfl_entry(const SelEntry& a, int d) {
    SelEntry b;
    b.key = __shfl_xor_sync(FULL, a.key, d);
    b.id = __shfl_xor_sync(FULL, a.id, d);
    b.src = __shfl_xor_sync(FULL, a.src, d);
    return b;
}

// entry e holding `own` meets its partner's `other` in a network block of
// `size` (ascending when e & size == 0): it keeps the earlier of the two if
// it is the lower position of an ascending pair or the upper of a
// descending one, else the later.  Only padding entries compare equal, and
// those are identical.
__device__ __forceinline__ SelEntry pick(const SelEntry& own, const SelEntry& other, int e, int d, int size) {
    const bool lower = (e & d) == 0, up = (e & size) == 0;
    const bool own_first = sel_before(own, other);
    return (lower == up) == own_first ? own : other;
}

// the compares at distance DJ * SELECT_THREADS, inside each thread
template <int E, int DJ>
__device__ __forceinline__ void step_in_thread(SelEntry (&x)[E], int size, int tid) {
    if constexpr (DJ < E) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            if (j & DJ) continue;
            const int e = j * SELECT_THREADS + tid;
            const bool up = (e & size) == 0;
            const SelEntry a = x[j], b = x[j | DJ];
            const bool swap = up ? sel_before(b, a) : sel_before(a, b);
            x[j] = swap ? b : a;
            x[j | DJ] = swap ? a : b;
        }
    }
}

template <int E>
__device__ void sort_and_emit(SelEntry* sel, unsigned int cnt, int kk, const double* __restrict__ cu,
                              int32_t* topk_id, double* topk_l, double* topk_u, Ctrl* ctrl) {
    constexpr int P = E * SELECT_THREADS;
    const int tid = threadIdx.x;
    SelEntry x[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int e = j * SELECT_THREADS + tid;
        x[j] = e < (int)cnt ? sel[e] : SelEntry{0ULL, 0x7fffffff, -1};
    }
    for (int size = 2; size <= P; size <<= 1) {
        for (int d = size >> 1; d > 0; d >>= 1) {
            if (d >= SELECT_THREADS) {
                const int dj = d / SELECT_THREADS;  // 1, 2 or 4: register indices stay compile-time
                if (dj == 1) step_in_thread<E, 1>(x, size, tid);
                else if (dj == 2) step_in_thread<E, 2>(x, size, tid);
                else step_in_thread<E, 4>(x, size, tid);
            } else if (d >= 32) {
                __syncthreads();  // earlier readers of sel are done
#pragma unroll
                for (int j = 0; j < E; ++j) sel[j * SELECT_THREADS + tid] = x[j];
                __syncthreads();
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const int e = j * SELECT_THREADS + tid;
                    x[j] = pick(x[j], sel[e ^ d], e, d, size);
                }
            } else {
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const int e = j * SELECT_THREADS + tid;
                    x[j] = pick(x[j], shfl_entry(x[j], d), e, d, size);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int e = j * SELECT_THREADS + tid;
        if (e < kk) {
            topk_id[e] = x[j].id;
            topk_l[e] = __longlong_as_double((long long)x[j].key);
            topk_u[e] = cu[x[j].src];
        }
        if (e == kk - 1) {
            ctrl->theta = __longlong_as_double((long long)x[j].key);
            ctrl->theta_id = x[j].id;
        }
    }
}

// The candidate order as one 96-bit key: the bits of l (monotone for
// l >= 0), then the complemented id, so that descending keys are
// (l desc, id asc).
typedef unsigned __int128 u128;

__device__ __forceinline__ u128 cand_key(double l, int32_t id) {
    return ((u128)(unsigned long long)__double_as_longlong(l) << 32) | (u128)(0xffffffffu ^ (uint32_t)id);
}

// The min(k, |C|) largest keys of C = {candidates with l >= tau} gathered
// into sel, for a C larger than the shared-memory sort holds: a radix select
// of the k-th key inside this CTA (8-bit digits, most significant first,
// with a 256-bin shared histogram per digit; the select ends at the first
// digit whose bucket holds exactly the keys still missing), then one pass
// that gathers every key at or above it.  Returns the number gathered.
__device__ unsigned int select_large(const double* __restrict__ cl, const int32_t* __restrict__ cid,
                                     unsigned long long nc, double tau, long long k, SelEntry* sel) {
    __shared__ unsigned int hist[256];
    __shared__ unsigned long long s_pre_hi, s_krem;  // selected digits: key bits 95..32 ...
    __shared__ unsigned int s_pre_lo, s_cnt;         // ... and 31..0
    __shared__ int s_done;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        s_pre_hi = 0ull;
        s_pre_lo = 0u;
        s_krem = 0ull;
        s_done = 0;
        s_cnt = 0u;
    }
    for (int pass = 0; pass < 12; ++pass) {
        for (int q = tid; q < 256; q += SELECT_THREADS) hist[q] = 0u;
        __syncthreads();
        const int shift = 88 - 8 * pass;
        const u128 prefix = ((u128)s_pre_hi << 32) | s_pre_lo;
        for (unsigned long long q = tid; q < nc; q += SELECT_THREADS) {
            const double l = cl[q];
            if (!(l >= tau)) continue;
            const u128 key = cand_key(l, cid[q]);
            if (pass == 0 || (key >> (shift + 8)) == (prefix >> (shift + 8)))
                atomicAdd(&hist[(unsigned)(key >> shift) & 0xffu], 1u);
        }
        __syncthreads();
        if (tid == 0) {
            unsigned long long krem = s_krem;
            if (pass == 0) {
                unsigned long long total = 0;
                for (int b = 0; b < 256; ++b) total += hist[b];
                krem = min((unsigned long long)k, total);
            }
            if (krem == 0) {
                s_done = 2;  // no candidate
            } else {
                unsigned long long cum = 0;
                int bsel = 0;
                for (int b = 255; b >= 0; --b) {
                    if (cum + hist[b] >= krem) {
                        bsel = b;
                        break;
                    }
                    cum += hist[b];
                }
                const u128 pre = prefix | ((u128)bsel << shift);
                s_pre_hi = (unsigned long long)(pre >> 32);
                s_pre_lo = (unsigned int)pre;
                krem -= cum;
                if (hist[bsel] == krem) s_done = 1;  // the whole bucket is in: threshold = prefix, lower bits 0
                s_krem = krem;
            }
        }
        __syncthreads();
        if (s_done) break;
    }
    if (s_done == 2) return 0u;
    const u128 th = ((u128)s_pre_hi << 32) | s_pre_lo;
    for (unsigned long long base = 0; base < nc; base += SELECT_THREADS) {
        const unsigned long long q = base + tid;
        const double l = q < nc ? cl[q] : -1.0;
        const bool take = q < nc && l >= tau && cand_key(l, cid[q]) >= th;
        const unsigned m = __ballot_sync(FULL, take);
        unsigned int wpos = 0;
        if (lane == 0 && m) wpos = atomicAdd(&s_cnt, (unsigned int)__popc(m));
        wpos = __shfl_sync(FULL, wpos, 0);
        if (take) {
            const unsigned int pos = wpos + __popc(m & ((1u << lane) - 1u));
            if (pos < (unsigned int)SELECT_CAP)
                sel[pos] = SelEntry{(unsigned long long)__double_as_longlong(l), cid[q], (int32_t)q};
        }
    }
    __syncthreads();
    return min(s_cnt, (unsigned int)SELECT_CAP);
}

template <typename T>
__global__ void __launch_bounds__(SELECT_THREADS)
select_kernel(const double* __restrict__ cl, const double* __restrict__ cu, const int32_t* __restrict__ cid,
              const T* walk, const double* c, const double* c32, const double* lb, const int32_t* __restrict__ inv,
              int32_t* topk_id, double* topk_l, double* topk_u, Ctrl* ctrl, IterParams p) {
    extern __shared__ SelEntry sel[];
    __shared__ unsigned int s_cnt;
    __shared__ double s_tau;
    __shared__ int s_big;
    if (ctrl->stop) return;
    const int tid = threadIdx.x;
    const unsigned long long nc = ctrl->n_cand;
    const int r_cur = ctrl->r + 1;
    if (tid == 0) {
        s_cnt = 0;
        s_tau = -1.0;
        s_big = 0;
    }
    __syncthreads();
    {
        // Narrow the candidates: the previous top-k nodes are still active and
        // each has l_r >= tau := min of their l_r, so the top-k of M lies in
        // {l_r >= tau} (a far smaller sort than all of {l_r >= theta_{r-1}}).
        const int kprev = ctrl->k_eff;
        if (r_cur <= 1 || kprev < (int)p.k) {
            if (tid == 0 && nc > (unsigned long long)SELECT_CAP) s_big = 1;
        } else {
            const BState bs = bstate(ctrl, p);
            const int f32_from = ctrl->f32_from;
            double m = 1.0 / 0.0;
            for (int q = tid; q < kprev; q += SELECT_THREADS) {
                const int32_t v = inv[topk_id[q]];
                double l, u;
                if (p.cert) l = lb[v];
                else node_bounds(c[v], 0.0, walk_value(walk, p, f32_from, r_cur, v), p, bs, l, u);
                m = fmin(m, l);
            }
            for (int off = 16; off; off >>= 1) m = fmin(m, __shfl_xor_sync(FULL, m, off));
            __shared__ double wmin[SELECT_THREADS / 32];
            if ((tid & 31) == 0) wmin[tid >> 5] = m;
            __syncthreads();
            if (tid == 0) {
                double mm = wmin[0];
                for (int w = 1; w < SELECT_THREADS / 32; ++w) mm = fmin(mm, wmin[w]);
                s_tau = mm;
            }
        }
        __syncthreads();
    }
    const double tau = s_tau;
    unsigned int cnt = 0;
    if (!s_big) {
        // the candidates with l >= tau, one shared-memory atomic per warp
        const int lane = tid & 31;
        for (unsigned long long base = 0; base < nc; base += SELECT_THREADS) {
            const unsigned long long q = base + tid;
            const double l = q < nc ? cl[q] : -1.0;
            const bool take = q < nc && l >= tau;
            const unsigned m = __ballot_sync(FULL, take);
            unsigned int wpos = 0;
            if (lane == 0 && m) wpos = atomicAdd(&s_cnt, (unsigned int)__popc(m));
            wpos = __shfl_sync(FULL, wpos, 0);
            if (take) {
                const unsigned int pos = wpos + __popc(m & ((1u << lane) - 1u));
                if (pos < (unsigned int)SELECT_CAP)
                    sel[pos] = SelEntry{(unsigned long long)__double_as_longlong(l), cid[q], (int32_t)q};
            }
        }
        __syncthreads();
        cnt = s_cnt;
    }
    // more candidates than the sort holds: select the top k of them first,
    // here on the device (the loop never waits for the host)
    if (s_big || cnt > (unsigned int)SELECT_CAP) cnt = select_large(cl, cid, nc, tau, (long long)p.k, sel);
    const int kk = (int)min((long long)p.k, (long long)cnt);
    if (cnt <= (unsigned int)SELECT_THREADS) sort_and_emit<1>(sel, cnt, kk, cu, topk_id, topk_l, topk_u, ctrl);
    else if (cnt <= 2u * SELECT_THREADS) sort_and_emit<2>(sel, cnt, kk, cu, topk_id, topk_l, topk_u, ctrl);
    else if (cnt <= 4u * SELECT_THREADS) sort_and_emit<4>(sel, cnt, kk, cu, topk_id, topk_l, topk_u, ctrl);
    else sort_and_emit<8>(sel, cnt, kk, cu, topk_id, topk_l, topk_u, ctrl);
    if (tid == 0) {
        ctrl->k_eff = kk;
        ctrl->tau = tau;
    }
}

// ---------------------------------------------------------------------------
// count: deactivate nodes of M outside the top-k with u_r - eps < theta_r and
// count the ones that remain (converged() returns false if any remain).
//
// M is read from a compact list of its nodes: the first count after all
// nodes became active scans the flags of all of V instead.  Either way the
// survivors are written, in tiles, to the other list buffer (one atomic per
// tile for its place), which finalize then makes current.  The order of a
// list is arbitrary; nothing computed from it depends on the order.
// ---------------------------------------------------------------------------
constexpr int COUNT_THREADS = 256;
constexpr int COUNT_U = 4;  // nodes per thread and tile, their loads issued together
constexpr int COUNT_TILE = COUNT_THREADS * COUNT_U;

template <typename T>
__global__ void __launch_bounds__(COUNT_THREADS)
count_kernel(const T* walk, const double* __restrict__ c, const double* __restrict__ c32,
             const double* __restrict__ lb, const double* __restrict__ ub, const int32_t* __restrict__ perm,
             uint8_t* active, int32_t* alist0, int32_t* alist1, Ctrl* ctrl, IterParams p) {
    __shared__ int s_wcnt[COUNT_THREADS / 32];
    __shared__ unsigned long long s_base;
    if (ctrl->stop) return;
    const int r_cur = ctrl->r + 1;
    const int f32_from = ctrl->f32_from;
    const BState bs = bstate(ctrl, p);
    const double th = ctrl->theta;
    const int32_t thid = ctrl->theta_id;
    const bool full = !ctrl->list_ready;
    const int cur = ctrl->list_cur;
    const int32_t* in = cur ? alist1 : alist0;
    int32_t* out = cur ? alist0 : alist1;
    const int64_t total = full ? p.n : (int64_t)ctrl->n_list;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    unsigned long long cross = 0, act = 0;
    double roundw = 0.0;
    // cert mode: the maxima of s_r and, over nodes with c32 = +0 (all of them
    // before the switch to FP32 levels), of c64, taken on bit patterns (the
    // values are non-negative); the tail and rounding widths follow from them
    // below, because rounding a product with a non-negative factor is monotone
    long long smax_b = 0, cmax_b = 0;
    const double d64 = bs.hi64 - bs.lo64, d32 = bs.hi32 - bs.lo32;
    // l, th >= 0 (sums of non-negative terms): they order like their bit patterns
    const long long th_bits = __double_as_longlong(th);
    // the trip count depends on the block only, so the barriers below are uniform
    for (int64_t t0 = (int64_t)blockIdx.x * COUNT_TILE; t0 < total; t0 += (int64_t)gridDim.x * COUNT_TILE) {
        bool on[COUNT_U], keep[COUNT_U];
        int32_t v[COUNT_U];
#pragma unroll
        for (int q = 0; q < COUNT_U; ++q) {
            const int64_t i = t0 + q * COUNT_THREADS + tid;
            on[q] = i < total;
            v[q] = on[q] ? (full ? (int32_t)i : in[i]) : 0;
        }
        if (full) {
#pragma unroll
            for (int q = 0; q < COUNT_U; ++q) on[q] = on[q] && active[v[q]];
        }
        double l[COUNT_U], u[COUNT_U];
        int32_t ov[COUNT_U];
#pragma unroll
        for (int q = 0; q < COUNT_U; ++q) {
            l[q] = on[q] ? lb[v[q]] : 0.0;  // stored by the SpMV epilogue of this level
            u[q] = on[q] ? ub[v[q]] : 0.0;
            ov[q] = on[q] ? perm[v[q]] : 0;  // ties are broken by the original id
        }
        int mine = 0;
#pragma unroll
        for (int q = 0; q < COUNT_U; ++q) {
            keep[q] = false;
            if (!on[q]) continue;
            const long long l_bits = __double_as_longlong(l[q]);
            const bool top = l_bits > th_bits || (l_bits == th_bits && ov[q] <= thid);
            if (!top) {
                if (__dsub_rn(u[q], p.eps) < th) {
                    active[v[q]] = 0;
                    continue;
                }
                ++cross;
            }
            keep[q] = true;
            ++mine;
            if (p.cert) {
                const double sv = walk_value(walk, p, f32_from, r_cur, v[q]);
                const double c64v = c[v[q]], c32v = c32 ? c32[v[q]] : 0.0;
                smax_b = max(smax_b, __double_as_longlong(sv));
                if (__double_as_longlong(c32v) == 0) cmax_b = max(cmax_b, __double_as_longlong(c64v));
                else roundw = fmax(roundw, __fma_rn(c64v, d64, __dmul_rn(c32v, d32)));
            }
        }
        act += (unsigned long long)mine;
        // places of the survivors: scan within the warp, then over the warps
        int incl = mine;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) s_wcnt[wid] = incl;
        __syncthreads();
        if (tid == 0) {
            int run = 0;
            for (int w = 0; w < COUNT_THREADS / 32; ++w) {
                const int x = s_wcnt[w];
                s_wcnt[w] = run;
                run += x;
            }
            s_base = run ? atomicAdd(&ctrl->n_list_next, (unsigned long long)run) : 0ull;
        }
        __syncthreads();
        unsigned long long pos = s_base + (unsigned long long)(s_wcnt[wid] + incl - mine);
#pragma unroll
        for (int q = 0; q < COUNT_U; ++q)
            if (keep[q]) out[pos++] = v[q];
        __syncthreads();  // s_wcnt and s_base are rewritten by the next tile
    }
    double smax = 0.0, tailw = 0.0;
    if (p.cert) {
        smax = __longlong_as_double(smax_b);
        tailw = __dmul_rn(p.ag, smax);  // = the largest of ag s_r over this thread's nodes
        roundw = fmax(roundw, __dmul_rn(__longlong_as_double(cmax_b), d64));
    }
    // block totals first: one atomic per block and counter
    __shared__ unsigned long long s_cross[32], s_act[32];
    __shared__ double s_smax[32], s_tailw[32], s_roundw[32];
    for (int off = 16; off; off >>= 1) {
        cross += __shfl_xor_sync(FULL, cross, off);
        act += __shfl_xor_sync(FULL, act, off);
        smax = fmax(smax, __shfl_xor_sync(FULL, smax, off));
        tailw = fmax(tailw, __shfl_xor_sync(FULL, tailw, off));
        roundw = fmax(roundw, __shfl_xor_sync(FULL, roundw, off));
    }
    const int nw = blockDim.x >> 5;
    if (lane == 0) {
        s_cross[wid] = cross;
        s_act[wid] = act;
        s_smax[wid] = smax;
        s_tailw[wid] = tailw;
        s_roundw[wid] = roundw;
    }
    __syncthreads();
    if (wid == 0) {
        cross = lane < nw ? s_cross[lane] : 0ull;
        act = lane < nw ? s_act[lane] : 0ull;
        smax = lane < nw ? s_smax[lane] : 0.0;
        tailw = lane < nw ? s_tailw[lane] : 0.0;
        roundw = lane < nw ? s_roundw[lane] : 0.0;
        for (int off = 16; off; off >>= 1) {
            cross += __shfl_xor_sync(FULL, cross, off);
            act += __shfl_xor_sync(FULL, act, off);
            smax = fmax(smax, __shfl_xor_sync(FULL, smax, off));
            tailw = fmax(tailw, __shfl_xor_sync(FULL, tailw, off));
            roundw = fmax(roundw, __shfl_xor_sync(FULL, roundw, off));
        }
        if (lane == 0) {
            if (cross) atomicAdd(&ctrl->cnt_cross, cross);
            if (act) atomicAdd(&ctrl->n_active, act);
            if (p.cert) {  // non-negative doubles order like their bit patterns
                atomicMax(&ctrl->smax_bits, (unsigned long long)__double_as_longlong(smax));
                atomicMax(&ctrl->tailw_bits, (unsigned long long)__double_as_longlong(tailw));
                atomicMax(&ctrl->roundw_bits, (unsigned long long)__double_as_longlong(roundw));
            }
        }
    }
}

// gamma_m = m u / (1 - m u) (Higham), rounded up
__device__ __forceinline__ double gamma_up(double m, double u) {
    const double mu = __dmul_ru(m, u);
    return __ddiv_ru(mu, __dsub_rd(1.0, mu));
}

// FP32-certified mode: error bounds and widening factors of level `lvl`
// (relative error e_lvl of its stored s, the largest error e64 of the FP64
// levels, and how many terms the FP64 accumulations of c64 / c32 hold).
__device__ void set_level_state(Ctrl* ctrl, const IterParams& p, int lvl, double e_lvl, double a_lvl) {
    const double u64 = 0x1p-53;
    const int f32_from = ctrl->f32_from;
    ctrl->e_cur = e_lvl;
    if (lvl < f32_from) ctrl->e64 = e_lvl;
    const int n64 = lvl < f32_from ? lvl : f32_from - 1;
    const int n32 = lvl < f32_from ? 0 : lvl - f32_from + 1;
    // c_hat = sum of stored terms with relative errors <= e, accumulated in
    // FP64 (relative error <= (terms + 1) u64 for non-negative terms)
    const double w64 = __dadd_ru(ctrl->e64, __dmul_ru((double)(n64 + 2), u64));
    const double w32 = __dadd_ru(e_lvl, __dmul_ru((double)(n32 + 2), u64));
    ctrl->lo64 = __dsub_rd(1.0, w64);
    ctrl->hi64 = __dadd_ru(1.0, __dmul_ru(2.0, w64));
    ctrl->lo32 = n32 ? __dsub_rd(1.0, w32) : 1.0;
    ctrl->hi32 = n32 ? __dadd_ru(1.0, __dmul_ru(2.0, w32)) : 1.0;
    ctrl->los = __dsub_rd(1.0, e_lvl);
    ctrl->his = __dadd_ru(1.0, __dmul_ru(2.0, e_lvl));
    ctrl->tail_lo = __dmul_rd(p.alpha, ctrl->los);
    ctrl->tail_hi = __dmul_ru(p.ag_hi, ctrl->his);
    // With stored s_i = s_i (1 + t) + h, |t| <= e_i, |h| <= a_i on the FP32
    // levels: the exact FP32-level part of c lies in [c32 lo32 - a_sum,
    // c32 hi32 + 2 a_sum] (hi32 >= 1 / (1 - e)), the tail alpha gamma s_r
    // below s_r tail_hi + 2 alpha gamma a_r, and alpha s_r above
    // s_r tail_lo - alpha a_r.  Every node with a walk has c64 >= s_1 =
    // alpha deg >= alpha (level 1 is FP64), and a node without one has exact
    // zeros everywhere; so the absolute terms A are covered by the c64
    // factors: c64 (lo64 - A_lo / alpha) <= c64 lo64 - A_lo, likewise above.
    ctrl->a_cur = lvl < f32_from ? 0.0 : a_lvl;
    ctrl->a_sum = lvl < f32_from ? 0.0 : __dadd_ru(ctrl->a_sum, a_lvl);
    if (ctrl->a_sum > 0.0) {
        const double abs_hi = __dmul_ru(2.0, __fma_ru(p.ag_hi, ctrl->a_cur, ctrl->a_sum));
        const double abs_lo = p.undirected ? __fma_ru(p.alpha, ctrl->a_cur, ctrl->a_sum) : ctrl->a_sum;
        ctrl->hi64 = __dadd_ru(ctrl->hi64, __ddiv_ru(abs_hi, p.alpha));
        ctrl->lo64 = fmax(__dsub_rd(ctrl->lo64, __ddiv_ru(abs_lo, p.alpha)), 0.0);
    }
}

// error bound of level lvl from the bound of level lvl - 1
__device__ double next_error(const Ctrl* ctrl, const IterParams& p, int lvl, double e_prev) {
    const double g = lvl >= ctrl->f32_from ? gamma_up((double)(p.depth + 3), 0x1p-24)
                                          : gamma_up((double)(p.depth + 1), 0x1p-53);
    return __dsub_ru(__dmul_ru(__dadd_ru(1.0, e_prev), __dadd_ru(1.0, g)), 1.0);
}

// Absolute error bound of an FP32 level from that of level lvl - 1.  With
// gradual underflow an FP32 addition has no absolute error (a sum in the
// subnormal range is exact); a product or a conversion to FP32 may lose up to
// half the smallest subnormal, 2^-150.  The row sum of level lvl carries its
// inputs' absolute errors times alpha_f (1 + g) deg <= 1 + g (alpha D < 1),
// plus its own product; the first FP32 level's inputs are conversions.
__device__ double next_abs(const Ctrl* ctrl, const IterParams& p, int lvl, double a_prev) {
    if (lvl < ctrl->f32_from) return 0.0;
    const double half_sub = 0x1p-150;
    const double g = gamma_up((double)(p.depth + 3), 0x1p-24);
    const double in = lvl == ctrl->f32_from ? half_sub : a_prev;
    return __fma_ru(__dadd_ru(1.0, g), in, half_sub);
}

__global__ void cert_init_kernel(Ctrl* ctrl, IterParams p) {
    ctrl->f32_from = (p.cert && p.fp32_from >= 2) ? p.fp32_from : 0x7fffffff;
    ctrl->e64 = 0.0;
    ctrl->a_sum = 0.0;
    set_level_state(ctrl, p, 1, p.cert ? next_error(ctrl, p, 1, 0.0) : 0.0, 0.0);
}

// FP32-certified handles whose summation depth grew (an update batch made a
// row longer than its row mode's nominal limit): the error state of level r
// replayed from level 1 with the new depth.  This is the recursion the
// ranking ran level by level (cert_init, then finalize), with the switch
// level it chose; the repaired levels satisfy the larger bounds, and so do
// the levels left as they were.
__global__ void cert_replay_kernel(Ctrl* ctrl, IterParams p, int r) {
    if (!p.cert) return;
    ctrl->e64 = 0.0;
    ctrl->a_sum = 0.0;
    double e = 0.0, a = 0.0;
    for (int lvl = 1; lvl <= r; ++lvl) {
        e = next_error(ctrl, p, lvl, e);
        a = next_abs(ctrl, p, lvl, a);
        set_level_state(ctrl, p, lvl, e, a);
    }
}

__global__ void finalize_kernel(const double* __restrict__ topk_l, const double* __restrict__ topk_u,
                                int64_t* trace, Ctrl* ctrl, IterParams p, unsigned long long cond, int use_cond) {
    __shared__ int bad;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    __syncthreads();
    if (ctrl->stop) {  // the loop was already over: leave the device-side while loop too
        if (tid == 0 && use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0);
        return;
    }
    if (tid == 0) ctrl->body_runs += 1;
    const int kk = ctrl->k_eff;
    const bool none_cross = ctrl->cnt_cross == 0;
    if (none_cross) {
        for (int q = tid + 1; q < kk; q += blockDim.x)
            if (__dsub_rn(topk_u[q], p.eps) >= topk_l[q - 1]) bad = 1;
    }
    __syncthreads();
    if (tid == 0) {
        const int conv = none_cross && !bad;
        const int r_cur = ctrl->r + 1;
        if (r_cur <= p.r_max) trace[r_cur] = (int64_t)ctrl->n_active;
        ctrl->r = r_cur;
        ctrl->converged = conv;
        ctrl->theta_prev = ctrl->theta;
        ctrl->n_cand = 0;
        ctrl->cnt_cross = 0;
        ctrl->n_active = 0;
        // the survivors of this count become the active list
        ctrl->list_cur ^= 1;
        ctrl->n_list = ctrl->n_list_next;
        ctrl->n_list_next = 0;
        ctrl->list_ready = 1;
        int stop = conv || r_cur >= p.r_max;
        if (p.cert) {
            const double smax = __longlong_as_double((long long)ctrl->smax_bits);
            const double sprev = __longlong_as_double((long long)ctrl->smax_prev_bits);
            const double tailw = __longlong_as_double((long long)ctrl->tailw_bits);
            const double roundw = __longlong_as_double((long long)ctrl->roundw_bits);
            // stall: over the active set the rounding widening is wider than the
            // Theorem-1 tail term, so further iterations cannot separate it
            if (!conv && r_cur >= ctrl->f32_from && tailw < roundw) {
                ctrl->stall = 1;
                stop = 1;
            }
            if (!stop) {
                const int next = r_cur + 1;
                // switch to FP32 once the terms still to come (predicted from the
                // decay of max s_r over M) carry a rounding widening below eps/16
                if (ctrl->f32_from == 0x7fffffff && p.fp32_from == 0 && r_cur >= 2 && sprev > 0.0 &&
                    smax < 0.5 * sprev) {
                    const double rho = smax / sprev;
                    const double tail_est = smax * rho / (1.0 - rho);
                    const double e32 = ctrl->e_cur + 64.0 * gamma_up((double)(p.depth + 3), 0x1p-24);
                    if (2.0 * tail_est * e32 <= p.eps / 16.0) ctrl->f32_from = next;
                }
                set_level_state(ctrl, p, next, next_error(ctrl, p, next, ctrl->e_cur),
                                next_abs(ctrl, p, next, ctrl->a_cur));
            }
            ctrl->smax_prev_bits = ctrl->smax_bits;
            ctrl->smax_bits = 0;
            ctrl->tailw_bits = 0;
            ctrl->roundw_bits = 0;
        }
        ctrl->stop = stop;
        if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, stop ? 0u : 1u);
    }
}

template <typename T>
__global__ void bounds_out_kernel(const T* walk, const double* __restrict__ c, const double* __restrict__ c32,
                                  const double* __restrict__ lb, const double* __restrict__ ub,
                                  const uint8_t* __restrict__ active, const int32_t* __restrict__ inv,
                                  const Ctrl* ctrl, IterParams p, int level, double* lower, double* upper,
                                  double* err) {
    const BState bs = bstate(ctrl, p);
    const int f32_from = ctrl->f32_from;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += stride) {
        const int32_t w = inv[v];
        const double sv = walk_value(walk, p, f32_from, level, w);
        const double c32v = c32 ? c32[w] : 0.0;
        double l, u;
        node_bounds(c[w], c32v, sv, p, bs, l, u);
        if (p.cert && active[w]) {
            l = fmax(l, lb[w]);
            u = fmin(u, ub[w]);
        }
        if (err) {
            // the width of the rounding interval around each bound (zero in
            // FP64 mode): the exact partial sum lies in [c lo, c hi] and the
            // exact level value in [s los, s his], so l and u each lie within
            // this of the bound of Theorem 1 evaluated exactly at r (alpha
            // gamma >= alpha, so the upper tail's term covers the lower's)
            err[v] = p.cert ? c[w] * (bs.hi64 - bs.lo64) + c32v * (bs.hi32 - bs.lo32) +
                                  p.ag_hi * sv * (ctrl->his - ctrl->los)
                            : 0.0;
        }
        if (lower) lower[v] = l;
        if (upper) upper[v] = u;
    }
}

template <typename T>
__global__ void walk_out_kernel(const T* walk, const int32_t* __restrict__ inv, const Ctrl* ctrl, IterParams p,
                                int level, double* out) {
    const int f32_from = ctrl->f32_from;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += stride)
        out[v] = walk_value(walk, p, f32_from, level, inv[v]);
}


__global__ void narrow_kernel(const int64_t* __restrict__ in, int32_t* __restrict__ out, int64_t count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride) out[q] = (int32_t)in[q];
}

inline int grid_for(int64_t n, int threads, int max_blocks = 152 * 8) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

}  // namespace

// ---- launchers --------------------------------------------------------------

cudaError_t launch_narrow_rowptr(const int64_t* in, int32_t* out, int64_t count, cudaStream_t st) {
    narrow_kernel<<<grid_for(count, 256), 256, 0, st>>>(in, out, count);
    return cudaGetLastError();
}

cudaError_t launch_validate_csr(const DeviceGraph& g, unsigned long long* d_bad, int64_t* d_degmax,
                                cudaStream_t st) {
    const int blocks = grid_for(g.n > g.nnz ? g.n : g.nnz, 256);
    if (g.off64)
        validate_kernel<int64_t><<<blocks, 256, 0, st>>>((const int64_t*)g.rowptr, g.col, g.n, g.nnz, d_bad, d_degmax);
    else
        validate_kernel<int32_t><<<blocks, 256, 0, st>>>((const int32_t*)g.rowptr, g.col, g.n, g.nnz, d_bad, d_degmax);
    return cudaGetLastError();
}

cudaError_t launch_init_walk(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, bool fp32,
                             cudaStream_t st) {
    (void)g;
    (void)fp32;
    init_walk_kernel<double><<<grid_for(p.n, 256), 256, 0, st>>>((double*)b.walk, b.c, b.c32, b.lb, b.ub, b.active, p);
    return cudaGetLastError();
}

cudaError_t launch_cert_init(const IterBuffers& b, const IterParams& p, cudaStream_t st) {
    cert_init_kernel<<<1, 1, 0, st>>>(b.ctrl, p);
    return cudaGetLastError();
}

cudaError_t launch_cert_replay(const IterBuffers& b, const IterParams& p, int r, cudaStream_t st) {
    cert_replay_kernel<<<1, 1, 0, st>>>(b.ctrl, p, r);
    return cudaGetLastError();
}

cudaError_t launch_theta0(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, uint32_t* d_deghist,
                          int64_t top, cudaStream_t st) {
    cudaError_t err = cudaMemsetAsync(d_deghist, 0, (size_t)(top + 1) * sizeof(uint32_t), st);
    if (err != cudaSuccess) return err;
    const int blocks = grid_for(g.n, 256);
    if (g.off64)
        deg_hist_kernel<int64_t><<<blocks, 256, 0, st>>>((const int64_t*)g.rowptr, g.n, top, d_deghist);
    else
        deg_hist_kernel<int32_t><<<blocks, 256, 0, st>>>((const int32_t*)g.rowptr, g.n, top, d_deghist);
    kth_degree_kernel<double><<<1, SELECT_THREADS, 0, st>>>(d_deghist, top, p, b.ctrl);
    return cudaGetLastError();
}

cudaError_t launch_theta0_class(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int64_t a,
                                int64_t bend, int64_t lo, int bits, int64_t kk, cudaStream_t st) {
    if (g.off64)
        kth_degree_class_kernel<int64_t, double><<<1, SELECT_THREADS, 0, st>>>((const int64_t*)g.rowptr, a, bend, lo,
                                                                               bits, kk, p, b.ctrl);
    else
        kth_degree_class_kernel<int32_t, double><<<1, SELECT_THREADS, 0, st>>>((const int32_t*)g.rowptr, a, bend, lo,
                                                                               bits, kk, p, b.ctrl);
    return cudaGetLastError();
}

cudaError_t prepare_kernels() {
    const int smem = SELECT_CAP * (int)sizeof(SelEntry);
    return cudaFuncSetAttribute(select_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_select(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, const double* cl,
                          const double* cu, const int32_t* cid, bool fp32, cudaStream_t st) {
    (void)fp32;
    const int smem = SELECT_CAP * (int)sizeof(SelEntry);
    select_kernel<double><<<1, SELECT_THREADS, smem, st>>>(cl, cu, cid, (const double*)b.walk, b.c, b.c32, b.lb, g.inv,
                                                           b.topk_id, b.topk_l, b.topk_u, b.ctrl, p);
    return cudaGetLastError();
}

cudaError_t launch_count(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, bool fp32,
                         cudaStream_t st) {
    (void)fp32;
    // a fixed grid (the launch may sit in a captured graph); the blocks stride
    // over tiles of the list, or of V for the first count
    count_kernel<double><<<grid_for(p.n, COUNT_TILE, 152 * 4), COUNT_THREADS, 0, st>>>(
        (const double*)b.walk, b.c, b.c32, b.lb, b.ub, g.perm, b.active, b.alist[0], b.alist[1], b.ctrl, p);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const IterBuffers& b, const IterParams& p, cudaStream_t st) {
    finalize_kernel<<<1, 256, 0, st>>>(b.topk_l, b.topk_u, b.trace, b.ctrl, p, b.cond_handle, b.use_cond);
    return cudaGetLastError();
}

cudaError_t launch_bounds_out(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int level, bool fp32,
                              double* lower, double* upper, double* err, cudaStream_t st) {
    (void)fp32;
    bounds_out_kernel<double><<<grid_for(p.n, 256), 256, 0, st>>>((const double*)b.walk, b.c, b.c32, b.lb, b.ub,
                                                                 b.active, g.inv, b.ctrl, p, level, lower, upper, err);
    return cudaGetLastError();
}

cudaError_t launch_walk_out(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int level, bool fp32,
                            double* out, cudaStream_t st) {
    (void)fp32;
    walk_out_kernel<double><<<grid_for(p.n, 256), 256, 0, st>>>((const double*)b.walk, g.inv, b.ctrl, p, level, out);
    return cudaGetLastError();
}


}  // namespace katz
