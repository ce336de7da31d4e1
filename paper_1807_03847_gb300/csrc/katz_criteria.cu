// The other stopping criteria of Sec. 3.1, checked after each iteration of
// the walk recurrence (the SpMV of katz_spmv.cu, all nodes kept active):
//   ranking criterion  all nodes eps-separated (Eq. 3) from each other: the
//                      top-k criterion with k = n.  The nodes are sorted by
//                      (l desc, original id asc) and every adjacent pair is
//                      checked; by transitivity adjacent pairs suffice.
//   score criterion    u_r(v) - l_r(v) < eps for every node.
//   pair criterion     two given nodes eps-separated.
// The sort is a stable least-significant-digit radix sort over the 96-bit key
// (complemented bits of l, which order like l reversed because l >= 0, then
// the original id): twelve passes of 8-bit digits, each a per-tile
// histogram, an exclusive scan of the counts in digit-major order, and a
// stable scatter.
#include <stdint.h>

#include "katz_common.cuh"

namespace katz {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;  // elements per block
constexpr int RS_PASSES = 12;                     // 4 over the id, 8 over the key

__device__ __forceinline__ int digit(const uint64_t* hi, const uint32_t* lo, int64_t i, int pass) {
    return pass < 4 ? (int)((lo[i] >> (8 * pass)) & 255u) : (int)((hi[i] >> (8 * (pass - 4))) & 255ull);
}

// key of internal node v: ~bits(l) (ascending = l descending), original id
__global__ void rs_keys_kernel(const double* __restrict__ lb, const int32_t* __restrict__ perm, int64_t n,
                               uint64_t* hi, uint32_t* lo, int32_t* val) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        hi[v] = ~(uint64_t)__double_as_longlong(lb[v]);
        lo[v] = (uint32_t)perm[v];
        val[v] = (int32_t)v;
    }
}

// counts[d * blocks + b] = elements of tile b with digit d
__global__ void __launch_bounds__(RS_THREADS)
rs_hist_kernel(const uint64_t* __restrict__ hi, const uint32_t* __restrict__ lo, int64_t n, int pass,
               int64_t* counts, int64_t blocks) {
    __shared__ unsigned int h[256];
    const int tid = threadIdx.x;
    h[tid] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int q = 0; q < RS_ROUNDS; ++q) {
        const int64_t i = base + q * RS_THREADS + tid;
        if (i < n) atomicAdd(&h[digit(hi, lo, i, pass)], 1u);
    }
    __syncthreads();
    counts[(int64_t)tid * blocks + blockIdx.x] = h[tid];
}

// stable scatter: tile b's elements with digit d go, in their order, to
// offs[d * blocks + b] onwards.  The tile is first ordered by digit in shared
// memory (its digit counts come from the histogram pass), then written out in
// that order, so that consecutive threads write consecutive slots of one
// digit's run instead of one slot each in up to 256 runs.
__global__ void __launch_bounds__(RS_THREADS)
rs_scatter_kernel(const uint64_t* __restrict__ hi, const uint32_t* __restrict__ lo, const int32_t* __restrict__ val,
                  int64_t n, int pass, const int64_t* __restrict__ counts, const int64_t* __restrict__ offs,
                  int64_t blocks, uint64_t* __restrict__ hi2, uint32_t* __restrict__ lo2, int32_t* __restrict__ val2) {
    __shared__ uint64_t s_hi[RS_TILE];
    __shared__ uint32_t s_lo[RS_TILE];
    __shared__ int32_t s_val[RS_TILE];
    __shared__ uint8_t s_d[RS_TILE];
    __shared__ long long gbase[256];
    __shared__ int lstart[256], run[256];
    __shared__ int wc[RS_WARPS][256];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t tile = (int64_t)blockIdx.x * RS_TILE;
    const int in_tile = (int)min((int64_t)RS_TILE, n - tile);
    // exclusive scan of the tile's digit counts: each digit's first local slot
    int c = (int)counts[(int64_t)tid * blocks + blockIdx.x];
    int incl = c;
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) wc[0][wid] = incl;
    gbase[tid] = offs[(int64_t)tid * blocks + blockIdx.x];
    __syncthreads();
    int wsum = 0;
    for (int w = 0; w < wid; ++w) wsum += wc[0][w];
    lstart[tid] = wsum + incl - c;
    run[tid] = wsum + incl - c;
    __syncthreads();
    for (int q = 0; q < RS_ROUNDS; ++q) {
        for (int w = 0; w < RS_WARPS; ++w) wc[w][tid] = 0;
        __syncthreads();
        const int li = q * RS_THREADS + tid;
        const bool valid = li < in_tile;
        const int d = valid ? digit(hi, lo, tile + li, pass) : 256;
        const unsigned peers = __match_any_sync(FULL, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && lane == __ffs(peers) - 1) wc[wid][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pos = run[d] + rank;
            for (int w = 0; w < wid; ++w) pos += wc[w][d];
            s_hi[pos] = hi[tile + li];
            s_lo[pos] = lo[tile + li];
            s_val[pos] = val[tile + li];
            s_d[pos] = (uint8_t)d;
        }
        __syncthreads();
        int add = 0;
        for (int w = 0; w < RS_WARPS; ++w) add += wc[w][tid];
        run[tid] += add;
        __syncthreads();
    }
    for (int j = tid; j < in_tile; j += RS_THREADS) {
        const int d = s_d[j];
        const long long pos = gbase[d] + (j - lstart[d]);
        hi2[pos] = s_hi[j];
        lo2[pos] = s_lo[j];
        val2[pos] = s_val[j];
    }
}

// block total of a count, one atomic per block
__device__ __forceinline__ void add_block_count(unsigned long long c, unsigned long long* out) {
    __shared__ unsigned long long part[32];
    for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) part[wid] = c;
    __syncthreads();
    if (wid == 0) {
        c = lane < nw ? part[lane] : 0ull;
        for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
        if (lane == 0 && c) atomicAdd(out, c);
    }
}

// ranking criterion on the sorted order: u(M[i]) - eps < l(M[i-1]) for all
// i >= 1; the order leaves the library in original ids
__global__ void rank_check_kernel(const int32_t* __restrict__ order, const double* __restrict__ lb,
                                  const double* __restrict__ ub, const int32_t* __restrict__ perm, int64_t n,
                                  double eps, int32_t* rank_ids, Ctrl* ctrl) {
    if (ctrl->stop) return;
    unsigned long long bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t v = order[i];
        rank_ids[i] = perm[v];
        if (i > 0 && __dsub_rn(ub[v], eps) >= lb[order[i - 1]]) ++bad;
    }
    add_block_count(bad, &ctrl->cnt_cross);
}

// score criterion: every node's bounds closer than eps
__global__ void score_check_kernel(const double* __restrict__ lb, const double* __restrict__ ub, int64_t n,
                                   double eps, Ctrl* ctrl) {
    if (ctrl->stop) return;
    unsigned long long bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (!(__dsub_rn(ub[v], lb[v]) < eps)) ++bad;
    add_block_count(bad, &ctrl->cnt_cross);
}

// pair criterion: nodes oa, ob (original ids) eps-separated; the one with
// the larger l (ties: smaller id) first
__global__ void pair_check_kernel(const double* __restrict__ lb, const double* __restrict__ ub,
                                  const int32_t* __restrict__ inv, int32_t oa, int32_t ob, double eps,
                                  int32_t* topk_id, Ctrl* ctrl) {
    if (ctrl->stop) return;
    const int32_t ia = inv[oa], ib = inv[ob];
    const double la = lb[ia], lbv = lb[ib];
    const bool a_first = la > lbv || (la == lbv && oa < ob);
    const int32_t w = a_first ? ia : ib, v = a_first ? ib : ia;
    if (!(__dsub_rn(ub[v], eps) < lb[w])) ctrl->cnt_cross = 1;
    topk_id[0] = a_first ? oa : ob;
    topk_id[1] = a_first ? ob : oa;
}

__global__ void crit_init_kernel(Ctrl* ctrl) {
    ctrl->theta_prev = 1.0 / 0.0;  // no candidate lists: every node stays active
}

__global__ void finalize_crit_kernel(int64_t* trace, Ctrl* ctrl, IterParams p) {
    if (ctrl->stop) return;
    const int r_cur = ctrl->r + 1;
    if (r_cur <= p.r_max) trace[r_cur] = p.n;
    const int conv = ctrl->cnt_cross == 0;
    ctrl->r = r_cur;
    ctrl->converged = conv;
    ctrl->cnt_cross = 0;
    ctrl->n_cand = 0;
    ctrl->stop = conv || r_cur >= p.r_max;
}

int grid_for(int64_t n, int threads, int max_blocks = 152 * 16) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

}  // namespace

int64_t radix_tiles(int64_t n) { return (n + RS_TILE - 1) / RS_TILE; }

cudaError_t launch_crit_init(const IterBuffers& b, cudaStream_t st) {
    crit_init_kernel<<<1, 1, 0, st>>>(b.ctrl);
    return cudaGetLastError();
}

cudaError_t launch_score_check(const IterBuffers& b, const IterParams& p, cudaStream_t st) {
    score_check_kernel<<<grid_for(p.n, 256), 256, 0, st>>>(b.lb, b.ub, p.n, p.eps, b.ctrl);
    return cudaGetLastError();
}

cudaError_t launch_pair_check(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int32_t oa, int32_t ob,
                              cudaStream_t st) {
    pair_check_kernel<<<1, 1, 0, st>>>(b.lb, b.ub, g.inv, oa, ob, p.eps, b.topk_id, b.ctrl);
    return cudaGetLastError();
}

// Sort all nodes by (l desc, original id asc) and check the ranking criterion.
// rs: two buffers of each of hi (u64), lo (u32), val (i32), n entries; counts
// and offs: 256 * radix_tiles(n) entries; sums: scan scratch.
cudaError_t launch_ranking_check(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, RadixBuffers& rs,
                                 int32_t* rank_ids, cudaStream_t st) {
    const int64_t n = p.n, tiles = radix_tiles(n);
    rs_keys_kernel<<<grid_for(n, 256), 256, 0, st>>>(b.lb, g.perm, n, rs.hi[0], rs.lo[0], rs.val[0]);
    int cur = 0;
    for (int pass = 0; pass < RS_PASSES; ++pass) {
        rs_hist_kernel<<<(unsigned)tiles, RS_THREADS, 0, st>>>(rs.hi[cur], rs.lo[cur], n, pass, rs.counts, tiles);
        cudaError_t e = exclusive_scan_i64(rs.counts, 256 * tiles, rs.offs, rs.sums, st);
        if (e != cudaSuccess) return e;
        rs_scatter_kernel<<<(unsigned)tiles, RS_THREADS, 0, st>>>(rs.hi[cur], rs.lo[cur], rs.val[cur], n, pass,
                                                                  rs.counts, rs.offs, tiles, rs.hi[1 - cur], rs.lo[1 - cur],
                                                                  rs.val[1 - cur]);
        cur = 1 - cur;
    }
    rank_check_kernel<<<grid_for(n, 256), 256, 0, st>>>(rs.val[cur], b.lb, b.ub, g.perm, n, p.eps, rank_ids, b.ctrl);
    return cudaGetLastError();
}

// Stable LSD passes first..last (8-bit digits; 0-3 over lo, 4-11 over hi) of
// the (hi, lo, val) triples in rs buffer `cur`, n of them; cur ends on the
// buffer that holds the result.
cudaError_t radix_sort_passes(RadixBuffers& rs, int64_t n, int first, int last, int& cur, cudaStream_t st) {
    const int64_t tiles = radix_tiles(n);
    for (int pass = first; pass <= last; ++pass) {
        rs_hist_kernel<<<(unsigned)tiles, RS_THREADS, 0, st>>>(rs.hi[cur], rs.lo[cur], n, pass, rs.counts, tiles);
        cudaError_t e = exclusive_scan_i64(rs.counts, 256 * tiles, rs.offs, rs.sums, st);
        if (e != cudaSuccess) return e;
        rs_scatter_kernel<<<(unsigned)tiles, RS_THREADS, 0, st>>>(rs.hi[cur], rs.lo[cur], rs.val[cur], n, pass,
                                                                  rs.counts, rs.offs, tiles, rs.hi[1 - cur], rs.lo[1 - cur],
                                                                  rs.val[1 - cur]);
        cur = 1 - cur;
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize_crit(const IterBuffers& b, const IterParams& p, cudaStream_t st) {
    finalize_crit_kernel<<<1, 1, 0, st>>>(b.trace, b.ctrl, p);
    return cudaGetLastError();
}

}  // namespace katz
