// The walk-count SpMV of Algorithm 1, fused with the bound update:
//
//   s_r(u) = alpha * sum_{u->x} s_{r-1}(x)        (Eq. 4, scaled by alpha^r)
//   c_r(u) = c_{r-1}(u) + s_r(u)
//   l_r, u_r from c_r and s_r for u in M; u joins the candidate list when
//   l_r(u) >= theta_{r-1}.
//
// The graph is stored in internal order (katz_relabel.cu): rows grouped by
// degree class, largest first.  Rows are processed in four row modes chosen by
// degree, so the lanes that share a row (or the rows that share a warp) carry
// equal work, and no lane waits on a merge search or a block barrier:
//   THREAD  deg <= 16         one thread per row
//   OCTET   16 < deg <= 128   eight lanes per row
//   WARP    128 < deg <= 2048 one warp per row
//   CHUNK   deg > 2048        one warp per 2048-arc chunk; spmv_chunk_fixup adds
//                             a row's chunk sums in chunk order and finishes it
// The walk vector is gathered with read-only loads (one L2 request per arc:
// this access, not HBM bandwidth, bounds the kernel on power-law graphs).
// Every row sum is accumulated in a fixed order, so results are reproducible.
#include <stdint.h>

#include "katz_common.cuh"

namespace katz {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int BLOCK = 256;
constexpr int WARPS = BLOCK / 32;

struct Epi {
    double* y;
    double* c;
    uint8_t* active;
    const int32_t* perm;
    double* cand_l;
    double* cand_u;
    int32_t* cand_id;
    int64_t cand_cap;
    Ctrl* ctrl;
    double theta_prev;
};

// Finish row u: s_r(u) = alpha * sum, c_r = c_{r-1} + s_r, bounds, candidate
// (candidates carry the original id).
__device__ __forceinline__ void finish_row(int64_t u, double sum, const Epi& e, const IterParams& p) {
    const double s = __dmul_rn(p.alpha, sum);
    e.y[u] = s;
    const double cn = __dadd_rn(e.c[u], s);
    e.c[u] = cn;
    if (e.active[u]) {
        double l, up;
        node_bounds(cn, s, p, l, up);
        if (l >= e.theta_prev) {
            const unsigned long long pos = atomicAdd(&e.ctrl->n_cand, 1ULL);
            if (pos < (unsigned long long)e.cand_cap) {
                e.cand_l[pos] = l;
                e.cand_u[pos] = up;
                e.cand_id[pos] = e.perm[u];
            }
        }
    }
}

// sum of x[col[j]] for j in [a, b) with stride `step` starting at a + first,
// eight independent loads in flight, added in index order
__device__ __forceinline__ double strided_sum(const int32_t* __restrict__ col, const double* __restrict__ x,
                                              int64_t a, int64_t b, int first, int step) {
    double s = 0.0;
    for (int64_t j = a + first; j < b; j += 8 * (int64_t)step) {
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t jj = j + (int64_t)q * step;
            v[q] = jj < b ? __ldg(x + col[jj]) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) s = __dadd_rn(s, v[q]);
    }
    return s;
}

template <typename Off>
__global__ void __launch_bounds__(BLOCK)
spmv_rows_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col, SpmvLayout L, double* walk,
                 double* c, uint8_t* active, const int32_t* __restrict__ perm, const int32_t* __restrict__ chunk_row,
                 const int64_t* __restrict__ chunk_first, double* chunk_part, double* cand_l, double* cand_u,
                 int32_t* cand_id, int64_t cand_cap, Ctrl* ctrl, IterParams p) {
    if (ctrl->stop) return;
    const int r_cur = ctrl->r + 1;
    const double* __restrict__ x = walk_slot(walk, p, r_cur - 1);
    double* y = walk_slot(walk, p, r_cur);
    const Epi ep{y, c, active, perm, cand_l, cand_u, cand_id, cand_cap, ctrl, ctrl->theta_prev};
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t b = blockIdx.x;

    if (b >= L.blk_thread) {  // THREAD rows
        const int64_t u = L.row_thread + (b - L.blk_thread) * BLOCK + tid;
        if (u < L.n) finish_row(u, strided_sum(col, x, rowptr[u], rowptr[u + 1], 0, 1), ep, p);
    } else if (b >= L.blk_octet) {  // OCTET rows
        const int64_t u = L.row_octet + (b - L.blk_octet) * (BLOCK / 8) + (tid >> 3);
        const int sub = tid & 7;
        double s = 0.0;
        if (u < L.row_thread) s = strided_sum(col, x, rowptr[u], rowptr[u + 1], sub, 8);
#pragma unroll
        for (int off = 4; off; off >>= 1) s = __dadd_rn(s, __shfl_down_sync(FULL, s, off, 8));
        if (sub == 0 && u < L.row_thread) finish_row(u, s, ep, p);
    } else if (b >= L.blk_warp) {  // WARP rows
        const int64_t u = L.row_warp + (b - L.blk_warp) * WARPS + wid;
        double s = 0.0;
        if (u < L.row_octet) s = strided_sum(col, x, rowptr[u], rowptr[u + 1], lane, 32);
#pragma unroll
        for (int off = 16; off; off >>= 1) s = __dadd_rn(s, __shfl_down_sync(FULL, s, off));
        if (lane == 0 && u < L.row_octet) finish_row(u, s, ep, p);
    } else {  // CHUNK rows: one warp per chunk of CHUNK_ARCS arcs
        const int64_t ch = b * WARPS + wid;
        double s = 0.0;
        if (ch < L.chunks) {
            const int64_t u = chunk_row[ch];
            const int64_t j0 = (int64_t)rowptr[u] + (ch - chunk_first[u]) * (int64_t)CHUNK_ARCS;
            const int64_t j1 = min(j0 + (int64_t)CHUNK_ARCS, (int64_t)rowptr[u + 1]);
            s = strided_sum(col, x, j0, j1, lane, 32);
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) s = __dadd_rn(s, __shfl_down_sync(FULL, s, off));
        if (lane == 0 && ch < L.chunks) chunk_part[ch] = s;
    }
}

// CHUNK rows: add the chunk sums of each row in chunk order, then finish it.
__global__ void spmv_chunk_fixup(SpmvLayout L, double* walk, double* c, uint8_t* active,
                                 const int32_t* __restrict__ perm, const int64_t* __restrict__ chunk_first,
                                 const double* __restrict__ chunk_part, double* cand_l, double* cand_u,
                                 int32_t* cand_id, int64_t cand_cap, Ctrl* ctrl, IterParams p) {
    if (ctrl->stop) return;
    const int r_cur = ctrl->r + 1;
    double* y = walk_slot(walk, p, r_cur);
    const Epi ep{y, c, active, perm, cand_l, cand_u, cand_id, cand_cap, ctrl, ctrl->theta_prev};
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= L.row_warp) return;
    double s = 0.0;
    for (int64_t ch = chunk_first[u]; ch < chunk_first[u + 1]; ++ch) s = __dadd_rn(s, chunk_part[ch]);
    finish_row(u, s, ep, p);
}

}  // namespace

cudaError_t launch_spmv(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, bool fp32,
                        cudaStream_t st) {
    if (fp32) return cudaErrorNotSupported;
    const SpmvLayout& L = g.layout;
    if (L.blocks_total > 0) {
        if (g.off64)
            spmv_rows_kernel<int64_t><<<(unsigned)L.blocks_total, BLOCK, 0, st>>>(
                (const int64_t*)g.rowptr, g.col, L, (double*)b.walk, b.c, b.active, g.perm, g.chunk_row,
                g.chunk_first, g.chunk_part, b.cand_l, b.cand_u, b.cand_id, b.cand_cap, b.ctrl, p);
        else
            spmv_rows_kernel<int32_t><<<(unsigned)L.blocks_total, BLOCK, 0, st>>>(
                (const int32_t*)g.rowptr, g.col, L, (double*)b.walk, b.c, b.active, g.perm, g.chunk_row,
                g.chunk_first, g.chunk_part, b.cand_l, b.cand_u, b.cand_id, b.cand_cap, b.ctrl, p);
    }
    if (L.row_warp > 0)
        spmv_chunk_fixup<<<(unsigned)((L.row_warp + 127) / 128), 128, 0, st>>>(
            L, (double*)b.walk, b.c, b.active, g.perm, g.chunk_first, g.chunk_part, b.cand_l, b.cand_u, b.cand_id,
            b.cand_cap, b.ctrl, p);
    return cudaGetLastError();
}

// Block ranges of the four row modes from the internal row boundaries.
SpmvLayout make_layout(int64_t n, int64_t row_warp, int64_t row_octet, int64_t row_thread, int64_t chunks) {
    SpmvLayout L{};
    L.n = n;
    L.row_warp = row_warp;
    L.row_octet = row_octet;
    L.row_thread = row_thread;
    L.chunks = chunks;
    const int64_t bc = (chunks + WARPS - 1) / WARPS;
    const int64_t bw = (row_octet - row_warp + WARPS - 1) / WARPS;
    const int64_t bo = (row_thread - row_octet + BLOCK / 8 - 1) / (BLOCK / 8);
    const int64_t bt = (n - row_thread + BLOCK - 1) / BLOCK;
    L.blk_warp = bc;
    L.blk_octet = bc + bw;
    L.blk_thread = bc + bw + bo;
    L.blocks_total = bc + bw + bo + bt;
    return L;
}

}  // namespace katz
