// Degree-class relabelling of the graph at create time.
//
// Internal vertex order: vertices grouped by degree class (class 0 = degree
// 0, class k >= 1 = degree in (2^(k-2), 2^(k-1)], i.e. ceil(log2 deg) + 1),
// classes in decreasing order, original id order inside a class (a stable
// counting sort).  perm[u] = original id of internal vertex u; inv = perm^-1.
// In this order the rows a thread, a lane group or a warp processes together
// have degrees within a factor of two, the hub rows come first, and the
// walk-vector entries gathered most often sit together at the front.
//
// Only the walk-count SpMV sees internal ids; every result (ranking, bounds,
// walk vectors) leaves the library in original ids, and every tie between
// equal lower bounds is broken by the original id.
#include <stdint.h>

#include "katz_common.cuh"

namespace katz {

namespace {

constexpr int RL_THREADS = 1024;   // ids per block of the counting sort
constexpr int SCAN_THREADS = 1024;

__device__ __forceinline__ int degree_class(int64_t d) {
    if (d <= 0) return 0;
    return (d == 1) ? 1 : 65 - __clzll((unsigned long long)(d - 1)) + 0;  // ceil(log2 d) + 1
}

// counts[(NUM_CLASSES - 1 - c) * nb + b] = vertices of class c in block b:
// the classes from the highest down, so that one exclusive scan of the array
// gives every (class, block) its first slot
template <typename Off>
__global__ void class_hist_kernel(const Off* __restrict__ rowptr, int64_t n, int nb, int64_t* counts) {
    __shared__ uint32_t h[NUM_CLASSES];
    const int tid = threadIdx.x;
    if (tid < NUM_CLASSES) h[tid] = 0;
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * RL_THREADS + tid;
    if (v < n) atomicAdd(&h[degree_class((int64_t)rowptr[v + 1] - (int64_t)rowptr[v])], 1u);
    __syncthreads();
    if (tid < NUM_CLASSES) counts[(size_t)(NUM_CLASSES - 1 - tid) * nb + blockIdx.x] = h[tid];
}

__global__ void class_start_kernel(const int64_t* __restrict__ offs, int nb, uint64_t* class_start) {
    const int c = threadIdx.x;
    if (c < NUM_CLASSES) class_start[c] = (uint64_t)offs[(size_t)(NUM_CLASSES - 1 - c) * nb];
}

// stable scatter: within a block, vertices of the same class keep id order
template <typename Off>
__global__ void class_scatter_kernel(const Off* __restrict__ rowptr, int64_t n, int nb, const int64_t* offs,
                                     int32_t* perm, int32_t* inv) {
    __shared__ uint32_t base[NUM_CLASSES];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid < NUM_CLASSES) base[tid] = (uint32_t)offs[(size_t)(NUM_CLASSES - 1 - tid) * nb + blockIdx.x];
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * RL_THREADS + tid;
    const int cls = v < n ? degree_class((int64_t)rowptr[v + 1] - (int64_t)rowptr[v]) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, cls);
    const int rank_in_warp = __popc(peers & ((1u << lane) - 1u));
    // warps take their turn in id order so that ranks are stable across warps
    for (int w = 0; w < RL_THREADS / 32; ++w) {
        if (wid == w && v < n) {
            const uint32_t u = base[cls] + rank_in_warp;
            perm[u] = (int32_t)v;
            inv[v] = (int32_t)u;
        }
        __syncthreads();
        if (wid == w && v < n && lane == 31 - __clz(peers)) base[cls] += __popc(peers);
        __syncthreads();
    }
}

// exclusive scan of int64 values in three passes (block sums, scan of the
// sums in one block, block scans with offsets); out may alias nothing
__global__ void scan_block_sums(const int64_t* __restrict__ in, int64_t n, int64_t* sums) {
    __shared__ long long red[SCAN_THREADS / 32];
    const int64_t i = (int64_t)blockIdx.x * SCAN_THREADS + threadIdx.x;
    long long x = i < n ? in[i] : 0;
    for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += red[w];
        sums[blockIdx.x] = t;
    }
}

__global__ void scan_sums_inplace(int64_t* sums, int64_t nb) {
    __shared__ long long part[SCAN_THREADS];
    const int tid = threadIdx.x;
    const int64_t chunk = (nb + SCAN_THREADS - 1) / SCAN_THREADS;
    long long s = 0;
    for (int64_t e = tid * chunk; e < min(nb, (int64_t)(tid + 1) * chunk); ++e) s += sums[e];
    part[tid] = s;
    __syncthreads();
    for (int off = 1; off < SCAN_THREADS; off <<= 1) {
        const long long a = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += a;
        __syncthreads();
    }
    long long run = tid ? part[tid - 1] : 0;
    for (int64_t e = tid * chunk; e < min(nb, (int64_t)(tid + 1) * chunk); ++e) {
        const long long x = sums[e];
        sums[e] = run;
        run += x;
    }
}

__global__ void scan_finish(const int64_t* __restrict__ in, int64_t n, const int64_t* __restrict__ offs,
                            int64_t* out) {
    __shared__ long long ws[SCAN_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t i = (int64_t)blockIdx.x * SCAN_THREADS + tid;
    const long long x = i < n ? in[i] : 0;
    long long v = x;
    for (int off = 1; off < 32; off <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += y;
    }
    if (lane == 31) ws[wid] = v;
    __syncthreads();
    if (tid == 0) {
        long long t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) {
            const long long y = ws[w];
            ws[w] = t;
            t += y;
        }
    }
    __syncthreads();
    if (i < n) out[i] = offs[blockIdx.x] + ws[wid] + v - x;
}

template <typename Off>
__global__ void new_degree_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ perm, int64_t n,
                                  int64_t* deg_new) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const int64_t v = perm[u];
        deg_new[u] = (int64_t)rowptr[v + 1] - (int64_t)rowptr[v];
    }
}

constexpr unsigned FULL_MASK = 0xffffffffu;

constexpr int REMAP_UNROLL = 4;  // arcs per lane in flight

// Arcs of the original rows [v0, v1), renamed, into their new rows inv[v].
// One warp per 32 consecutive rows.  The lanes scan the rows' lengths, then
// walk the group's arcs together, REMAP_UNROLL arcs per lane at a time: arc t
// of the group belongs to the first lane whose inclusive prefix exceeds t (a
// binary search over the lanes).  Rows that become CHUNK rows
// (inv[v] < row_warp) count as empty here and are left to
// remap_hub_chunks_kernel, so every other row holds at most 2048 arcs and a
// group at most 2^16.  A column entry outside [0, n) is counted in *bad and
// stored as 0 (the caller rejects the graph).
template <typename Off>
__global__ void remap_src_rows_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                                      const int32_t* __restrict__ inv, const int64_t* __restrict__ rowptr_new,
                                      int64_t v0, int64_t v1, int64_t n, int64_t row_warp,
                                      int32_t* __restrict__ col_new, unsigned long long* bad) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const int lane = threadIdx.x & 31;
    const int64_t groups = (v1 - v0 + 31) / 32;
    unsigned long long nb = 0;
    for (int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; gi < groups; gi += warps) {
        const int64_t v = v0 + gi * 32 + lane;
        int64_t a = 0, o = 0;
        int len = 0;
        if (v < v1) {
            const int64_t u = inv[v];
            if (u >= row_warp) {
                a = rowptr[v];
                len = (int)((int64_t)rowptr[v + 1] - a);
                o = rowptr_new[u];
            }
        }
        int pre = len;  // inclusive prefix over the lanes
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(FULL_MASK, pre, off);
            if (lane >= off) pre += y;
        }
        const int total = __shfl_sync(FULL_MASK, pre, 31);
        // arc t of this lane's row sits at src_base + t and goes to dst_base + t
        const int64_t src_base = a - (pre - len), dst_base = o - (pre - len);
        for (int t0 = 0; t0 < total; t0 += 32 * REMAP_UNROLL) {
            int32_t x[REMAP_UNROLL];
            int64_t dst[REMAP_UNROLL];
#pragma unroll
            for (int k = 0; k < REMAP_UNROLL; ++k) {
                const int t = t0 + k * 32 + lane;
                int q = 0;
#pragma unroll
                for (int s = 16; s; s >>= 1)
                    if (__shfl_sync(FULL_MASK, pre, q + s - 1) <= t) q += s;
                const int64_t sb = __shfl_sync(FULL_MASK, src_base, q), db = __shfl_sync(FULL_MASK, dst_base, q);
                x[k] = 0;
                dst[k] = -1;
                if (t < total) {
                    x[k] = col[sb + t];
                    dst[k] = db + t;
                }
            }
#pragma unroll
            for (int k = 0; k < REMAP_UNROLL; ++k) {
                if (dst[k] < 0) continue;
                int32_t xv = x[k];
                if (xv < 0 || (int64_t)xv >= n) {
                    ++nb;
                    xv = 0;
                }
                col_new[dst[k]] = inv[xv];
            }
        }
    }
    for (int off = 16; off; off >>= 1) nb += __shfl_xor_sync(FULL_MASK, nb, off);
    if (lane == 0 && nb) atomicAdd(bad, nb);
}

// CHUNK rows (new ids below row_warp) of the original rows [v0, v1): one warp
// per chunk of CHUNK_ARCS arcs (the chunk count is chunk_first[row_warp]),
// REMAP_UNROLL arcs per lane in flight
template <typename Off>
__global__ void remap_hub_chunks_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                                        const int32_t* __restrict__ perm, const int32_t* __restrict__ inv,
                                        const int64_t* __restrict__ rowptr_new, const int32_t* __restrict__ chunk_row,
                                        const int64_t* __restrict__ chunk_first, int64_t row_warp, int64_t v0,
                                        int64_t v1, int64_t n, int32_t* __restrict__ col_new,
                                        unsigned long long* bad) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const int lane = threadIdx.x & 31;
    const int64_t chunks = chunk_first[row_warp];
    unsigned long long nb = 0;
    for (int64_t ch = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; ch < chunks; ch += warps) {
        const int64_t u = chunk_row[ch];
        const int64_t v = perm[u];
        if (v < v0 || v >= v1) continue;
        const int64_t a = rowptr[v], b = rowptr[v + 1];
        const int64_t j0 = a + (ch - chunk_first[u]) * (int64_t)CHUNK_ARCS;
        const int64_t j1 = min(j0 + (int64_t)CHUNK_ARCS, b);
        const int64_t o = rowptr_new[u] + (j0 - a);
        for (int64_t jb = j0; jb < j1; jb += 32 * REMAP_UNROLL) {
            int32_t x[REMAP_UNROLL];
#pragma unroll
            for (int k = 0; k < REMAP_UNROLL; ++k) {
                const int64_t j = jb + k * 32 + lane;
                x[k] = j < j1 ? col[j] : 0;
            }
#pragma unroll
            for (int k = 0; k < REMAP_UNROLL; ++k) {
                const int64_t j = jb + k * 32 + lane;
                if (j >= j1) continue;
                int32_t xv = x[k];
                if (xv < 0 || (int64_t)xv >= n) {
                    ++nb;
                    xv = 0;
                }
                col_new[o + (j - j0)] = inv[xv];
            }
        }
    }
    for (int off = 16; off; off >>= 1) nb += __shfl_xor_sync(FULL_MASK, nb, off);
    if (lane == 0 && nb) atomicAdd(bad, nb);
}

// chunks of each CHUNK row (u < row_warp) from its new degree; cnt[row_warp] = 0;
// *max_chunks = the largest count
__global__ void chunk_count_kernel(const int64_t* __restrict__ rowptr_new, int64_t row_warp, int64_t* cnt,
                                   unsigned long long* max_chunks) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long mx = 0;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= row_warp; u += stride) {
        const int64_t c = u < row_warp ? (rowptr_new[u + 1] - rowptr_new[u] + CHUNK_ARCS - 1) / CHUNK_ARCS : 0;
        cnt[u] = c;
        mx = max(mx, (unsigned long long)c);
    }
    for (int off = 16; off; off >>= 1) mx = max(mx, __shfl_xor_sync(FULL_MASK, mx, off));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(max_chunks, mx);
}

// chunk_row[q] = u for the chunks q of row u (one warp per row)
__global__ void chunk_fill_kernel(const int64_t* __restrict__ chunk_first, int64_t row_warp, int32_t* chunk_row) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const int lane = threadIdx.x & 31;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; u < row_warp; u += warps)
        for (int64_t q = chunk_first[u] + lane; q < chunk_first[u + 1]; q += 32) chunk_row[q] = (int32_t)u;
}

// ---- reverse graphs ----------------------------------------------------------
// in-degree of every node (cnt zero on entry)
__global__ void indegree_kernel(const int32_t* __restrict__ col, int64_t nnz, unsigned long long* cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz; j += stride)
        atomicAdd(&cnt[col[j]], 1ull);
}

// arc v -> x of the input becomes x -> v: one warp per row; cursor[x] starts
// at the first slot of row x of the reverse graph
__global__ void reverse_fill_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t n,
                                    unsigned long long* cursor, int32_t* col_rev) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; v < n; v += warps)
        for (int64_t j = rowptr[v] + lane; j < rowptr[v + 1]; j += 32)
            col_rev[atomicAdd(&cursor[col[j]], 1ull)] = (int32_t)v;
}

int grid_for(int64_t n, int threads, int max_blocks = 152 * 16) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

}  // namespace

int degree_class_host(int64_t d) {
    if (d <= 0) return 0;
    int k = 0;
    while (((int64_t)1 << k) < d) ++k;  // ceil(log2 d)
    return k + 1;
}

int64_t relabel_scratch(int64_t n) {
    const int64_t cells = (int64_t)NUM_CLASSES * relabel_blocks(n);
    return 2 * cells + scan_blocks(cells);
}

cudaError_t relabel_by_degree_class(const int64_t* rowptr64, int64_t n, int64_t* scratch, int32_t* perm, int32_t* inv,
                                    uint64_t* class_start_dev, cudaStream_t st) {
    const int nb = relabel_blocks(n);
    const int64_t cells = (int64_t)NUM_CLASSES * nb;
    int64_t* counts = scratch;
    int64_t* offs = scratch + cells;
    class_hist_kernel<int64_t><<<nb, RL_THREADS, 0, st>>>(rowptr64, n, nb, counts);
    cudaError_t e = exclusive_scan_i64(counts, cells, offs, scratch + 2 * cells, st);
    if (e != cudaSuccess) return e;
    class_start_kernel<<<1, 64, 0, st>>>(offs, nb, class_start_dev);
    class_scatter_kernel<int64_t><<<nb, RL_THREADS, 0, st>>>(rowptr64, n, nb, offs, perm, inv);
    return cudaGetLastError();
}

namespace {

// Locality keys of the low-degree end (internal ids u >= start, rows of at
// most 16 arcs) of the graph in degree-class order (rowptr1/col1, internal
// ids), at index u - start.  The sort key is the row's degree class (in the
// class order) and its anchor, the smallest internal id among its neighbours
// (the neighbour whose row the SpMV reaches first; n if none): packed into
// lo as class_rank << abits | anchor when that fits 32 bits, else the anchor
// in lo and the class in the low byte of hi.  hi carries the row's degree
// (bits 8-12) and original id (bits 13-43), val its class-order id u.
__global__ void tail_keys_kernel(const int64_t* __restrict__ rowptr1, const int32_t* __restrict__ col1,
                                 const int32_t* __restrict__ perm, int64_t n, int64_t start, int abits,
                                 uint64_t* __restrict__ hi, uint32_t* __restrict__ lo, int32_t* __restrict__ val) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n - start; i += stride) {
        const int64_t a = rowptr1[start + i], b = rowptr1[start + i + 1];
        uint32_t m = (uint32_t)n;
        for (int64_t j = a; j < b; ++j) m = min(m, (uint32_t)col1[j]);
        const int cls = degree_class(b - a);  // 0..5
        hi[i] = (uint64_t)(NUM_CLASSES - 1 - cls) | (uint64_t)(b - a) << 8 | (uint64_t)(uint32_t)perm[start + i] << 13;
        lo[i] = abits > 0 ? (uint32_t)(5 - cls) << abits | m : m;
        val[i] = (int32_t)(start + i);
    }
}

// The row at sorted position i (class-order id u1 = sorted[i], degree and
// original id v in hi_sorted[i]) becomes start + i: sigma[u1 - start] =
// start + i, v goes to perm_tail[i] (copied into perm[start..] afterwards)
// and inv, the degree to deg[start + i]; the head rows' degrees and
// deg[n] = 0 complete deg
__global__ void tail_order_kernel(const int32_t* __restrict__ sorted, const uint64_t* __restrict__ hi_sorted,
                                  const int64_t* __restrict__ rowptr1, int64_t n, int64_t start,
                                  int32_t* __restrict__ sigma, int32_t* __restrict__ perm_tail,
                                  int32_t* __restrict__ inv, int64_t* __restrict__ deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t u = t0; u < start; u += stride) deg[u] = rowptr1[u + 1] - rowptr1[u];  // head rows keep theirs
    if (t0 == 0) deg[n] = 0;
    for (int64_t i = t0; i < n - start; i += stride) {
        const int32_t u1 = sorted[i];
        const uint64_t h = hi_sorted[i];
        const int32_t v = (int32_t)(h >> 13);
        sigma[u1 - start] = (int32_t)(start + i);
        perm_tail[i] = v;
        inv[v] = (int32_t)(start + i);
        deg[start + i] = (int64_t)((h >> 8) & 31u);
    }
}

// every arc target u >= start renamed to sigma[u - start]: in place in the
// head rows (arcs below rowptr1[start]), into tail_copy for the tail rows
__global__ void tail_rename_kernel(const int64_t* __restrict__ rowptr1, int64_t nnz, int64_t start,
                                   const int32_t* __restrict__ sigma, int32_t* __restrict__ col1,
                                   int32_t* __restrict__ tail_copy) {
    const int64_t head = rowptr1[start];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz; j += stride) {
        const int32_t x = col1[j];
        const int32_t y = x >= start ? sigma[x - start] : x;
        if (j >= head) tail_copy[j - head] = y;
        else if (y != x) col1[j] = y;
    }
}

// tail row start + i of the final order is class-order row sorted[i]
__global__ void tail_rows_kernel(const int32_t* __restrict__ sorted, const int64_t* __restrict__ rowptr1,
                                 const int64_t* __restrict__ rowptr_fin, int64_t n, int64_t start,
                                 const int32_t* __restrict__ tail_copy, int32_t* __restrict__ col) {
    const int64_t head = rowptr1[start];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n - start; i += stride) {
        const int32_t u1 = sorted[i];
        const int64_t a = rowptr1[u1] - head, len = rowptr1[u1 + 1] - rowptr1[u1];
        const int64_t o = rowptr_fin[start + i];
        for (int64_t k = 0; k < len; ++k) col[o + k] = tail_copy[a + k];
    }
}

}  // namespace

// Reorder the vertices from internal id `start` on (the rows of degree <= 16,
// already grouped by degree class) within their classes by anchor, ties kept
// in their current order (a stable sort): the walk values that one hub row
// gathers from low-degree rows then sit together, so a line fetched from DRAM
// serves several of its gathers.  Works on the graph already renamed into
// degree-class order (rowptr1, col1, perm, inv) and moves it to the new
// order: perm/inv updated, col1 rewritten in place, the new offsets in
// rowptr_fin (n + 1).  deg: n + 1 int64 of scratch; tail_copy: rowptr1[n] - rowptr1[start] entries; sums: scan
// scratch for n + 1; rs: radix buffers for n - start entries.
cudaError_t locality_order(int64_t n, int64_t nnz, int64_t start, const int64_t* rowptr1, int32_t* col1,
                           int32_t* perm, int32_t* inv, int64_t* deg, int64_t* rowptr_fin, int32_t* tail_copy,
                           int64_t* sums, RadixBuffers& rs, cudaStream_t st) {
    const int64_t m = n - start;
    if (m <= 1) return cudaSuccess;
    int abits = 1;  // bits of an anchor (<= n)
    while (abits < 31 && ((int64_t)1 << abits) <= n) ++abits;
    const bool packed = abits + 3 <= 32;  // class rank (0..5) above the anchor in lo
    tail_keys_kernel<<<grid_for(m, 256), 256, 0, st>>>(rowptr1, col1, perm, n, start, packed ? abits : 0, rs.hi[0],
                                                       rs.lo[0], rs.val[0]);
    int cur = 0;
    cudaError_t e = packed ? radix_sort_passes(rs, m, 0, (abits + 3 + 7) / 8 - 1, cur, st)
                           : radix_sort_passes(rs, m, 0, 4, cur, st);  // the anchor (4 digits), then the class
    if (e != cudaSuccess) return e;
    const int32_t* sorted = rs.val[cur];
    int32_t* sigma = (int32_t*)rs.lo[1 - cur];
    int32_t* perm_tail = rs.val[1 - cur];
    tail_order_kernel<<<grid_for(m, 256), 256, 0, st>>>(sorted, rs.hi[cur], rowptr1, n, start, sigma, perm_tail, inv,
                                                        deg);
    if ((e = cudaMemcpyAsync(perm + start, perm_tail, (size_t)m * sizeof(int32_t), cudaMemcpyDeviceToDevice, st)) !=
            cudaSuccess ||
        (e = exclusive_scan_i64(deg, n + 1, rowptr_fin, sums, st)) != cudaSuccess)
        return e;
    tail_rename_kernel<<<grid_for(nnz, 256, 152 * 32), 256, 0, st>>>(rowptr1, nnz, start, sigma, col1, tail_copy);
    tail_rows_kernel<<<grid_for(m, 256), 256, 0, st>>>(sorted, rowptr1, rowptr_fin, n, start, tail_copy, col1);
    return cudaGetLastError();
}

cudaError_t exclusive_scan_i64(const int64_t* in, int64_t n, int64_t* out, int64_t* sums_scratch,
                               cudaStream_t st) {
    const int64_t nb = (n + SCAN_THREADS - 1) / SCAN_THREADS;
    scan_block_sums<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, sums_scratch);
    scan_sums_inplace<<<1, SCAN_THREADS, 0, st>>>(sums_scratch, nb);
    scan_finish<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, sums_scratch, out);
    return cudaGetLastError();
}

cudaError_t relabel_offsets(const int64_t* rowptr64, const int32_t* perm, int64_t n, int64_t* deg_new_scratch,
                            int64_t* rowptr_new, int64_t* sums_scratch, cudaStream_t st) {
    new_degree_kernel<int64_t><<<grid_for(n, 256), 256, 0, st>>>(rowptr64, perm, n, deg_new_scratch);
    cudaError_t e = cudaMemsetAsync(deg_new_scratch + n, 0, sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
    return exclusive_scan_i64(deg_new_scratch, n + 1, rowptr_new, sums_scratch, st);
}

cudaError_t remap_src_rows(const int64_t* rowptr64, const int32_t* col, const int32_t* inv, const int64_t* rowptr_new,
                           int64_t v0, int64_t v1, int64_t n, int64_t row_warp, int32_t* col_new,
                           unsigned long long* bad, cudaStream_t st) {
    if (v1 <= v0) return cudaSuccess;
    remap_src_rows_kernel<int64_t><<<grid_for(v1 - v0, 256, 152 * 32), 256, 0, st>>>(
        rowptr64, col, inv, rowptr_new, v0, v1, n, row_warp, col_new, bad);
    return cudaGetLastError();
}

cudaError_t remap_hub_chunks(const int64_t* rowptr64, const int32_t* col, const int32_t* perm, const int32_t* inv,
                             const int64_t* rowptr_new, const int32_t* chunk_row, const int64_t* chunk_first,
                             int64_t row_warp, int64_t chunks_cap, int64_t v0, int64_t v1, int64_t n,
                             int32_t* col_new, unsigned long long* bad, cudaStream_t st) {
    if (row_warp <= 0) return cudaSuccess;
    remap_hub_chunks_kernel<int64_t><<<grid_for(chunks_cap * 32, 256, 152 * 32), 256, 0, st>>>(
        rowptr64, col, perm, inv, rowptr_new, chunk_row, chunk_first, row_warp, v0, v1, n, col_new, bad);
    return cudaGetLastError();
}

cudaError_t build_chunk_table(const int64_t* rowptr_new, int64_t row_warp, int64_t* cnt_scratch, int64_t* sums_scratch,
                              int64_t* chunk_first, int32_t* chunk_row, unsigned long long* max_chunks,
                              cudaStream_t st) {
    chunk_count_kernel<<<grid_for(row_warp + 1, 256), 256, 0, st>>>(rowptr_new, row_warp, cnt_scratch, max_chunks);
    cudaError_t e = exclusive_scan_i64(cnt_scratch, row_warp + 1, chunk_first, sums_scratch, st);
    if (e != cudaSuccess) return e;
    if (row_warp > 0) chunk_fill_kernel<<<grid_for(row_warp * 32, 256), 256, 0, st>>>(chunk_first, row_warp, chunk_row);
    return cudaGetLastError();
}

int64_t scan_blocks(int64_t n) { return (n + SCAN_THREADS - 1) / SCAN_THREADS; }

cudaError_t launch_indegree(const int32_t* col, int64_t nnz, int64_t* cnt, cudaStream_t st) {
    if (nnz > 0) indegree_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(col, nnz, (unsigned long long*)cnt);
    return cudaGetLastError();
}

cudaError_t reverse_csr(const int64_t* rowptr, const int32_t* col, int64_t n, int64_t nnz, int64_t* cnt,
                        int64_t* sums, int64_t* rowptr_rev, int32_t* col_rev, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)(n + 1) * sizeof(int64_t), st);
    if (e == cudaSuccess) e = launch_indegree(col, nnz, cnt, st);
    if (e == cudaSuccess) e = exclusive_scan_i64(cnt, n + 1, rowptr_rev, sums, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cnt, rowptr_rev, (size_t)n * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess || nnz == 0) return e;
    reverse_fill_kernel<<<grid_for(n * 32, 256), 256, 0, st>>>(rowptr, col, n, (unsigned long long*)cnt, col_rev);
    return cudaGetLastError();
}
int relabel_blocks(int64_t n) { return (int)((n + RL_THREADS - 1) / RL_THREADS); }

}  // namespace katz
