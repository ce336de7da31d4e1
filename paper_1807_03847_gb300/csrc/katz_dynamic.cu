// Dynamic graphs (Sec. 4, Algorithm 2): a batch of edge insertions and
// deletions is validated, applied to the device CSR, and the stored walk
// vectors s_1..s_r are repaired level by level.  An undirected edge {a, b} is
// the two arcs a -> b and b -> a (Sec. 2.1); a directed update a -> b changes
// the row of a alone.
//
// Repair (the pull form of Algorithm 2's update, see katz_api.cu):
//   F_1 = the rows the batch changed (both endpoints when undirected, the
//         sources when directed);
//   F_i = F_{i-1} + in-neighbours of the nodes that joined F_{i-1} (reverse
//         BFS; in-neighbours = neighbours for undirected graphs, and a
//         transposed CSR of the updated graph when directed);
//   s_i(w) is recomputed for w in F_i from the already repaired level i-1
//   with the lane partition of the static SpMV, so the repaired vectors equal
//   a full recomputation on the updated graph.  Once F_i holds more than
//   frontier_abort_frac of the nodes or of the arcs, the remaining levels are
//   recomputed for all nodes (the paper aborts the BFS when S becomes large;
//   on graphs with hubs the arcs of S, not its size, measure the work).
// Nothing is changed unless the whole batch passes validation.
//
// The adjacency is rebuilt into a spare array: runs of untouched rows move as
// one contiguous copy (their offsets shift by a constant), touched rows drop
// their deleted arcs (looked up in the batch's pair table) and append their
// inserted ones; CHUNK rows (the hubs) are copied chunk-parallel or compacted
// by a whole block.
#include <stdint.h>

#include <algorithm>

#include "katz_common.cuh"

namespace katz {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// position of `target` in row u (first match), -1 if absent; one warp
template <typename Off>
__device__ __forceinline__ int64_t find_in_row(const Off* rowptr, const int32_t* col, int64_t u, int32_t target) {
    const int lane = threadIdx.x & 31;
    const int64_t a = rowptr[u], b = rowptr[u + 1];
    for (int64_t base = a; base < b; base += 32) {
        const int64_t j = base + lane;
        const bool hit = j < b && col[j] == target;
        const unsigned m = __ballot_sync(FULL, hit);
        if (m) return base + (__ffs(m) - 1);
    }
    return -1;
}

constexpr unsigned long long DEL_BIT = 1ull << 63;

// key of the edge u -> v of internal ids: the unordered pair {u, v} when
// undirected, the ordered pair when directed (never 0, bit 63 clear)
__device__ __forceinline__ unsigned long long pair_key(int32_t u, int32_t v, bool und) {
    const int32_t a = und ? min(u, v) : u, b = und ? max(u, v) : v;
    return (((unsigned long long)(uint32_t)a << 32) | (uint32_t)b) + 1ull;
}

// the stored entry of `key` (with its delete bit), 0 if absent
__device__ __forceinline__ unsigned long long table_find(const unsigned long long* __restrict__ table, int64_t mask,
                                                         unsigned long long key) {
    int64_t h = (int64_t)(mix64(key) & (unsigned long long)mask);
    for (int64_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long t = table[h];
        if (t == 0ull) return 0ull;
        if ((t & ~DEL_BIT) == key) return t;
        h = (h + 1) & mask;
    }
    return 0ull;
}

// out[j - a] = col[j] for j in [a, b): one warp, eight loads in flight per
// lane (one load at a time left the copy at a third of the bandwidth)
__device__ __forceinline__ void warp_copy(const int32_t* __restrict__ col, int64_t a, int64_t b,
                                          int32_t* __restrict__ out) {
    constexpr int U = 8;
    int64_t j = a + (threadIdx.x & 31);
    for (; j + (U - 1) * 32 < b; j += U * 32) {
        int32_t v[U];
#pragma unroll
        for (int q = 0; q < U; ++q) v[q] = col[j + q * 32];
#pragma unroll
        for (int q = 0; q < U; ++q) out[j + q * 32 - a] = v[q];
    }
    for (; j < b; j += 32) out[j - a] = col[j];
}

// One warp per update: range, self-loop, duplicate (the pair table, which
// also records deletions for the rebuild), presence (I and E disjoint, D a
// subset of E; an undirected graph is symmetric, so the shorter of the two
// rows decides; a directed arc is looked up in its source's row), degree
// deltas and the touched rows.
template <typename Off>
__global__ void validate_batch_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                                      const int32_t* __restrict__ inv, int64_t n, const int32_t* __restrict__ src,
                                      const int32_t* __restrict__ dst, const uint8_t* __restrict__ ins, int64_t m,
                                      bool und, unsigned long long* table, int64_t table_mask, int32_t* delta,
                                      uint8_t* touched, int32_t* err) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; e < m; e += warps) {
        const int32_t a = src[e], b = dst[e];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b) {
            if (lane == 0) atomicOr(err, DYN_E_INVAL);
            continue;
        }
        const int32_t ua = inv[a], ub = inv[b];
        if (lane == 0) {  // duplicate pair inside the batch
            const unsigned long long key = pair_key(ua, ub, und);
            const unsigned long long entry = key | (ins[e] ? 0ull : DEL_BIT);
            int64_t h = (int64_t)(mix64(key) & (unsigned long long)table_mask);
            for (int64_t probe = 0; probe <= table_mask; ++probe) {
                const unsigned long long old = atomicCAS(&table[h], 0ull, entry);
                if (old == 0ull) break;
                if ((old & ~DEL_BIT) == key) {
                    atomicOr(err, DYN_E_INVAL);
                    break;
                }
                h = (h + 1) & table_mask;
            }
        }
        const int64_t da = (int64_t)rowptr[ua + 1] - (int64_t)rowptr[ua];
        const int64_t db = (int64_t)rowptr[ub + 1] - (int64_t)rowptr[ub];
        const int64_t pos =
            (!und || da <= db) ? find_in_row(rowptr, col, ua, ub) : find_in_row(rowptr, col, ub, ua);
        if (lane == 0) {
            if (ins[e] ? pos >= 0 : pos < 0) atomicOr(err, DYN_E_INVAL);
            const int d = ins[e] ? 1 : -1;
            atomicAdd(&delta[ua], d);
            touched[ua] = 1;
            if (und) {
                atomicAdd(&delta[ub], d);
                touched[ub] = 1;
            }
        }
    }
}

// the rows the batch changes stay within D arcs (out-degrees when directed)
template <typename Off>
__global__ void degree_check_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ inv,
                                    const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                                    int64_t n, bool und, const int32_t* __restrict__ delta, int64_t D, int32_t* err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t a = src[e], b = dst[e];
        if (a < 0 || b < 0 || a >= n || b >= n) continue;
        const int32_t ends[2] = {inv[a], inv[b]};
        for (int q = 0; q < (und ? 2 : 1); ++q) {
            const int64_t u = ends[q];
            if ((int64_t)rowptr[u + 1] - (int64_t)rowptr[u] + delta[u] > D) atomicOr(err, DYN_E_ALPHA);
        }
    }
}

// undo the per-node scratch of a batch (delta, insertion counters, marks)
__global__ void clear_batch_kernel(const int32_t* __restrict__ inv, const int32_t* __restrict__ src,
                                   const int32_t* __restrict__ dst, int64_t m, int64_t n, int32_t* delta,
                                   int32_t* ins_cnt, int32_t* cursor, uint8_t* touched) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t a = src[e], b = dst[e];
        if (a < 0 || b < 0 || a >= n || b >= n) continue;
        const int32_t ends[2] = {inv[a], inv[b]};
        for (int q = 0; q < 2; ++q) {
            delta[ends[q]] = 0;
            ins_cnt[ends[q]] = 0;
            cursor[ends[q]] = 0;
            touched[ends[q]] = 0;
        }
    }
}

// insertions: count per row and list the rows that receive arcs
__global__ void count_inserts_kernel(const int32_t* __restrict__ inv, const int32_t* __restrict__ src,
                                     const int32_t* __restrict__ dst, const uint8_t* __restrict__ ins, int64_t m,
                                     bool und, int32_t* ins_cnt, int32_t* ins_rows,
                                     unsigned long long* n_ins_rows) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        if (!ins[e]) continue;
        const int32_t ends[2] = {inv[src[e]], inv[dst[e]]};
        for (int q = 0; q < (und ? 2 : 1); ++q)
            if (atomicAdd(&ins_cnt[ends[q]], 1) == 0) ins_rows[atomicAdd(n_ins_rows, 1ULL)] = ends[q];
    }
}

// exclusive offsets of the insertion buckets (one block; the row list is short)
__global__ void bucket_offsets_kernel(const int32_t* __restrict__ ins_rows, const unsigned long long* n_ins_rows,
                                      const int32_t* __restrict__ ins_cnt, int64_t* ins_start) {
    __shared__ long long part[1024];
    const int tid = threadIdx.x;
    const int64_t cnt = (int64_t)*n_ins_rows;
    const int64_t chunk = (cnt + 1023) / 1024;
    long long s = 0;
    for (int64_t q = tid * chunk; q < min(cnt, (int64_t)(tid + 1) * chunk); ++q) s += ins_cnt[ins_rows[q]];
    part[tid] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const long long a = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += a;
        __syncthreads();
    }
    long long run = tid ? part[tid - 1] : 0;
    for (int64_t q = tid * chunk; q < min(cnt, (int64_t)(tid + 1) * chunk); ++q) {
        ins_start[ins_rows[q]] = run;
        run += ins_cnt[ins_rows[q]];
    }
}

// place the inserted arcs (original id of the target kept for the sort)
__global__ void bucket_fill_kernel(const int32_t* __restrict__ inv, const int32_t* __restrict__ src,
                                   const int32_t* __restrict__ dst, const uint8_t* __restrict__ ins, int64_t m,
                                   bool und, const int64_t* __restrict__ ins_start, int32_t* cursor,
                                   int32_t* bucket) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        if (!ins[e]) continue;
        const int32_t a = src[e], b = dst[e];
        const int32_t ua = inv[a], ub = inv[b];
        bucket[ins_start[ua] + atomicAdd(&cursor[ua], 1)] = b;
        if (und) bucket[ins_start[ub] + atomicAdd(&cursor[ub], 1)] = a;
    }
}

// each bucket sorted by original id (deterministic row contents), then
// renamed to internal ids
__global__ void bucket_sort_kernel(const int32_t* __restrict__ ins_rows, const unsigned long long* n_ins_rows,
                                   const int32_t* __restrict__ ins_cnt, const int64_t* __restrict__ ins_start,
                                   const int32_t* __restrict__ inv, int32_t* bucket) {
    const int64_t cnt = (int64_t)*n_ins_rows;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += stride) {
        const int32_t u = ins_rows[q];
        int32_t* bkt = bucket + ins_start[u];
        const int c = ins_cnt[u];
        for (int i = 1; i < c; ++i) {
            const int32_t v = bkt[i];
            int j = i - 1;
            while (j >= 0 && bkt[j] > v) {
                bkt[j + 1] = bkt[j];
                --j;
            }
            bkt[j + 1] = v;
        }
        for (int i = 0; i < c; ++i) bkt[i] = inv[bkt[i]];
    }
}

template <typename Off>
__global__ void new_degrees_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ delta, int64_t n,
                                   int64_t* deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride)
        deg[u] = (int64_t)rowptr[u + 1] - (int64_t)rowptr[u] + delta[u];
}

// a touched row: its arcs minus the deleted ones (in their order), then its
// inserted arcs; one warp.  A row without deletions is copied as it is.
template <typename Off>
__device__ __forceinline__ void rebuild_touched_row(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                    int64_t v, int64_t o, const int32_t* __restrict__ ins_cnt,
                                                    const int64_t* __restrict__ ins_start,
                                                    const int32_t* __restrict__ bucket,
                                                    const unsigned long long* __restrict__ table, int64_t mask,
                                                    bool und, bool no_deletes, int32_t* col_new) {
    const int lane = threadIdx.x & 31;
    const int64_t a = rowptr[v], b = rowptr[v + 1];
    if (no_deletes) {
        warp_copy(col, a, b, col_new + o);
        o += b - a;
    }
    for (int64_t base = a; !no_deletes && base < b; base += 32) {
        const int64_t j = base + lane;
        const int32_t x = j < b ? col[j] : -1;
        const bool keep = x >= 0 && !(table_find(table, mask, pair_key((int32_t)v, x, und)) & DEL_BIT);
        const unsigned kb = __ballot_sync(FULL, keep);
        if (keep) col_new[o + __popc(kb & ((1u << lane) - 1u))] = x;
        o += __popc(kb);
    }
    const int c = ins_cnt[v];
    const int32_t* bkt = bucket + ins_start[v];
    for (int q = lane; q < c; q += 32) col_new[o + q] = bkt[q];
}

// rows from row_lo on (no CHUNK rows): one warp per 32 consecutive rows; a
// run without touched rows is one contiguous copy
template <typename Off>
__global__ void rebuild_groups_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                                      const int64_t* __restrict__ rowptr_new, const uint8_t* __restrict__ touched,
                                      const int32_t* __restrict__ ins_cnt, const int64_t* __restrict__ ins_start,
                                      const int32_t* __restrict__ bucket, const unsigned long long* __restrict__ table,
                                      int64_t mask, bool und, int64_t row_lo, int64_t n, int32_t* col_new) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t groups = (n - row_lo + 31) / 32;
    for (int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; gi < groups; gi += warps) {
        const int64_t u0 = row_lo + gi * 32, u1 = min(u0 + 32, n);
        const bool t = u0 + lane < u1 && touched[u0 + lane];
        const unsigned tb = __ballot_sync(FULL, t);
        // the runs of untouched rows between touched ones, each one copy
        // (touched rows are rebuilt by rebuild_touched_kernel)
        int64_t v = u0;
        while (v < u1) {
            while (v < u1 && ((tb >> (v - u0)) & 1u)) ++v;
            int64_t w = v;
            while (w < u1 && !((tb >> (w - u0)) & 1u)) ++w;
            if (w > v) warp_copy(col, rowptr[v], rowptr[w], col_new + rowptr_new[v]);
            v = w;
        }
    }
}

// the first caller for row u gets true (its touched byte gains bit 1; the
// array is padded to whole words)
__device__ __forceinline__ bool claim_row(uint8_t* touched, int64_t u) {
    unsigned int* w = (unsigned int*)(touched + (u & ~(int64_t)3));
    const unsigned int bit = 2u << (8u * (unsigned int)(u & 3));
    return !(atomicOr(w, bit) & bit);
}

// touched rows from row_lo on: one warp per update claims each of its rows
// once and rebuilds it, so the rows of a batch are rebuilt in parallel
template <typename Off>
__global__ void rebuild_touched_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                                       const int64_t* __restrict__ rowptr_new, const int32_t* __restrict__ inv,
                                       const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                                       bool und, int64_t row_lo, uint8_t* touched,
                                       const int32_t* __restrict__ ins_cnt, const int32_t* __restrict__ delta,
                                       const int64_t* __restrict__ ins_start, const int32_t* __restrict__ bucket,
                                       const unsigned long long* __restrict__ table, int64_t mask,
                                       int32_t* col_new) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; e < m; e += warps) {
        for (int q = 0; q < (und ? 2 : 1); ++q) {
            const int64_t u = inv[q ? dst[e] : src[e]];
            if (u < row_lo) continue;  // CHUNK rows: the hub kernels
            int mine = lane == 0 ? (int)claim_row(touched, u) : 0;
            if (!__shfl_sync(FULL, mine, 0)) continue;
            rebuild_touched_row(rowptr, col, u, rowptr_new[u], ins_cnt, ins_start, bucket, table, mask, und,
                                ins_cnt[u] == delta[u], col_new);
        }
    }
}

// untouched CHUNK rows: one warp per chunk copies it to its new place
template <typename Off>
__global__ void rebuild_chunks_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                                      const int64_t* __restrict__ rowptr_new, const uint8_t* __restrict__ touched,
                                      const int32_t* __restrict__ chunk_row, const int64_t* __restrict__ chunk_first,
                                      int64_t chunks, int32_t* col_new) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t ch = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; ch < chunks; ch += warps) {
        const int64_t u = chunk_row[ch];
        if (touched[u]) continue;
        const int64_t j0 = (int64_t)rowptr[u] + (ch - chunk_first[u]) * (int64_t)CHUNK_ARCS;
        const int64_t j1 = min(j0 + (int64_t)CHUNK_ARCS, (int64_t)rowptr[u + 1]);
        warp_copy(col, j0, j1, col_new + rowptr_new[u] + (j0 - (int64_t)rowptr[u]));
    }
}

// Touched CHUNK rows, compacted chunk by chunk: (A) one warp per chunk counts
// the arcs it keeps, (B) one warp per row turns the counts into the chunks'
// places in the new row and appends the inserted arcs after them, (C) one
// warp per chunk writes its kept arcs, in order, at its place.
template <typename Off>
__device__ __forceinline__ void hub_chunk_range(const Off* __restrict__ rowptr, const int32_t* __restrict__ chunk_row,
                                                const int64_t* __restrict__ chunk_first, int64_t ch, int64_t& u,
                                                int64_t& j0, int64_t& j1) {
    u = chunk_row[ch];
    j0 = (int64_t)rowptr[u] + (ch - chunk_first[u]) * (int64_t)CHUNK_ARCS;
    j1 = min(j0 + (int64_t)CHUNK_ARCS, (int64_t)rowptr[u + 1]);
}

template <typename Off>
__global__ void hub_keep_count_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                                      const uint8_t* __restrict__ touched, const int32_t* __restrict__ chunk_row,
                                      const int64_t* __restrict__ chunk_first, int64_t chunks,
                                      const unsigned long long* __restrict__ table, int64_t mask, bool und,
                                      int64_t* keep) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t ch = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; ch < chunks; ch += warps) {
        int64_t u, j0, j1;
        hub_chunk_range(rowptr, chunk_row, chunk_first, ch, u, j0, j1);
        if (!touched[u]) continue;
        int64_t cnt = 0;
        for (int64_t base = j0; base < j1; base += 32) {
            const int64_t j = base + lane;
            const int32_t x = j < j1 ? col[j] : -1;
            const bool k = x >= 0 && !(table_find(table, mask, pair_key((int32_t)u, x, und)) & DEL_BIT);
            cnt += __popc(__ballot_sync(FULL, k));
        }
        if (lane == 0) keep[ch] = cnt;
    }
}

template <typename Off>
__global__ void hub_keep_scan_kernel(const uint8_t* __restrict__ touched, const int64_t* __restrict__ chunk_first,
                                     const int64_t* __restrict__ rowptr_new, const int32_t* __restrict__ ins_cnt,
                                     const int64_t* __restrict__ ins_start, const int32_t* __restrict__ bucket,
                                     int64_t row_warp, int64_t* keep, int32_t* col_new) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; u < row_warp; u += warps) {
        if (!touched[u]) continue;
        int64_t run = rowptr_new[u];
        for (int64_t c0 = chunk_first[u]; c0 < chunk_first[u + 1]; c0 += 32) {
            const int64_t ch = c0 + lane;
            const int64_t k = ch < chunk_first[u + 1] ? keep[ch] : 0;
            int64_t incl = k;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int64_t y = __shfl_up_sync(FULL, incl, off);
                if (lane >= off) incl += y;
            }
            if (ch < chunk_first[u + 1]) keep[ch] = run + incl - k;  // the chunk's first place
            run += __shfl_sync(FULL, incl, 31);
        }
        const int c = ins_cnt[u];
        const int32_t* bkt = bucket + ins_start[u];
        for (int q = lane; q < c; q += 32) col_new[run + q] = bkt[q];
    }
}

template <typename Off>
__global__ void hub_keep_write_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                                      const uint8_t* __restrict__ touched, const int32_t* __restrict__ chunk_row,
                                      const int64_t* __restrict__ chunk_first, int64_t chunks,
                                      const unsigned long long* __restrict__ table, int64_t mask, bool und,
                                      const int64_t* __restrict__ place, int32_t* col_new) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t ch = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; ch < chunks; ch += warps) {
        int64_t u, j0, j1;
        hub_chunk_range(rowptr, chunk_row, chunk_first, ch, u, j0, j1);
        if (!touched[u]) continue;
        int64_t o = place[ch];
        for (int64_t base = j0; base < j1; base += 32) {
            const int64_t j = base + lane;
            const int32_t x = j < j1 ? col[j] : -1;
            const bool k = x >= 0 && !(table_find(table, mask, pair_key((int32_t)u, x, und)) & DEL_BIT);
            const unsigned kb = __ballot_sync(FULL, k);
            if (k) col_new[o + __popc(kb & ((1u << lane) - 1u))] = x;
            o += __popc(kb);
        }
    }
}

template <typename Off>
__global__ void narrow_kernel(const int64_t* __restrict__ in, Off* __restrict__ out, int64_t count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride) out[q] = (Off)in[q];
}

// test-and-set of u's visit bit; true if u was not visited before
__device__ __forceinline__ bool visit(uint32_t* vbits, int32_t u) {
    const uint32_t bit = 1u << (u & 31);
    return !(atomicOr(&vbits[u >> 5], bit) & bit);
}

template <typename Off>
__device__ __forceinline__ int64_t degree(const Off* __restrict__ rowptr, int64_t u) {
    return (int64_t)rowptr[u + 1] - (int64_t)rowptr[u];
}

// a node joins the frontier: listed, its degree counted by the caller, a
// CHUNK row remembers the level it joined at
__device__ __forceinline__ void join(int32_t x, int level, int64_t row_warp, int32_t* frontier,
                                     unsigned long long* fsize, int32_t* hub_epoch) {
    frontier[atomicAdd(&fsize[0], 1ULL)] = x;
    if (x < row_warp) hub_epoch[x] = level;
}

// F_1: the rows every update changed (both endpoints when undirected, the
// source when directed)
template <typename Off>
__global__ void seed_frontier_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ inv,
                                     const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                                     bool und, int64_t row_warp, uint32_t* vbits, int32_t* frontier,
                                     unsigned long long* fsize, int32_t* hub_epoch) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t ends[2] = {inv[src[e]], inv[dst[e]]};
        for (int q = 0; q < (und ? 2 : 1); ++q) {
            if (visit(vbits, ends[q])) {
                join(ends[q], 1, row_warp, frontier, fsize, hub_epoch);
                atomicAdd(&fsize[1], (unsigned long long)degree(rowptr, ends[q]));
            }
        }
    }
}

// neighbours of the arcs [j0, j1) join F_{level+1}; returns the degrees added
template <typename Off>
__device__ __forceinline__ unsigned long long expand_arcs(const Off* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col, int64_t j0, int64_t j1,
                                                          int level, int64_t row_warp, uint32_t* vbits,
                                                          int32_t* frontier, unsigned long long* fsize,
                                                          int32_t* hub_epoch) {
    unsigned long long vol = 0;
    for (int64_t j = j0 + (threadIdx.x & 31); j < j1; j += 32) {
        const int32_t x = col[j];
        if (visit(vbits, x)) {
            join(x, level + 1, row_warp, frontier, fsize, hub_epoch);
            vol += (unsigned long long)degree(rowptr, x);
        }
    }
    return vol;
}

__device__ __forceinline__ void add_warp_volume(unsigned long long vol, unsigned long long* fsize) {
#pragma unroll
    for (int off = 16; off; off >>= 1) vol += __shfl_xor_sync(FULL, vol, off);
    if ((threadIdx.x & 31) == 0 && vol) atomicAdd(&fsize[1], vol);
}

// the neighbours of frontier[lo, hi) join the frontier; one warp per node
// (CHUNK rows are expanded chunk by chunk by expand_hubs_kernel)
template <typename Off>
__global__ void expand_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col, int32_t* frontier,
                              int64_t lo, int64_t hi, int level, int64_t row_warp, uint32_t* vbits,
                              unsigned long long* fsize, int32_t* hub_epoch) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    unsigned long long vol = 0;
    for (int64_t q = lo + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; q < hi; q += warps) {
        const int64_t w = frontier[q];
        if (w < row_warp) continue;
        vol += expand_arcs(rowptr, col, (int64_t)rowptr[w], (int64_t)rowptr[w + 1], level, row_warp, vbits, frontier,
                           fsize, hub_epoch);
    }
    add_warp_volume(vol, fsize);
}

// CHUNK rows that joined at `level`: one warp per chunk
template <typename Off>
__global__ void expand_hubs_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                                   const int32_t* __restrict__ chunk_row, const int64_t* __restrict__ chunk_first,
                                   int64_t chunks, int32_t* frontier, int level, int64_t row_warp, uint32_t* vbits,
                                   unsigned long long* fsize, int32_t* hub_epoch) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    unsigned long long vol = 0;
    for (int64_t ch = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; ch < chunks; ch += warps) {
        const int64_t u = chunk_row[ch];
        if (hub_epoch[u] != level) continue;
        const int64_t j0 = (int64_t)rowptr[u] + (ch - chunk_first[u]) * (int64_t)CHUNK_ARCS;
        const int64_t j1 = min(j0 + (int64_t)CHUNK_ARCS, (int64_t)rowptr[u + 1]);
        vol += expand_arcs(rowptr, col, j0, j1, level, row_warp, vbits, frontier, fsize, hub_epoch);
    }
    add_warp_volume(vol, fsize);
}

// ---- directed graphs: the transposed CSR of the updated graph ----------------
// arcs of the rows from row_lo on into the transposed rows: one warp per 32
// consecutive rows; cursor[x] starts at the first slot of x's in-arcs
template <typename Off>
__global__ void transpose_rows_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t row_lo,
                                      int64_t n, unsigned long long* cursor, int32_t* rcol) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t groups = (n - row_lo + 31) / 32;
    for (int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; gi < groups; gi += warps) {
        const int64_t u0 = row_lo + gi * 32, u1 = min(u0 + 32, n);
        for (int64_t v = u0; v < u1; ++v) {
            const int64_t a = rowptr[v], b = rowptr[v + 1];
            for (int64_t j = a + lane; j < b; j += 32) rcol[atomicAdd(&cursor[col[j]], 1ull)] = (int32_t)v;
        }
    }
}

// the same for the CHUNK rows: one warp per chunk
template <typename Off>
__global__ void transpose_chunks_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                                        const int32_t* __restrict__ chunk_row, const int64_t* __restrict__ chunk_first,
                                        int64_t chunks, unsigned long long* cursor, int32_t* rcol) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t ch = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; ch < chunks; ch += warps) {
        const int64_t u = chunk_row[ch];
        const int64_t j0 = (int64_t)rowptr[u] + (ch - chunk_first[u]) * (int64_t)CHUNK_ARCS;
        const int64_t j1 = min(j0 + (int64_t)CHUNK_ARCS, (int64_t)rowptr[u + 1]);
        for (int64_t j = j0 + lane; j < j1; j += 32) rcol[atomicAdd(&cursor[col[j]], 1ull)] = (int32_t)u;
    }
}

// directed: the in-neighbours of frontier[lo, hi) join the frontier; one
// warp per node, the in-arcs from the transposed CSR, the volume counted in
// out-degrees (the rows a repair recomputes)
template <typename Off>
__global__ void expand_in_kernel(const Off* __restrict__ rowptr, const int64_t* __restrict__ rrowptr,
                                 const int32_t* __restrict__ rcol, int32_t* frontier, int64_t lo, int64_t hi,
                                 int level, int64_t row_warp, uint32_t* vbits, unsigned long long* fsize,
                                 int32_t* hub_epoch) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    unsigned long long vol = 0;
    for (int64_t q = lo + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; q < hi; q += warps) {
        const int64_t w = frontier[q];
        vol += expand_arcs(rowptr, rcol, rrowptr[w], rrowptr[w + 1], level, row_warp, vbits, frontier, fsize,
                           hub_epoch);
    }
    add_warp_volume(vol, fsize);
}

// FP32-certified handles: the largest new degree among the batch's rows in
// each row mode (THREAD, OCTET, WARP), from which the host bounds the chain of
// FP32 additions of a repaired row.  Directed: only the source rows change.
__global__ void mode_degree_max_kernel(const int32_t* __restrict__ inv, const int32_t* __restrict__ src,
                                       const int32_t* __restrict__ dst, int64_t m, int und,
                                       const int64_t* __restrict__ rp_new, SpmvLayout L, unsigned long long* dmax) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += stride) {
        for (int side = 0; side <= und; ++side) {
            const int64_t u = inv[side ? dst[q] : src[q]];
            if (u < L.row_warp) continue;  // CHUNK rows: the host counts their chunks
            const unsigned long long deg = (unsigned long long)(rp_new[u + 1] - rp_new[u]);
            const int slot = u >= L.row_thread ? 0 : (u >= L.row_octet ? 1 : 2);
            atomicMax(dmax + slot, deg);
        }
    }
}

// c_r = s_1 + ... + s_r in level order (the order the static iteration adds
// them).  FP32-certified mode: the FP64 levels into c, the FP32 levels
// (exact in FP64) into c32, as the two partial sums of the ranking.
__global__ void recompute_c_kernel(const double* walk, IterParams p, int r, const int32_t* __restrict__ rows,
                                   const unsigned long long* nrows, int64_t n, double* c, double* c32,
                                   const Ctrl* ctrl) {
    const int64_t cnt = rows ? (int64_t)*nrows : n;
    const int f32_from = ctrl->f32_from;
    const int r64 = min(r, f32_from - 1);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += stride) {
        const int64_t v = rows ? rows[q] : q;
        double acc = 0.0;
        for (int i = 1; i <= r64; ++i) acc = __dadd_rn(acc, walk_slot(walk, p, i)[v]);
        c[v] = acc;
        if (p.cert && c32) {
            double acc32 = 0.0;
            for (int i = f32_from; i <= r; ++i) acc32 = __dadd_rn(acc32, walk_value(walk, p, f32_from, i, v));
            c32[v] = acc32;
        }
    }
}

// a valid candidate threshold after the update: min of the new l_r over the
// previous top-k (at least k nodes reach it)
__global__ void theta_lb_kernel(const int32_t* __restrict__ topk_id, const int32_t* __restrict__ inv,
                                const double* walk, const double* __restrict__ c, const double* __restrict__ c32,
                                IterParams p, int r, Ctrl* ctrl) {
    __shared__ double wmin[32];
    const int kk = ctrl->k_eff;
    const int f32_from = ctrl->f32_from;
    const BState bs = bstate(ctrl, p);
    double m = 1.0 / 0.0;
    for (int q = threadIdx.x; q < kk; q += blockDim.x) {
        const int32_t v = inv[topk_id[q]];
        double l, u;
        node_bounds(c[v], (p.cert && c32) ? c32[v] : 0.0, walk_value(walk, p, f32_from, r, v), p, bs, l, u);
        m = fmin(m, l);
    }
    for (int off = 16; off; off >>= 1) m = fmin(m, __shfl_xor_sync(FULL, m, off));
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = 1.0 / 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) mm = fmin(mm, wmin[w]);
        ctrl->theta_prev = kk > 0 ? mm : 0.0;
        ctrl->r = r - 1;  // the check that follows evaluates level r
        ctrl->n_cand = 0;
        ctrl->cnt_cross = 0;
        ctrl->n_active = 0;
        ctrl->stop = 0;
        ctrl->flags = 0;
        ctrl->converged = 0;
        ctrl->stall = 0;
        ctrl->list_ready = 0;  // every node is reactivated: the next count scans all of V
        ctrl->n_list_next = 0;
    }
}

// Reactivation: the active set is re-derived from all of V (a node outside
// it satisfies the paper's reactivation test exactly when converged() would
// keep it), and the candidates of the check at level r are collected.
__global__ void reactivate_kernel(const double* walk, const double* __restrict__ c, const double* __restrict__ c32,
                                  const int32_t* __restrict__ perm, IterParams p, int r, uint8_t* active,
                                  double* lb, double* ub, double* cand_l, double* cand_u, int32_t* cand_id,
                                  int64_t cand_cap, Ctrl* ctrl) {
    const double th = ctrl->theta_prev;
    const int f32_from = ctrl->f32_from;
    const BState bs = bstate(ctrl, p);
    const bool two = p.cert && c32;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += stride) {
        active[v] = 1;
        double l, u;
        node_bounds(c[v], two ? c32[v] : 0.0, walk_value(walk, p, f32_from, r, v), p, bs, l, u);
        // FP32-certified mode: fresh bounds of the updated graph (the stored
        // ones, which later levels tighten monotonically, belong to the old one)
        lb[v] = l;  // the bounds the deactivation count reads
        ub[v] = u;
        if (l >= th) {
            const unsigned long long pos = atomicAdd(&ctrl->n_cand, 1ULL);
            if (pos < (unsigned long long)cand_cap) {
                cand_l[pos] = l;
                cand_u[pos] = u;
                cand_id[pos] = perm[v];
            }
        }
    }
}

int grid_for(int64_t n, int threads, int max_blocks = 152 * 16) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

}  // namespace

// ---- launchers ---------------------------------------------------------------

cudaError_t dyn_validate(const DeviceGraph& g, const DynBuffers& d, int64_t m, int64_t D, cudaStream_t st) {
    const int wblocks = grid_for(m * 32, 256);
    if (g.off64)
        validate_batch_kernel<int64_t><<<wblocks, 256, 0, st>>>((const int64_t*)g.rowptr, g.col, g.inv, g.n, d.src,
                                                               d.dst, d.ins, m, d.undirected, d.table, d.table_mask,
                                                               d.delta, d.touched, d.err);
    else
        validate_batch_kernel<int32_t><<<wblocks, 256, 0, st>>>((const int32_t*)g.rowptr, g.col, g.inv, g.n, d.src,
                                                               d.dst, d.ins, m, d.undirected, d.table, d.table_mask,
                                                               d.delta, d.touched, d.err);
    if (g.off64)
        degree_check_kernel<int64_t><<<grid_for(m, 256), 256, 0, st>>>((const int64_t*)g.rowptr, g.inv, d.src, d.dst,
                                                                      m, g.n, d.undirected, d.delta, D, d.err);
    else
        degree_check_kernel<int32_t><<<grid_for(m, 256), 256, 0, st>>>((const int32_t*)g.rowptr, g.inv, d.src, d.dst,
                                                                      m, g.n, d.undirected, d.delta, D, d.err);
    return cudaGetLastError();
}

cudaError_t dyn_clear(const DeviceGraph& g, const DynBuffers& d, int64_t m, cudaStream_t st) {
    clear_batch_kernel<<<grid_for(m, 256), 256, 0, st>>>(g.inv, d.src, d.dst, m, g.n, d.delta, d.ins_cnt, d.cursor,
                                                          d.touched);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(d.table, 0, (size_t)(d.table_mask + 1) * sizeof(unsigned long long), st);
}

// sorted insertion buckets and the new row offsets
// (int64, n+1 entries, into rowptr_new); the total is rowptr_new[n]
cudaError_t dyn_prepare(const DeviceGraph& g, const DynBuffers& d, int64_t m, int64_t* rowptr_new, int64_t* deg,
                        int64_t* sums, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d.n_ins_rows, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    count_inserts_kernel<<<grid_for(m, 256), 256, 0, st>>>(g.inv, d.src, d.dst, d.ins, m, d.undirected, d.ins_cnt,
                                                           d.ins_rows, d.n_ins_rows);
    bucket_offsets_kernel<<<1, 1024, 0, st>>>(d.ins_rows, d.n_ins_rows, d.ins_cnt, d.ins_start);
    bucket_fill_kernel<<<grid_for(m, 256), 256, 0, st>>>(g.inv, d.src, d.dst, d.ins, m, d.undirected, d.ins_start,
                                                         d.cursor, d.bucket);
    bucket_sort_kernel<<<grid_for(2 * m, 128), 128, 0, st>>>(d.ins_rows, d.n_ins_rows, d.ins_cnt, d.ins_start, g.inv,
                                                            d.bucket);
    if (g.off64)
        new_degrees_kernel<int64_t><<<grid_for(g.n, 256), 256, 0, st>>>((const int64_t*)g.rowptr, d.delta, g.n, deg);
    else
        new_degrees_kernel<int32_t><<<grid_for(g.n, 256), 256, 0, st>>>((const int32_t*)g.rowptr, d.delta, g.n, deg);
    e = cudaMemsetAsync(deg + g.n, 0, sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return exclusive_scan_i64(deg, g.n + 1, rowptr_new, sums, st);
}

template <typename Off>
static void rebuild_launch(const DeviceGraph& g, const DynBuffers& d, int64_t m, const int64_t* rowptr_new,
                           int32_t* col_new, cudaStream_t st) {
    const Off* rp = (const Off*)g.rowptr;
    const SpmvLayout& L = g.layout;
    const int64_t groups = (g.n - L.row_warp + 31) / 32;
    if (groups > 0) {
        rebuild_groups_kernel<Off><<<grid_for(groups * 32, 256), 256, 0, st>>>(
            rp, g.col, rowptr_new, d.touched, d.ins_cnt, d.ins_start, d.bucket, d.table, d.table_mask, d.undirected,
            L.row_warp, g.n, col_new);
        rebuild_touched_kernel<Off><<<grid_for(m * 32, 256), 256, 0, st>>>(
            rp, g.col, rowptr_new, g.inv, d.src, d.dst, m, d.undirected, L.row_warp, d.touched, d.ins_cnt, d.delta,
            d.ins_start, d.bucket, d.table, d.table_mask, col_new);
    }
    if (L.chunks > 0)
        rebuild_chunks_kernel<Off><<<grid_for(L.chunks * 32, 256), 256, 0, st>>>(
            rp, g.col, rowptr_new, d.touched, g.chunk_row, g.chunk_first, L.chunks, col_new);
    if (L.row_warp > 0) {
        hub_keep_count_kernel<Off><<<grid_for(L.chunks * 32, 256), 256, 0, st>>>(
            rp, g.col, d.touched, g.chunk_row, g.chunk_first, L.chunks, d.table, d.table_mask, d.undirected,
            d.hub_keep);
        hub_keep_scan_kernel<Off><<<grid_for(L.row_warp * 32, 256), 256, 0, st>>>(
            d.touched, g.chunk_first, rowptr_new, d.ins_cnt, d.ins_start, d.bucket, L.row_warp, d.hub_keep, col_new);
        hub_keep_write_kernel<Off><<<grid_for(L.chunks * 32, 256), 256, 0, st>>>(
            rp, g.col, d.touched, g.chunk_row, g.chunk_first, L.chunks, d.table, d.table_mask, d.undirected,
            d.hub_keep, col_new);
    }
}

// rows into col_new (read through the old layout and chunk table), and the
// new offsets into rowptr_out: int64 when g has int64 offsets or out64 is set
// (a batch that outgrows int32 offsets), else int32 (g itself unchanged)
cudaError_t dyn_rebuild(const DeviceGraph& g, const DynBuffers& d, int64_t m, const int64_t* rowptr_new,
                        int32_t* col_new, void* rowptr_out, bool out64, cudaStream_t st) {
    if (g.off64)
        rebuild_launch<int64_t>(g, d, m, rowptr_new, col_new, st);
    else
        rebuild_launch<int32_t>(g, d, m, rowptr_new, col_new, st);
    if (g.off64 || out64)
        narrow_kernel<int64_t><<<grid_for(g.n + 1, 256), 256, 0, st>>>(rowptr_new, (int64_t*)rowptr_out, g.n + 1);
    else
        narrow_kernel<int32_t><<<grid_for(g.n + 1, 256), 256, 0, st>>>(rowptr_new, (int32_t*)rowptr_out, g.n + 1);
    return cudaGetLastError();
}

// F_1 on the updated graph; fsize = {|F_1|, sum of degrees}
cudaError_t dyn_seed(const DeviceGraph& g, const DynBuffers& d, int64_t m, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d.vbits, 0, (size_t)((g.n + 31) / 32) * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.fsize, 0, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess && g.layout.row_warp > 0)
        e = cudaMemsetAsync(d.hub_epoch, 0, (size_t)g.layout.row_warp * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    if (g.off64)
        seed_frontier_kernel<int64_t><<<grid_for(m, 256), 256, 0, st>>>((const int64_t*)g.rowptr, g.inv, d.src, d.dst,
                                                                       m, d.undirected, g.layout.row_warp, d.vbits,
                                                                       d.frontier, d.fsize, d.hub_epoch);
    else
        seed_frontier_kernel<int32_t><<<grid_for(m, 256), 256, 0, st>>>((const int32_t*)g.rowptr, g.inv, d.src, d.dst,
                                                                       m, d.undirected, g.layout.row_warp, d.vbits,
                                                                       d.frontier, d.fsize, d.hub_epoch);
    return cudaGetLastError();
}

// F_{level+1} from the nodes that joined at `level` (frontier[lo, hi))
cudaError_t dyn_expand(const DeviceGraph& g, const DynBuffers& d, int64_t lo, int64_t hi, int level,
                       cudaStream_t st) {
    if (hi <= lo) return cudaSuccess;
    const SpmvLayout& L = g.layout;
    if (!d.undirected) {
        if (g.off64)
            expand_in_kernel<int64_t><<<grid_for((hi - lo) * 32, 256), 256, 0, st>>>(
                (const int64_t*)g.rowptr, d.rrowptr, d.rcol, d.frontier, lo, hi, level, L.row_warp, d.vbits, d.fsize,
                d.hub_epoch);
        else
            expand_in_kernel<int32_t><<<grid_for((hi - lo) * 32, 256), 256, 0, st>>>(
                (const int32_t*)g.rowptr, d.rrowptr, d.rcol, d.frontier, lo, hi, level, L.row_warp, d.vbits, d.fsize,
                d.hub_epoch);
        return cudaGetLastError();
    }
    if (g.off64) {
        expand_kernel<int64_t><<<grid_for((hi - lo) * 32, 256), 256, 0, st>>>(
            (const int64_t*)g.rowptr, g.col, d.frontier, lo, hi, level, L.row_warp, d.vbits, d.fsize, d.hub_epoch);
        if (L.chunks > 0)
            expand_hubs_kernel<int64_t><<<grid_for(L.chunks * 32, 256), 256, 0, st>>>(
                (const int64_t*)g.rowptr, g.col, g.chunk_row, g.chunk_first, L.chunks, d.frontier, level, L.row_warp,
                d.vbits, d.fsize, d.hub_epoch);
    } else {
        expand_kernel<int32_t><<<grid_for((hi - lo) * 32, 256), 256, 0, st>>>(
            (const int32_t*)g.rowptr, g.col, d.frontier, lo, hi, level, L.row_warp, d.vbits, d.fsize, d.hub_epoch);
        if (L.chunks > 0)
            expand_hubs_kernel<int32_t><<<grid_for(L.chunks * 32, 256), 256, 0, st>>>(
                (const int32_t*)g.rowptr, g.col, g.chunk_row, g.chunk_first, L.chunks, d.frontier, level, L.row_warp,
                d.vbits, d.fsize, d.hub_epoch);
    }
    return cudaGetLastError();
}

// directed graphs: the transposed CSR of the current graph into d.rrowptr /
// d.rcol (capacity d.rcap >= nnz); cnt: n + 1 int64 of scratch
cudaError_t dyn_transpose(const DeviceGraph& g, const DynBuffers& d, int64_t* cnt, int64_t* sums, cudaStream_t st) {
    const int64_t n = g.n;
    const SpmvLayout& L = g.layout;
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)(n + 1) * sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
    if ((e = launch_indegree(g.col, g.nnz, cnt, st)) != cudaSuccess) return e;
    if ((e = exclusive_scan_i64(cnt, n + 1, d.rrowptr, sums, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(cnt, d.rrowptr, (size_t)n * sizeof(int64_t), cudaMemcpyDeviceToDevice, st)) !=
        cudaSuccess)
        return e;
    if (g.nnz == 0) return cudaSuccess;
    unsigned long long* cur = (unsigned long long*)cnt;
    const int64_t groups = (n - L.row_warp + 31) / 32;
    if (g.off64) {
        if (groups > 0)
            transpose_rows_kernel<int64_t><<<grid_for(groups * 32, 256), 256, 0, st>>>(
                (const int64_t*)g.rowptr, g.col, L.row_warp, n, cur, d.rcol);
        if (L.chunks > 0)
            transpose_chunks_kernel<int64_t><<<grid_for(L.chunks * 32, 256), 256, 0, st>>>(
                (const int64_t*)g.rowptr, g.col, g.chunk_row, g.chunk_first, L.chunks, cur, d.rcol);
    } else {
        if (groups > 0)
            transpose_rows_kernel<int32_t><<<grid_for(groups * 32, 256), 256, 0, st>>>(
                (const int32_t*)g.rowptr, g.col, L.row_warp, n, cur, d.rcol);
        if (L.chunks > 0)
            transpose_chunks_kernel<int32_t><<<grid_for(L.chunks * 32, 256), 256, 0, st>>>(
                (const int32_t*)g.rowptr, g.col, g.chunk_row, g.chunk_first, L.chunks, cur, d.rcol);
    }
    return cudaGetLastError();
}

cudaError_t dyn_mode_degree_max(const DeviceGraph& g, const DynBuffers& d, int64_t m, const int64_t* rp_new,
                                cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d.mode_dmax, 0, 3 * sizeof(unsigned long long), st);
    if (e != cudaSuccess || m <= 0) return e;
    mode_degree_max_kernel<<<grid_for(m, 256), 256, 0, st>>>(g.inv, d.src, d.dst, m, d.undirected ? 1 : 0, rp_new,
                                                             g.layout, d.mode_dmax);
    return cudaGetLastError();
}

cudaError_t dyn_recompute_c(const DeviceGraph& g, const IterBuffers& b, const DynBuffers& d, const IterParams& p,
                            int r, bool all, cudaStream_t st) {
    recompute_c_kernel<<<grid_for(g.n, 256), 256, 0, st>>>((const double*)b.walk, p, r, all ? nullptr : d.frontier,
                                                           d.fsize, g.n, b.c, b.c32, b.ctrl);
    return cudaGetLastError();
}

cudaError_t dyn_reactivate(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int r, cudaStream_t st) {
    theta_lb_kernel<<<1, 1024, 0, st>>>(b.topk_id, g.inv, (const double*)b.walk, b.c, b.c32, p, r, b.ctrl);
    reactivate_kernel<<<grid_for(g.n, 256), 256, 0, st>>>((const double*)b.walk, b.c, b.c32, g.perm, p, r, b.active,
                                                          b.lb, b.ub, b.cand_l, b.cand_u, b.cand_id, b.cand_cap,
                                                          b.ctrl);
    return cudaGetLastError();
}

}  // namespace katz
