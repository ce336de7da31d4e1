// Internal declarations shared by the kernels and the C-ABI driver.
//
// Data layout in device memory (one handle), vertices in internal order
// (degree classes, largest first; see katz_relabel.cu):
//   rowptr   Off[n+1]     CSR row offsets (Off = int32 when n+nnz < 2^31, else int64)
//   col      int32[nnz]   CSR column ids (out-neighbours, internal ids)
//   perm/inv int32[n]     internal -> original id and back
//   chunk_*               the 2048-arc chunks of rows of degree > 2048
//   walk     T[slots][stride]  scaled walk vectors s_i = alpha^i omega_i,
//                         slot i % slots; entry n of every slot is 0
//   c        f64[n]       Katz partial sum c_r (Eq. 1 truncated at r)
//   active   u8[n]        membership in the active set M (Alg. 1)
//   cand     {f64 l, f64 u, i32 id}[n]  nodes of M with l_r >= theta_{r-1}
//   topk     {i32 id, f64 l, f64 u}[KATZ_MAX_K]  current top-k, sorted
//   ctrl     Ctrl         iteration counters read and written by the kernels
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/katz.h"

namespace katz {

constexpr int NUM_CLASSES = 34;   // degree classes: 0, then ceil(log2 deg) + 1
constexpr int CHUNK_ARCS = 2048;  // arcs per warp for rows of degree > 2048
constexpr int SELECT_CAP = KATZ_MAX_K;
constexpr int SELECT_THREADS = 1024;

enum : int32_t { DYN_E_INVAL = 1, DYN_E_ALPHA = 2 };  // batch validation failures

// Iteration state kept on the device so that a captured graph can loop
// without host round trips.
struct Ctrl {
    int32_t r;           // iterations completed
    int32_t converged;   // result of the last converged() evaluation
    int32_t stop;        // 1: leave the loop
    int32_t flags;       // reserved (0)
    unsigned long long n_cand;     // |{v in M : l_r(v) >= theta_{r-1}}|
    unsigned long long cnt_cross;  // active nodes outside the top-k with u_r - eps >= theta_r
    unsigned long long n_active;   // |M| after deactivation
    double theta_prev;   // theta_{r-1}: k-th largest lower bound of the previous iteration
    double theta;        // theta_r
    int32_t theta_id;    // original id of the k-th node (ties of l broken by smaller id)
    int32_t k_eff;       // entries in the top-k list
    double tau;          // candidate filter used by the select (diagnostic)
    unsigned long long body_runs;  // loop bodies executed (finalize calls that did work)
    // FP32-certified mode (unused in FP64 mode): levels >= f32_from are FP32
    int32_t f32_from;    // first FP32 level (INT32_MAX: none yet)
    int32_t stall;       // 1: rounding widening dominates; more iterations cannot certify
    double e_cur;        // relative error bound of the stored s_r of the current level
    double e64;          // largest relative error bound over the FP64 levels
    double lo64, hi64;   // c64 * lo64 <= exact FP64-level part <= c64 * hi64
    double lo32, hi32;   // same for c32, the FP32-level part
    double los, his;     // same for the stored s_r of the current level
    double tail_lo, tail_hi;  // RD(alpha los), RU(alpha gamma his): the tail factors of l and u
    // FP32 results that fall into the subnormal range carry an absolute error
    // (at most 2^-150 per rounding) instead of a relative one: a_cur bounds it
    // for the stored s_r, a_sum for the FP32 levels summed in c32 (both are
    // folded into lo64 / hi64)
    double a_cur, a_sum;
    unsigned long long smax_bits, smax_prev_bits;  // max s_r over M (this / previous level)
    unsigned long long tailw_bits, roundw_bits;    // max tail width / rounding width over M
    // the active set M as a compact list, kept by the count kernel
    int32_t list_ready;  // 1: alist[list_cur] holds exactly the active nodes (n_list of them)
    int32_t list_cur;
    unsigned long long n_list, n_list_next;
};

// Per-call constants.
struct IterParams {
    double alpha;      // attenuation
    double ag;         // alpha * gamma, gamma = D / (1 - alpha D) (Theorem 1)
    double eps;        // separation slack of Eq. (3)
    int64_t n;
    int64_t k;         // effective k
    int64_t stride;    // elements per walk slot (8-byte units)
    int32_t slots;     // walk slots (ring of `slots` levels)
    int32_t undirected;
    int32_t r_max;
    int32_t cert;      // 1: FP32-certified mode (rigorous widening, FP32 levels)
    double ag_hi;      // an upper bound of alpha*gamma (cert mode)
    float alpha_f;     // alpha rounded to FP32 (cert mode, FP32 levels)
    int32_t depth;     // longest chain of additions in one row sum of the SpMV
    int32_t fp32_from; // cert mode: forced first FP32 level (0: automatic)
};

// Lower and upper bound of Alg. 1 from the Katz partial sum and s_r:
//   l_r = c_r + alpha * s_r   (undirected; Sec. 3.1)      l_r = c_r (directed)
//   u_r = c_r + alpha*gamma * s_r                          (Theorem 1)
// FP64 mode: c_r = c64, with round-to-nearest as the paper.  FP32-certified
// mode: the partial sum is c64 (FP64 levels) + c32 (FP32 levels) and every
// stored quantity carries a proven relative error; the bounds are widened by
// it and evaluated with directed rounding, so l_r <= Katz <= u_r holds for the
// exact Katz score.  Explicit rounding intrinsics: every kernel that re-derives
// the bounds gets bit-identical values (no contraction into FMA).
struct BState {
    double lo64, hi64, lo32, hi32;
    double a_lo, a_hi;  // cert mode: RD(alpha los) and RU(alpha gamma his), the tail factors of l and u
};

// the factors are derived once per level by the certification state machine
__device__ __forceinline__ BState bstate(const Ctrl* c, const IterParams& p) {
    (void)p;
    return BState{c->lo64, c->hi64, c->lo32, c->hi32, c->tail_lo, c->tail_hi};
}

__device__ __forceinline__ void node_bounds(double c64, double c32, double s_r, const IterParams& p,
                                            const BState& b, double& l, double& u) {
    if (!p.cert) {
        l = p.undirected ? __dadd_rn(c64, __dmul_rn(p.alpha, s_r)) : c64;
        u = __dadd_rn(c64, __dmul_rn(p.ag, s_r));
        return;
    }
    // c32 = +0 (every node before the switch to FP32 levels): its terms add
    // exactly nothing, and the FP64 pipe (narrow on this GPU) is spared them
    double c_lo, c_hi;
    if (__double_as_longlong(c32) == 0) {
        c_lo = __dmul_rd(c64, b.lo64);
        c_hi = __dmul_ru(c64, b.hi64);
    } else {
        c_lo = __dadd_rd(__dmul_rd(c64, b.lo64), __dmul_rd(c32, b.lo32));
        c_hi = __dadd_ru(__dmul_ru(c64, b.hi64), __dmul_ru(c32, b.hi32));
    }
    // s_r >= 0 and the exact level value lies in [s_r los, s_r his] (up to the
    // absolute terms folded into lo64 / hi64): with the factors rounded
    // outward, s_r a_lo <= alpha s_exact and s_r a_hi >= alpha gamma s_exact.
    // Each tail is one fused multiply-add, rounded once in the safe direction.
    l = p.undirected ? __fma_rd(s_r, b.a_lo, c_lo) : c_lo;
    u = __fma_ru(s_r, b.a_hi, c_hi);
}

template <typename T>
__device__ __forceinline__ T* walk_slot(T* base, const IterParams& p, int level) {
    return base + (size_t)(level % p.slots) * (size_t)p.stride;
}

// s_level(u) as FP64, whatever the level's storage type (slots are 8-byte
// units; an FP32 level uses the first half of its slot)
__device__ __forceinline__ double walk_value(const double* walk, const IterParams& p, int f32_from, int level,
                                             int64_t u) {
    const double* slot = walk_slot(walk, p, level);
    return level >= f32_from ? (double)((const float*)slot)[u] : slot[u];
}

// ---- launchers (katz_kernels.cu) -------------------------------------------

// Internal row ranges of the SpMV row modes and their block ranges.
struct SpmvLayout {
    int64_t n;
    int64_t row_warp;    // rows [0, row_warp): CHUNK mode (degree > 2048)
    int64_t row_octet;   // rows [row_warp, row_octet): WARP mode
    int64_t row_thread;  // rows [row_octet, row_thread): OCTET mode; [row_thread, n): THREAD
    int64_t chunks;      // CHUNK_ARCS-arc chunks of the CHUNK rows
    int64_t blk_warp, blk_octet, blk_thread, blocks_total;  // first block of each mode
};

struct DeviceGraph {
    int64_t n = 0, nnz = 0;
    bool off64 = false;
    void* rowptr = nullptr;   // int32_t* or int64_t*
    int32_t* col = nullptr;
    int32_t* perm = nullptr;  // internal -> original id
    int32_t* inv = nullptr;   // original -> internal id
    int32_t* chunk_row = nullptr;     // [chunks] row of each chunk
    int64_t* chunk_first = nullptr;   // [row_warp + 1] first chunk of each CHUNK row
    double* chunk_part = nullptr;     // [3 chunks] chunk partial sums (three words per chunk)
    SpmvLayout layout{};
};

struct IterBuffers {
    void* walk = nullptr;     // double* or float*
    double* c = nullptr;       // c64: Katz partial sum over the FP64 levels
    double* c32 = nullptr;     // FP32-certified mode: partial sum over the FP32 levels
    double* lb = nullptr;      // FP32-certified mode: stored bounds of active nodes, kept
    double* ub = nullptr;      //   monotone (l = max over levels, u = min over levels)
    uint8_t* active = nullptr;
    float* s32 = nullptr;      // FP32-certified mode: the latest FP64 level rounded to FP32 (the input of
                               //   the first FP32 level, which would otherwise convert every gathered value)
    int32_t* alist[2] = {nullptr, nullptr};  // [n] each: the active nodes (internal ids), double-buffered
    double* cand_l = nullptr;
    double* cand_u = nullptr;
    int32_t* cand_id = nullptr;
    int64_t cand_cap = 0;
    int32_t* topk_id = nullptr;
    double* topk_l = nullptr;
    double* topk_u = nullptr;
    int64_t* trace = nullptr; // |M| per iteration
    Ctrl* ctrl = nullptr;
    unsigned long long cond_handle = 0;  // cudaGraphConditionalHandle (0: none)
    int32_t use_cond = 0;
};

// Scratch of the dynamic update (katz_dynamic.cu); per-node arrays are zero
// between batches.
struct DynBuffers {
    int64_t cap = 0;                 // updates the batch arrays hold
    int32_t* src = nullptr;          // batch, original ids
    int32_t* dst = nullptr;
    uint8_t* ins = nullptr;
    bool undirected = true;          // edges are unordered pairs (both arcs) or ordered ones
    unsigned long long* table = nullptr;  // open-addressing set of the batch's internal-id pairs (bit 63: delete)
    int64_t table_mask = 0;
    int32_t* err = nullptr;
    int32_t* delta = nullptr;        // [n] degree change
    int32_t* ins_cnt = nullptr;      // [n] inserted arcs per row
    int32_t* cursor = nullptr;       // [n]
    uint8_t* touched = nullptr;      // [n] rows of the batch's endpoints
    int64_t* ins_start = nullptr;    // [n] bucket offset
    int32_t* ins_rows = nullptr;     // [2 cap] rows receiving insertions
    unsigned long long* n_ins_rows = nullptr;
    int32_t* bucket = nullptr;       // [2 cap] inserted arcs grouped by row
    uint32_t* vbits = nullptr;       // [n/32] frontier visit marks
    int32_t* frontier = nullptr;     // [n] affected nodes, in order of discovery
    unsigned long long* fsize = nullptr;  // [2] frontier size, sum of the frontier's degrees
    int32_t* hub_epoch = nullptr;    // [row_warp] level at which a CHUNK row joined the frontier
    int64_t* hub_keep = nullptr;     // [hub_keep_cap >= chunks] kept arcs, then place, of each hub chunk
    int64_t hub_keep_cap = 0;
    int64_t* rrowptr = nullptr;      // [n+1] directed: transposed CSR (in-arcs) of the current graph
    int32_t* rcol = nullptr;         // [rcap]
    int64_t rcap = 0;
    unsigned long long* mode_dmax = nullptr;  // [3] FP32-certified: largest new degree per row mode in a batch
};

// ---- stopping criteria other than top-k (katz_criteria.cu) -------------------
struct RadixBuffers {
    uint64_t* hi[2] = {nullptr, nullptr};
    uint32_t* lo[2] = {nullptr, nullptr};
    int32_t* val[2] = {nullptr, nullptr};
    int64_t* counts = nullptr;  // [256 * radix_tiles(n)]
    int64_t* offs = nullptr;
    int64_t* sums = nullptr;    // scan scratch
};
int64_t radix_tiles(int64_t n);
cudaError_t radix_sort_passes(RadixBuffers& rs, int64_t n, int first, int last, int& cur, cudaStream_t st);
// anchor order of the low-degree rows (internal ids >= start) of a graph
// already renamed into degree-class order; see katz_relabel.cu
cudaError_t locality_order(int64_t n, int64_t nnz, int64_t start, const int64_t* rowptr1, int32_t* col1,
                           int32_t* perm, int32_t* inv, int64_t* deg, int64_t* rowptr_fin, int32_t* tail_copy,
                           int64_t* sums, RadixBuffers& rs, cudaStream_t st);
cudaError_t launch_crit_init(const IterBuffers& b, cudaStream_t st);
cudaError_t launch_score_check(const IterBuffers& b, const IterParams& p, cudaStream_t st);
cudaError_t launch_pair_check(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int32_t oa, int32_t ob,
                              cudaStream_t st);
cudaError_t launch_ranking_check(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, RadixBuffers& rs,
                                 int32_t* rank_ids, cudaStream_t st);
cudaError_t launch_finalize_crit(const IterBuffers& b, const IterParams& p, cudaStream_t st);

cudaError_t dyn_validate(const DeviceGraph& g, const DynBuffers& d, int64_t m, int64_t D, cudaStream_t st);
cudaError_t dyn_clear(const DeviceGraph& g, const DynBuffers& d, int64_t m, cudaStream_t st);
cudaError_t dyn_prepare(const DeviceGraph& g, const DynBuffers& d, int64_t m, int64_t* rowptr_new, int64_t* deg,
                        int64_t* sums, cudaStream_t st);
cudaError_t dyn_rebuild(const DeviceGraph& g, const DynBuffers& d, int64_t m, const int64_t* rowptr_new,
                        int32_t* col_new, void* rowptr_out, bool out64, cudaStream_t st);
cudaError_t dyn_seed(const DeviceGraph& g, const DynBuffers& d, int64_t m, cudaStream_t st);
cudaError_t dyn_expand(const DeviceGraph& g, const DynBuffers& d, int64_t lo, int64_t hi, int level,
                       cudaStream_t st);
cudaError_t dyn_transpose(const DeviceGraph& g, const DynBuffers& d, int64_t* cnt, int64_t* sums, cudaStream_t st);
cudaError_t dyn_recompute_c(const DeviceGraph& g, const IterBuffers& b, const DynBuffers& d, const IterParams& p,
                            int r, bool all, cudaStream_t st);
cudaError_t dyn_reactivate(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int r, cudaStream_t st);
cudaError_t dyn_mode_degree_max(const DeviceGraph& g, const DynBuffers& d, int64_t m, const int64_t* rp_new,
                                cudaStream_t st);

cudaError_t prepare_kernels();  // one-time function attributes (outside any capture)
SpmvLayout make_layout(int64_t n, int64_t row_warp, int64_t row_octet, int64_t row_thread, int64_t chunks);
// create-time relabelling (katz_relabel.cu)
int relabel_blocks(int64_t n);
int64_t scan_blocks(int64_t n);
int degree_class_host(int64_t d);
// stable counting sort of the ids by degree class; scratch: relabel_scratch(n) int64
int64_t relabel_scratch(int64_t n);
cudaError_t relabel_by_degree_class(const int64_t* rowptr64, int64_t n, int64_t* scratch, int32_t* perm, int32_t* inv,
                                    uint64_t* class_start_dev, cudaStream_t st);
// in-degrees of a CSR's columns (cnt: n int64, zero on entry)
cudaError_t launch_indegree(const int32_t* col, int64_t nnz, int64_t* cnt, cudaStream_t st);
// the reverse graph of a validated CSR (int64 offsets): rowptr_rev[n+1],
// col_rev[nnz]; the order inside a reverse row is unspecified; cnt: n+1
// int64 of scratch, sums: scan_blocks(n+1)
cudaError_t reverse_csr(const int64_t* rowptr, const int32_t* col, int64_t n, int64_t nnz, int64_t* cnt,
                        int64_t* sums, int64_t* rowptr_rev, int32_t* col_rev, cudaStream_t st);
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t n, int64_t* out, int64_t* sums_scratch, cudaStream_t st);
// new row offsets (int64, n+1) of the relabelled adjacency
cudaError_t relabel_offsets(const int64_t* rowptr64, const int32_t* perm, int64_t n, int64_t* deg_new_scratch,
                            int64_t* rowptr_new, int64_t* sums_scratch, cudaStream_t st);
// arcs of the original rows [v0, v1) that do not become CHUNK rows, renamed
// into their new rows; then those of the CHUNK rows among them, chunk by chunk
cudaError_t remap_src_rows(const int64_t* rowptr64, const int32_t* col, const int32_t* inv, const int64_t* rowptr_new,
                           int64_t v0, int64_t v1, int64_t n, int64_t row_warp, int32_t* col_new,
                           unsigned long long* bad, cudaStream_t st);
cudaError_t remap_hub_chunks(const int64_t* rowptr64, const int32_t* col, const int32_t* perm, const int32_t* inv,
                             const int64_t* rowptr_new, const int32_t* chunk_row, const int64_t* chunk_first,
                             int64_t row_warp, int64_t chunks_cap, int64_t v0, int64_t v1, int64_t n,
                             int32_t* col_new, unsigned long long* bad, cudaStream_t st);
// chunk table of the CHUNK rows from the new offsets: chunk_first (row_warp + 1
// entries, exclusive scan of the chunk counts), chunk_row, and the largest count
cudaError_t build_chunk_table(const int64_t* rowptr_new, int64_t row_warp, int64_t* cnt_scratch, int64_t* sums_scratch,
                              int64_t* chunk_first, int32_t* chunk_row, unsigned long long* max_chunks,
                              cudaStream_t st);
cudaError_t launch_validate_csr(const DeviceGraph& g, unsigned long long* d_bad, int64_t* d_degmax,
                                cudaStream_t st);
cudaError_t launch_init_walk(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, bool fp32,
                             cudaStream_t st);
// theta_0 from the kk-th largest degree among rows [a, bend) of one exact
// degree class (degrees in (lo, lo + 2^bits])
cudaError_t launch_theta0_class(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int64_t a,
                                int64_t bend, int64_t lo, int bits, int64_t kk, cudaStream_t st);
// Top bin of the degree histogram of theta_0: degrees above it count in it,
// which can only lower theta_0 (still a valid threshold), and the histogram
// stays small whatever degree bound a handle is given.
inline int64_t deg_hist_top(int64_t D) { return D < ((int64_t)1 << 24) ? D : ((int64_t)1 << 24); }
cudaError_t launch_theta0(const DeviceGraph& g, const IterBuffers& b, const IterParams& p,
                          uint32_t* d_deghist, int64_t D, cudaStream_t st);
// the FP32-certified levels' binary64 -> binary32 rounding and exact widening
cudaError_t launch_convert(const double* in, int64_t n, float* out, double* back, cudaStream_t st);
// s_1 = alpha deg into its walk slot, nothing else (a full level 1 of a repair)
cudaError_t launch_degree_store(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, cudaStream_t st);
// level 1 of a ranking (s_1 = alpha deg) in one pass over the rows, fixup included
cudaError_t launch_degree_level(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, cudaStream_t st);
cudaError_t launch_spmv(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, bool fp32,
                        cudaStream_t st);
cudaError_t launch_spmv_store(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int level,
                              cudaStream_t st);
// s_level recomputed for the listed rows (CHUNK rows excepted) and for the
// CHUNK rows whose visit bit is set, with the lane partition of the SpMV
cudaError_t launch_pair_levels(const DeviceGraph& ga, const DeviceGraph& gb, const int32_t* bsrc,
                               const int32_t* bdst, int64_t m, const IterParams& p, int r, int f32_from,
                               int t_level, double* P, int64_t pstride, float* t_pair, double* part,
                               uint32_t* vbits, int32_t* rows, unsigned long long* nrows, cudaStream_t st);
cudaError_t launch_pair_split(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int r, int f32_from,
                              int state, const double* P, int64_t pstride, const float* t_pair, cudaStream_t st);
cudaError_t launch_rows_store(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, const int32_t* rows,
                              const unsigned long long* nrows_dev, int64_t nrows_max, const uint32_t* vbits,
                              int level, cudaStream_t st);
cudaError_t launch_select(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, const double* cl,
                          const double* cu, const int32_t* cid, bool fp32, cudaStream_t st);
cudaError_t launch_count(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, bool fp32,
                         cudaStream_t st);
cudaError_t launch_finalize(const IterBuffers& b, const IterParams& p, cudaStream_t st);
// outputs in original vertex order
cudaError_t launch_bounds_out(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int level, bool fp32,
                              double* lower, double* upper, double* err, cudaStream_t st);
cudaError_t launch_cert_init(const IterBuffers& b, const IterParams& p, cudaStream_t st);
cudaError_t launch_cert_replay(const IterBuffers& b, const IterParams& p, int r, cudaStream_t st);
int max_sum_depth(const SpmvLayout& L, int64_t max_chunks_per_row);
int sum_depth_of(int64_t deg_thread, int64_t deg_octet, int64_t deg_warp, bool has_octet, bool has_warp,
                 int64_t max_chunks_per_row);
cudaError_t launch_walk_out(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int level, bool fp32,
                            double* out, cudaStream_t st);
// radix select over candidates (large candidate sets): one pass of 8-bit digits


}  // namespace katz
