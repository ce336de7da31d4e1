// The opaque katz_handle behind include/katz.h (host-side state).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "katz_common.cuh"

struct katz_handle {
    katz_opts opts;
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool fp32 = false;
    katz::DeviceGraph g;
    int64_t deg_max = 0;
    int64_t D = 0;  // degree bound used for gamma
    int sum_depth = 1;   // longest addition chain of one SpMV row sum
    // first internal id of each degree class of the relabelling; exact until
    // an update batch changes degrees (theta_0 then falls back to a histogram)
    uint64_t cls_start[katz::NUM_CLASSES] = {};
    bool classes_exact = false;
    int f32_from = 0x7fffffff;  // first FP32 level of the last ranking
    katz::IterBuffers b;
    katz::IterParams p{};
    int walk_slots = 0;
    size_t walk_esz = 0;
    int64_t stride = 0;
    // scratch
    uint32_t* d_deghist = nullptr;
    double* d_scratch = nullptr;
    katz::Ctrl* h_ctrl = nullptr;  // pinned (one block with h_small)
    unsigned char* h_small = nullptr;  // pinned scratch of H_SMALL bytes for small device-to-host reads
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // profiling: one event pair per SpMV launch
    std::vector<cudaEvent_t> sp_ev;
    int64_t launches = 0;   // kernels launched by the current call (host-counted part)
    // CUDA graph of one iteration inside a device-side while loop
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    katz::IterParams graph_params{};
    bool graph_fp32 = false;
    // dynamic updates
    katz::DynBuffers dyn;
    int32_t* col_spare = nullptr;     // rebuilt col is written here, then swapped
    int64_t col_spare_cap = 0;
    int64_t col_cap = 0;              // capacity of g.col
    int64_t* rp_new = nullptr;        // [n+1]
    int64_t* deg_tmp = nullptr;       // [n+1]
    int64_t* scan_sums = nullptr;
    // Updates in two phases (katz_api.cu): prepare validates a batch against
    // the current graph and builds the next graph into the spare buffers on
    // stream_a; commit swaps them in and repairs on stream.  The server runs
    // the prepare of batch j+1 while batch j is repaired.
    cudaStream_t stream_a = nullptr;
    cudaEvent_t ev_prepared = nullptr;   // stream_a: the prepared graph is complete
    cudaEvent_t ev_committed = nullptr;  // stream: work on the previous graph is queued before this
    void* rowptr_spare = nullptr;        // [n+1], the offset type of g.rowptr
    // a batch that takes n + nnz past the int32 offset range: the new int64
    // offsets and the int64 spare that replace the two int32 arrays at its swap
    int64_t* rp64_next = nullptr;
    int64_t* rp64_spare_next = nullptr;
    int64_t* chunk_first_spare = nullptr;  // [row_warp+1]
    int32_t* chunk_row_spare = nullptr;
    int64_t chunk_row_cap = 0, chunk_row_spare_cap = 0, chunk_part_cap = 0;  // in chunks
    int32_t* bsrc[2] = {nullptr, nullptr};  // batch arrays, one set per phase in flight
    int32_t* bdst[2] = {nullptr, nullptr};
    uint8_t* bins[2] = {nullptr, nullptr};
    int64_t bcap = 0;
    int next_bset = 0;
    int64_t* t_cnt = nullptr;   // [n+1] transposition scratch of the repair (directed)
    int64_t* t_sums = nullptr;
    struct Pending {
        bool ready = false;
        katz_status status = KATZ_OK;
        std::string err;
        int64_t m = 0, nnz = 0, chunks = 0, launches = 0;
        int bset = 0;
        int depth = 0;          // FP32-certified: summation depth the updated rows need (0: not computed)
        bool applied = false;   // the batch changed the graph (m > 0 and valid)
        bool promote = false;   // the updated graph needs int64 row offsets (rp64_next)
    } pend;                     // written by the prepare
    Pending rep;                // the swapped-in batch, read by its repair
    // two-state pass (update_pair_levels): interleaved levels of the two
    // graph states, their FP32 roundings and the chunk partials of both
    double* pair_P = nullptr;
    size_t pair_P_cap = 0;      // doubles
    float* pair_t = nullptr;    // [2n]
    double* pair_part = nullptr;
    int64_t pair_part_cap = 0;  // doubles
    int pair_r = -1;            // r of the levels in pair_P (-1: none pending for the second state)
    int pair_f32_from = 0;      // the first FP32 level those levels used
    bool last_repair_whole = false;  // the last repair recomputed whole levels
    bool pair_second_used = false;   // update_pair_second finished from the two-state pass
    int64_t* rrowptr = nullptr; // [n+1] directed: transposed CSR of the current graph (the repair's)
    int32_t* rcol = nullptr;
    int64_t rcap = 0;
    // stopping criteria other than top-k
    int criterion = KATZ_CRIT_TOPK;
    int32_t* rank_ids = nullptr;      // [n] ranking criterion: the order, original ids
    katz::RadixBuffers rs;
    // result of the last rank/update call
    bool ranked = false;
    int r = 0;
    int converged = 0;
    int64_t k_eff = 0;
    double alpha = 0, gamma = 0, eps = 0;
    float last_ms = 0.f;
    std::vector<int64_t> trace;
    std::string err;
    // katz_submit_update_batch / katz_poll: a private serving queue, made at
    // the first submitted batch
    std::mutex async_mu;
    katz_server* async = nullptr;
};

namespace katz {
// the context's maximum L2 fetch granularity for the duration of one call
// (katz_opts.l2_fetch_bytes > 0), set back to the reported value afterwards
class L2FetchScope {
  public:
    explicit L2FetchScope(const katz_handle* h);
    ~L2FetchScope();
    L2FetchScope(const L2FetchScope&) = delete;
    L2FetchScope& operator=(const L2FetchScope&) = delete;

  private:
    size_t prev_ = 0;
    bool set_ = false;
};

constexpr size_t CTRL_BYTES = (sizeof(Ctrl) + 255) / 256 * 256;
constexpr size_t H_SMALL = 4096;

cudaMemPool_t library_pool(int dev);

// count elements of X from the library's pool, ordered on the handle's stream
template <typename X>
cudaError_t dmalloc(katz_handle* h, X** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaMemPool_t pool = library_pool(h->dev);
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync((void**)p, count * sizeof(X), pool, h->stream);
}

inline void dfree(katz_handle* h, void* p) {
    if (p) cudaFreeAsync(p, h->stream);
}

// the same, ordered on stream st instead of the handle's stream
template <typename X>
cudaError_t dmalloc_on(katz_handle* h, X** p, size_t count, cudaStream_t st) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaMemPool_t pool = library_pool(h->dev);
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync((void**)p, count * sizeof(X), pool, st);
}

inline void dfree_on(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

katz_status init_handle_runtime(katz_handle* h);
katz_status ensure_iter_buffers(katz_handle* h);
katz_status alloc_rank_scratch(katz_handle* h);
katz_status fail(katz_handle* h, katz_status s, const std::string& msg);
katz_status cuda_fail(katz_handle* h, cudaError_t e, const char* what);
bool is_device_ptr(const void* p);
void drop_graph(katz_handle* h);
cudaError_t launch_narrow_rowptr(const int64_t* in, int32_t* out, int64_t count, cudaStream_t st);
katz_status dyn_reserve(katz_handle* h, int64_t m, int64_t nnz_cap, cudaStream_t st);
katz_status update_allowed(katz_handle* h);
// Algorithm 2 in phases: prepare (stream_a; ready: an event the batch arrays
// wait for, or nullptr), then swap and repair (the handle's stream).  At most
// one prepared batch waits for its swap; a prepare reads the graph the
// latest swap made current.
katz_status update_prepare(katz_handle* h, const int32_t* src, const int32_t* dst, const uint8_t* is_insert,
                           int64_t m, cudaEvent_t ready);
katz_status update_swap(katz_handle* h);
katz_status update_repair(katz_handle* h, katz_info* info);
katz_status update_commit(katz_handle* h, katz_info* info);
// Two batches in one pass: after the first batch's swap (h->rep) and the
// second batch's prepare on top of it (h->pend), pair_possible says whether
// the pass applies; update_pair_first computes the levels of both graph
// states and finishes the first batch (its ranking is then current);
// update_pair_second swaps the second batch in and finishes it from the same
// pass, or repairs it alone when the first one changed r or the precision.
bool pair_possible(katz_handle* h);
katz_status update_pair_first(katz_handle* h, katz_info* info);
katz_status update_pair_second(katz_handle* h, katz_info* info);
}  // namespace katz
