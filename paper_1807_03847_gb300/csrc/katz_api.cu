// C-ABI entry points (include/katz.h): handle lifecycle, the driver of
// Algorithm 1's loop and the getters.  All arithmetic of the method runs in
// the kernels of katz_kernels.cu; this file only allocates, launches and
// copies.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "katz_common.cuh"
#include "katz_handle.h"

using namespace katz;

namespace {

const char* kStatusNames[] = {"KATZ_OK",     "KATZ_EINVAL",     "KATZ_EALPHA",   "KATZ_ENOMEM",
                              "KATZ_ECUDA",  "KATZ_ENOTCONV",   "KATZ_EPRECISION", "KATZ_ETIMEOUT",
                              "KATZ_EBUSY",  "KATZ_ESTATE"};

}  // namespace

namespace katz {

katz_status fail(katz_handle* h, katz_status s, const std::string& msg) {
    if (h) h->err = msg;
    return s;
}

katz_status cuda_fail(katz_handle* h, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (h) h->err = m;
    return e == cudaErrorMemoryAllocation ? KATZ_ENOMEM : KATZ_ECUDA;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory of the handles comes from one stream-ordered pool per
// device that the library keeps for the life of the process (no release
// threshold): destroying a handle returns its memory to the pool without a
// device-wide synchronisation, and the next handle reuses it.
cudaMemPool_t library_pool(int dev) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&pools[dev], &props) != cudaSuccess) {
            pools[dev] = nullptr;
            return nullptr;
        }
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    return pools[dev];
}

// The device, stream, events and pinned host block of a new handle.
katz_status init_handle_runtime(katz_handle* h) {
    cudaError_t e;
    if ((e = cudaGetDevice(&h->dev)) != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
    if ((e = prepare_kernels()) != cudaSuccess) return cuda_fail(h, e, "prepare kernels");
    if (h->opts.cuda_stream) {
        h->stream = (cudaStream_t)h->opts.cuda_stream;
        h->own_stream = false;
    } else {
        if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(h, e, "cudaStreamCreate");
        h->own_stream = true;
    }
    if ((e = cudaEventCreate(&h->ev0)) != cudaSuccess || (e = cudaEventCreate(&h->ev1)) != cudaSuccess)
        return cuda_fail(h, e, "cudaEventCreate");
    // one pinned block: the control block, then a small scratch for device-to-host reads
    void* blk = nullptr;
    if ((e = cudaMallocHost(&blk, CTRL_BYTES + H_SMALL)) != cudaSuccess) return cuda_fail(h, e, "cudaMallocHost");
    h->h_ctrl = (Ctrl*)blk;
    h->h_small = (unsigned char*)blk + CTRL_BYTES;
    return KATZ_OK;
}

// Scratch of the ranking loop that does not depend on the ranking's size.
katz_status alloc_rank_scratch(katz_handle* h) {
    cudaError_t e;
    if ((e = dmalloc(h, &h->d_deghist, (size_t)deg_hist_top(h->D) + 1)) != cudaSuccess)
        return cuda_fail(h, e, "cudaMalloc rank scratch");
    return KATZ_OK;
}

void free_iter(katz_handle* h) {
    IterBuffers& b = h->b;
    dfree(h, b.walk);
    dfree(h, b.c);
    dfree(h, b.c32);
    dfree(h, b.lb);
    dfree(h, b.ub);
    dfree(h, b.active);
    dfree(h, b.s32);
    dfree(h, b.alist[0]);
    dfree(h, b.alist[1]);
    dfree(h, b.cand_l);
    dfree(h, b.cand_u);
    dfree(h, b.cand_id);
    dfree(h, b.topk_id);
    dfree(h, b.topk_l);
    dfree(h, b.topk_u);
    dfree(h, b.trace);
    dfree(h, b.ctrl);
    b = IterBuffers();
    h->walk_slots = 0;
}

// (Re)allocate the per-iteration buffers for the handle's precision,
// history setting and r_max.
katz_status ensure_iter_buffers(katz_handle* h) {
    const int slots = h->opts.keep_history ? h->opts.r_max + 1 : 2;
    const size_t esz = sizeof(double);  // slots hold FP64 levels (an FP32 level uses half a slot)
    if (h->b.walk && h->walk_slots == slots && h->walk_esz == esz) return KATZ_OK;
    free_iter(h);
    IterBuffers& b = h->b;
    const int64_t n = h->g.n;
    const int64_t stride = ((n + 1) + 31) / 32 * 32;
    cudaError_t e;
#define KALLOC(ptr, cnt)                                          \
    if ((e = dmalloc(h, &(ptr), (size_t)(cnt))) != cudaSuccess) {    \
        free_iter(h);                                             \
        return cuda_fail(h, e, "cudaMalloc " #ptr);               \
    }
    char* walk = nullptr;
    KALLOC(walk, (size_t)slots * stride * esz);
    b.walk = walk;
    KALLOC(b.c, n);
    KALLOC(b.lb, n);  // bounds of the active nodes at the last level (cert mode: monotone)
    KALLOC(b.ub, n);
    if (h->fp32) KALLOC(b.c32, n);
    if (h->fp32) KALLOC(b.s32, n);
    KALLOC(b.active, n);
    KALLOC(b.alist[0], n);
    KALLOC(b.alist[1], n);
    KALLOC(b.cand_l, n);
    KALLOC(b.cand_u, n);
    KALLOC(b.cand_id, n);
    KALLOC(b.topk_id, KATZ_MAX_K);
    KALLOC(b.topk_l, KATZ_MAX_K);
    KALLOC(b.topk_u, KATZ_MAX_K);
    KALLOC(b.trace, h->opts.r_max + 2);
    KALLOC(b.ctrl, 1);
#undef KALLOC
    b.cand_cap = n;
    h->walk_slots = slots;
    h->walk_esz = esz;
    h->stride = stride;
    return KATZ_OK;
}

// One iteration of Algorithm 1 (five kernels, no host synchronisation).
// ev_pair: optional events recorded around the SpMV launch.
cudaError_t launch_iteration(katz_handle* h, cudaEvent_t* ev_pair = nullptr) {
    cudaError_t e;
    if (ev_pair && (e = cudaEventRecord(ev_pair[0], h->stream)) != cudaSuccess) return e;
    if ((e = launch_spmv(h->g, h->b, h->p, h->fp32, h->stream)) != cudaSuccess) return e;
    if (ev_pair && (e = cudaEventRecord(ev_pair[1], h->stream)) != cudaSuccess) return e;
    if ((e = launch_select(h->g, h->b, h->p, h->b.cand_l, h->b.cand_u, h->b.cand_id, h->fp32, h->stream)) != cudaSuccess)
        return e;
    if ((e = launch_count(h->g, h->b, h->p, h->fp32, h->stream)) != cudaSuccess) return e;
    return launch_finalize(h->b, h->p, h->stream);
}

// The first iteration of a ranking: level 1 is the degree vector (s_0 = 1,
// A 1 = deg), one O(n) pass instead of a gather level; then the same check.
cudaError_t launch_first_iteration(katz_handle* h, cudaEvent_t* ev_pair = nullptr) {
    cudaError_t e;
    if (ev_pair && (e = cudaEventRecord(ev_pair[0], h->stream)) != cudaSuccess) return e;
    if ((e = launch_degree_level(h->g, h->b, h->p, h->stream)) != cudaSuccess) return e;
    if (ev_pair && (e = cudaEventRecord(ev_pair[1], h->stream)) != cudaSuccess) return e;
    if ((e = launch_select(h->g, h->b, h->p, h->b.cand_l, h->b.cand_u, h->b.cand_id, h->fp32, h->stream)) != cudaSuccess)
        return e;
    if ((e = launch_count(h->g, h->b, h->p, h->fp32, h->stream)) != cudaSuccess) return e;
    return launch_finalize(h->b, h->p, h->stream);
}

bool same_params(const IterParams& a, const IterParams& b) { return std::memcmp(&a, &b, sizeof(a)) == 0; }

void drop_graph(katz_handle* h) {
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->graph_exec = nullptr;
    h->graph = nullptr;
}

// Capture one iteration as the body of a conditional while node; the
// finalize kernel clears the condition once converged() holds or r_max is hit.
katz_status ensure_graph(katz_handle* h) {
    if (h->graph_exec && same_params(h->graph_params, h->p) && h->graph_fp32 == h->fp32) return KATZ_OK;
    drop_graph(h);
    cudaError_t e;
    cudaGraph_t graph = nullptr;
    if ((e = cudaGraphCreate(&graph, 0)) != cudaSuccess) return cuda_fail(h, e, "cudaGraphCreate");
    cudaGraphConditionalHandle cond;
    if ((e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(h, e, "cudaGraphConditionalHandleCreate");
    }
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(h, e, "cudaGraphAddNode(conditional)");
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    h->b.cond_handle = (unsigned long long)cond;
    h->b.use_cond = 1;
    e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e2 = launch_iteration(h);
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(h->stream, &out);
        if (e2 != cudaSuccess) e = e2;
    }
    h->b.use_cond = 0;
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(h, e, "capture iteration");
    }
    if ((e = cudaGraphInstantiate(&h->graph_exec, graph, 0)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(h, e, "cudaGraphInstantiate");
    }
    h->graph = graph;
    h->graph_params = h->p;
    h->graph_fp32 = h->fp32;
    return KATZ_OK;
}

// Run iterations until the device sets ctrl.stop (converged or r_max).
// Graph mode: one graph launch runs the whole loop on the device; the host
// only steps in when the candidate set outgrows the one-CTA select.
// Host mode: iterations are launched in batches and ctrl is read between
// batches (launches after a stop return at once).  done: iterations already
// enqueued by the caller (profile events of the loop's launches follow theirs).
// one pair of timing events per iteration up to r_max (profile mode)
katz_status ensure_prof_events(katz_handle* h) {
    cudaError_t e;
    if (h->sp_ev.size() < 2 * (size_t)(h->opts.r_max + 8)) {
        for (cudaEvent_t ev : h->sp_ev) cudaEventDestroy(ev);
        h->sp_ev.assign(2 * (size_t)(h->opts.r_max + 8), nullptr);
        for (auto& ev : h->sp_ev)
            if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate");
    }
    return KATZ_OK;
}

katz_status run_loop(katz_handle* h, int done) {
    cudaError_t e;
    const bool graph_mode = h->opts.use_graph && !h->opts.profile;
    const bool prof = h->opts.profile != 0;
    const int batch = 4;
    if (prof) {
        const katz_status s = ensure_prof_events(h);
        if (s != KATZ_OK) return s;
    }
    if (graph_mode) {
        katz_status s = ensure_graph(h);
        if (s != KATZ_OK) return s;
    }
    int launched_iters = done;
    for (;;) {
        if (graph_mode) {
            if ((e = cudaGraphLaunch(h->graph_exec, h->stream)) != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
        } else {
            for (int q = 0; q < batch; ++q) {
                cudaEvent_t* ev = nullptr;
                if (prof && 2 * launched_iters + 1 < (int)h->sp_ev.size()) ev = &h->sp_ev[2 * launched_iters];
                if ((e = launch_iteration(h, ev)) != cudaSuccess) return cuda_fail(h, e, "launch iteration");
                h->launches += (h->g.layout.row_warp > 0 ? 5 : 4);
                ++launched_iters;
            }
        }
        if ((e = cudaMemcpyAsync(h->h_ctrl, h->b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
            return cuda_fail(h, e, "copy ctrl");
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(h, e, "iteration");
        if (h->h_ctrl->stop) return KATZ_OK;
    }
}

}  // namespace katz

namespace katz {

// Device buffers of the dynamic path for batches of up to m updates and a
// rebuilt adjacency of up to nnz_cap arcs (0: no spare adjacency yet).  A
// batch within these sizes allocates and frees nothing.
// alpha (Sec. 3.1: 1 / (D + 1) when not given), gamma of Theorem 1 and the
// iteration parameters of a ranking; the iteration buffers
// katz_opts.l2_fetch_bytes: the context's maximum L2 fetch granularity for
// the duration of one call, set back to the reported value afterwards.  A
// random gather that misses L2 moves a whole fetch unit from DRAM; with a
// walk vector far larger than L2 most of each unit is not used.
L2FetchScope::L2FetchScope(const katz_handle* h) {
    const int want = h->opts.l2_fetch_bytes;
    if (want <= 0) return;
    if (cudaDeviceGetLimit(&prev_, cudaLimitMaxL2FetchGranularity) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)want) == cudaSuccess) set_ = true;
    else cudaGetLastError();
}

L2FetchScope::~L2FetchScope() {
    if (set_ && cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, prev_) != cudaSuccess) cudaGetLastError();
}

katz_status setup_ranking(katz_handle* h, double alpha, int64_t k_eff, double eps, double& a, double& gamma) {
    const double D = (double)h->D;
    a = alpha > 0.0 ? alpha : 1.0 / (D + 1.0);
    if (!(a * D < 1.0)) return fail(h, KATZ_EALPHA, "alpha * deg_bound >= 1");
    katz_status st = ensure_iter_buffers(h);
    if (st != KATZ_OK) return st;
    gamma = D / (1.0 - a * D);
    IterParams& p = h->p;
    p.alpha = a;
    p.ag = a * gamma;
    p.eps = eps;
    p.n = h->g.n;
    p.k = k_eff;
    p.stride = h->stride;
    p.slots = h->walk_slots;
    p.undirected = h->opts.undirected ? 1 : 0;
    p.r_max = h->opts.r_max;
    p.cert = h->fp32 ? 1 : 0;
    {  // an upper bound of alpha * gamma: four ulps above the rounded product
        double ag_hi = p.ag;
        for (int q = 0; q < 4; ++q) ag_hi = std::nextafter(ag_hi, INFINITY);
        p.ag_hi = ag_hi;
    }
    p.alpha_f = (float)a;
    p.depth = h->sum_depth;
    p.fp32_from = h->fp32 ? std::max(0, h->opts.fp32_from) : 0;
    return KATZ_OK;
}

katz_status dyn_reserve(katz_handle* h, int64_t m, int64_t nnz_cap, cudaStream_t st) {
    cudaError_t e;
    DeviceGraph& g = h->g;
    DynBuffers& d = h->dyn;
    const int64_t n = g.n;
#define DALLOC(ptr, cnt)                                                      \
    if ((e = dmalloc_on(h, &(ptr), (size_t)(cnt), st)) != cudaSuccess) return cuda_fail(h, e, "cudaMalloc " #ptr);
    if (!h->stream_a) {
        if ((e = cudaStreamCreateWithFlags(&h->stream_a, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->ev_prepared, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->ev_committed, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(h, e, "update stream");
    }
    if (!d.delta) {
        DALLOC(d.delta, n);
        DALLOC(d.ins_cnt, n);
        DALLOC(d.cursor, n);
        DALLOC(d.touched, (n + 3) / 4 * 4);  // whole words: rows are claimed with word atomics
        DALLOC(d.ins_start, n);
        DALLOC(d.vbits, (n + 31) / 32);
        DALLOC(d.frontier, n);
        DALLOC(d.fsize, 2);
        DALLOC(d.hub_epoch, std::max<int64_t>(g.layout.row_warp, 1));
        DALLOC(d.n_ins_rows, 1);
        DALLOC(d.err, 1);
        DALLOC(d.mode_dmax, 3);
        DALLOC(h->rp_new, n + 1);
        DALLOC(h->deg_tmp, n + 1);
        DALLOC(h->scan_sums, scan_blocks(n + 1));
        if (g.off64) {
            int64_t* rp = nullptr;
            DALLOC(rp, n + 1);
            h->rowptr_spare = rp;
        } else {
            int32_t* rp = nullptr;
            DALLOC(rp, n + 1);
            h->rowptr_spare = rp;
        }
        DALLOC(h->chunk_first_spare, g.layout.row_warp + 1);
        DALLOC(h->chunk_row_spare, std::max<int64_t>(h->chunk_row_cap, 1));
        h->chunk_row_spare_cap = std::max<int64_t>(h->chunk_row_cap, 1);
        if ((e = cudaMemsetAsync(d.delta, 0, (size_t)n * sizeof(int32_t), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(d.ins_cnt, 0, (size_t)n * sizeof(int32_t), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(d.cursor, 0, (size_t)n * sizeof(int32_t), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(d.touched, 0, (size_t)((n + 3) / 4 * 4), st)) != cudaSuccess)
            return cuda_fail(h, e, "memset dynamic scratch");
        h->col_cap = g.nnz;
    }
    if (m > h->bcap) {  // both batch sets (called before any batch is in flight, or for the first one)
        for (int q = 0; q < 2; ++q) {
            dfree_on(h->bsrc[q], st);
            dfree_on(h->bdst[q], st);
            dfree_on(h->bins[q], st);
            h->bsrc[q] = nullptr;
            h->bdst[q] = nullptr;
            h->bins[q] = nullptr;
        }
        h->bcap = 0;
        const int64_t cap = std::max<int64_t>(m, 1024);
        for (int q = 0; q < 2; ++q) {
            DALLOC(h->bsrc[q], cap);
            DALLOC(h->bdst[q], cap);
            DALLOC(h->bins[q], cap);
        }
        h->bcap = cap;
    }
    if (m > d.cap) {
        dfree_on(d.ins_rows, st);
        dfree_on(d.bucket, st);
        dfree_on(d.table, st);
        d.ins_rows = nullptr;
        d.bucket = nullptr;
        d.table = nullptr;
        d.table_mask = 0;
        d.cap = 0;
        const int64_t cap = std::max<int64_t>(m, 1024);
        DALLOC(d.ins_rows, 2 * cap);
        DALLOC(d.bucket, 2 * cap);
        int64_t tsize = 1;
        while (tsize < 4 * cap) tsize <<= 1;
        DALLOC(d.table, tsize);
        d.table_mask = tsize - 1;
        d.cap = cap;
        if ((e = cudaMemsetAsync(d.table, 0, (size_t)tsize * sizeof(unsigned long long), st)) != cudaSuccess)
            return cuda_fail(h, e, "memset table");
    }
    if (nnz_cap > h->col_spare_cap) {
        dfree_on(h->col_spare, st);
        h->col_spare = nullptr;
        h->col_spare_cap = 0;
        DALLOC(h->col_spare, nnz_cap);
        h->col_spare_cap = nnz_cap;
    }
#undef DALLOC
    return KATZ_OK;
}

}  // namespace katz

namespace katz {

// The reverse graph of the input CSR (host or device pointers) into
// h->rp_new (n+1 int64) and h->col_spare (nnz), after checking the input in
// full (offsets and column range), which the scatter needs.
katz_status reverse_input(katz_handle* h, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col) {
    cudaError_t e = cudaSuccess;
    int64_t *rp_in = nullptr, *cnt = nullptr, *sums = nullptr, *d_degmax = nullptr;
    int32_t* col_in = nullptr;
    unsigned long long* d_bad = nullptr;
    const bool copy_rp = !is_device_ptr(rowptr), copy_col = nnz > 0 && !is_device_ptr(col);
    auto A = [&](auto** p, size_t count) {
        if (e == cudaSuccess) e = dmalloc(h, p, count);
    };
    if (copy_rp) A(&rp_in, (size_t)n + 1);
    if (copy_col) A(&col_in, (size_t)nnz);
    A(&cnt, (size_t)n + 1);
    A(&sums, (size_t)scan_blocks(n + 1));
    A(&d_bad, 1);
    A(&d_degmax, 1);
    A(&h->rp_new, (size_t)n + 1);
    A(&h->col_spare, (size_t)nnz);
    katz_status st = KATZ_OK;
    if (e == cudaSuccess) {
        h->col_spare_cap = std::max<int64_t>(nnz, 1);
        const int64_t* rp = copy_rp ? rp_in : rowptr;
        const int32_t* cl = copy_col ? col_in : col;
        if (copy_rp) e = cudaMemcpyAsync(rp_in, rowptr, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyDefault, h->stream);
        if (e == cudaSuccess && copy_col)
            e = cudaMemcpyAsync(col_in, col, (size_t)nnz * sizeof(int32_t), cudaMemcpyDefault, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_degmax, 0, sizeof(int64_t), h->stream);
        DeviceGraph gin;
        gin.n = n;
        gin.nnz = nnz;
        gin.off64 = true;
        gin.rowptr = (void*)rp;
        gin.col = (int32_t*)cl;
        if (e == cudaSuccess) e = launch_validate_csr(gin, d_bad, d_degmax, h->stream);
        unsigned long long* bad = (unsigned long long*)h->h_small;
        if (e == cudaSuccess) e = cudaMemcpyAsync(bad, d_bad, sizeof(*bad), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess && *bad) st = KATZ_EINVAL;
        if (e == cudaSuccess && st == KATZ_OK)
            e = reverse_csr(rp, cl, n, nnz, cnt, sums, h->rp_new, h->col_spare, h->stream);
    }
    for (void* p : {(void*)rp_in, (void*)col_in, (void*)cnt, (void*)sums, (void*)d_bad, (void*)d_degmax}) dfree(h, p);
    if (e != cudaSuccess) return cuda_fail(h, e, "reverse graph");
    return st;
}

}  // namespace katz

extern "C" {

katz_status katz_convert_f64_f32(const double* in, int64_t n, float* out, double* back) {
    if (n < 0 || (n > 0 && (!in || !out || !back))) return KATZ_EINVAL;
    if (n > 0 && (!is_device_ptr(in) || !is_device_ptr(out) || !is_device_ptr(back))) return KATZ_EINVAL;
    cudaError_t e = launch_convert(in, n, out, back, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    return e == cudaSuccess ? KATZ_OK : KATZ_ECUDA;
}

void katz_default_opts(katz_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = KATZ_FP64;
    o->undirected = 1;
    o->keep_history = 0;
    o->r_max = 128;
    o->deg_bound = 0;
    o->frontier_abort_frac = 0.05;
    o->cuda_stream = nullptr;
    o->use_graph = 1;
    o->inbound = 0;
    o->profile = 0;
    o->fp32_from = 0;
    o->offsets64 = 0;
    o->l2_fetch_bytes = 0;
    o->locality = 0;
}

const char* katz_status_string(katz_status s) {
    const int i = (int)s;
    return (i >= 0 && i < (int)(sizeof(kStatusNames) / sizeof(kStatusNames[0]))) ? kStatusNames[i] : "KATZ_UNKNOWN";
}

const char* katz_last_error(katz_h h) { return h ? h->err.c_str() : "null handle"; }

void katz_destroy(katz_h h) {
    if (!h) return;
    if (h->async) {  // the running batch finishes, queued ones are dropped
        katz_server_destroy(h->async);
        h->async = nullptr;
    }
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_iter(h);
    dfree(h, h->g.rowptr);
    dfree(h, h->g.col);
    dfree(h, h->g.perm);
    dfree(h, h->g.inv);
    dfree(h, h->g.chunk_row);
    dfree(h, h->g.chunk_first);
    dfree(h, h->g.chunk_part);
    dfree(h, h->d_deghist);
    dfree(h, h->d_scratch);
    dfree(h, h->rank_ids);
    dfree(h, h->pair_P);
    dfree(h, h->pair_t);
    dfree(h, h->pair_part);
    for (int q = 0; q < 2; ++q) {
        dfree(h, h->rs.hi[q]);
        dfree(h, h->rs.lo[q]);
        dfree(h, h->rs.val[q]);
    }
    dfree(h, h->rs.counts);
    dfree(h, h->rs.offs);
    dfree(h, h->rs.sums);
    {
        DynBuffers& d = h->dyn;
        for (void* ptr : {(void*)d.src, (void*)d.dst, (void*)d.ins, (void*)d.hub_epoch, (void*)d.table,
                          (void*)d.err, (void*)d.delta, (void*)d.ins_cnt, (void*)d.cursor, (void*)d.touched,
                          (void*)d.ins_start, (void*)d.ins_rows, (void*)d.n_ins_rows, (void*)d.bucket,
                          (void*)d.vbits, (void*)d.frontier, (void*)d.fsize, (void*)h->rrowptr, (void*)h->rcol,
                          (void*)d.hub_keep})
            dfree(h, ptr);
        dfree(h, h->col_spare);
        dfree(h, h->rp_new);
        dfree(h, h->deg_tmp);
        dfree(h, h->scan_sums);
        if (h->stream_a) cudaStreamSynchronize(h->stream_a);
        for (void* ptr : {(void*)h->rowptr_spare, (void*)h->rp64_next, (void*)h->rp64_spare_next,
                          (void*)h->chunk_first_spare, (void*)h->chunk_row_spare,
                          (void*)h->bsrc[0], (void*)h->bsrc[1], (void*)h->bdst[0], (void*)h->bdst[1],
                          (void*)h->bins[0], (void*)h->bins[1], (void*)h->t_cnt, (void*)h->t_sums})
            dfree(h, ptr);
        if (h->ev_prepared) cudaEventDestroy(h->ev_prepared);
        if (h->ev_committed) cudaEventDestroy(h->ev_committed);
        if (h->stream_a) cudaStreamDestroy(h->stream_a);
    }
    cudaFreeHost(h->h_ctrl);
    drop_graph(h);
    for (cudaEvent_t ev : h->sp_ev) cudaEventDestroy(ev);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

katz_status katz_create_csr(katz_h* out, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                            const katz_opts* opts) {
    if (!out) return KATZ_EINVAL;
    *out = nullptr;
    if (n < 1 || n > 0x7ffffffeLL || nnz < 0 || !rowptr || (nnz > 0 && !col)) return KATZ_EINVAL;
    katz_handle* h = new katz_handle();
    katz_default_opts(&h->opts);
    if (opts) h->opts = *opts;
    if (h->opts.r_max < 1) h->opts.r_max = 1;
    if (h->opts.precision != KATZ_FP64 && h->opts.precision != KATZ_FP32_CERT &&
        h->opts.precision != KATZ_FP32_CERT_AUTO) {
        delete h;
        return KATZ_EINVAL;
    }
    h->fp32 = h->opts.precision != KATZ_FP64;
    cudaError_t e;
    katz_status st = KATZ_OK;
#define KCHK(call, what)                       \
    if ((e = (call)) != cudaSuccess) {         \
        st = cuda_fail(h, e, what);            \
        katz_destroy(h);                       \
        return st;                             \
    }
    if ((st = init_handle_runtime(h)) != KATZ_OK) {
        katz_destroy(h);
        return st;
    }
    // inbound Katz of a directed graph is the outbound Katz of its reverse
    // graph (Sec. 2.1): reverse the input on the device and take that as the
    // input (held in rp_new / col_spare until the create has copied it)
    if (h->opts.inbound && !h->opts.undirected) {
        if ((st = reverse_input(h, n, nnz, rowptr, col)) != KATZ_OK) {
            katz_destroy(h);
            return st;
        }
        rowptr = h->rp_new;
        col = h->col_spare;
    }
    DeviceGraph& g = h->g;
    g.n = n;
    g.nnz = nnz;
    g.off64 = (n + nnz) >= 0x7fffffffLL || h->opts.offsets64 != 0;
    // Input: the row offsets are copied first and validated, and the
    // degree-class relabelling (which needs only them) runs while the column
    // array follows on a second stream in slices of rows; each slice is
    // renamed into internal order as soon as it has arrived.
    const bool host_rowptr = !is_device_ptr(rowptr);
    const int slices = (host_rowptr && nnz >= (1 << 22)) ? 8 : 1;
    std::vector<int64_t> vcut((size_t)slices + 1, 0), acut((size_t)slices + 1, 0);
    vcut[slices] = n;
    acut[slices] = nnz;
    for (int i = 1; i < slices; ++i) {  // rows with about nnz / slices arcs each
        const int64_t target = nnz / slices * i;
        int64_t lo = vcut[i - 1], hi = n;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (rowptr[mid] < target) lo = mid + 1;
            else hi = mid;
        }
        vcut[i] = lo;
        // copy ranges come from the offsets as given, made monotone and kept
        // inside [0, nnz], so that every copy stays in bounds even for a
        // malformed CSR (which the device check then rejects)
        acut[i] = std::min<int64_t>(std::max<int64_t>(rowptr[lo], acut[i - 1]), nnz);
    }
    int64_t* rp64 = nullptr;
    int32_t* col0 = nullptr;
    cudaStream_t cs = nullptr;
    std::vector<cudaEvent_t> ev((size_t)slices + 1, nullptr);
    auto drop_staging = [&]() {
        if (cs) cudaStreamSynchronize(cs);  // slices still in flight into col0
        dfree(h, rp64);
        dfree(h, col0);
        rp64 = nullptr;
        col0 = nullptr;
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
        ev.assign(ev.size(), nullptr);
        if (cs) cudaStreamDestroy(cs);
        cs = nullptr;
    };
#define KCHK2(call, what)                      \
    if ((e = (call)) != cudaSuccess) {         \
        drop_staging();                        \
        st = cuda_fail(h, e, what);            \
        katz_destroy(h);                       \
        return st;                             \
    }
    KCHK2(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
    for (int i = 0; i <= slices; ++i) KCHK2(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming), "cudaEventCreate");
    KCHK2(dmalloc(h, &rp64, (size_t)n + 1), "cudaMalloc rowptr");
    KCHK2(dmalloc(h, &col0, (size_t)nnz), "cudaMalloc col");
    KCHK2(cudaEventRecord(ev[slices], h->stream), "event");  // the allocations, for the copy stream
    KCHK2(cudaStreamWaitEvent(cs, ev[slices], 0), "event");
    KCHK2(cudaMemcpyAsync(rp64, rowptr, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyDefault, h->stream), "copy rowptr");
    for (int i = 0; i < slices; ++i) {
        if (acut[i + 1] > acut[i])
            KCHK2(cudaMemcpyAsync(col0 + acut[i], col + acut[i], (size_t)(acut[i + 1] - acut[i]) * sizeof(int32_t),
                                  cudaMemcpyDefault, cs), "copy col");
        KCHK2(cudaEventRecord(ev[i], cs), "event");
    }
    // offsets: monotone, rowptr[0] = 0, rowptr[n] = nnz, and deg_max
    unsigned long long* d_bad = nullptr;  // [0] offsets malformed, [1] column entries out of range, [2] max chunks
    int64_t* d_degmax = nullptr;
    KCHK2(dmalloc(h, &d_bad, 3), "cudaMalloc");
    KCHK2(dmalloc(h, &d_degmax, 1), "cudaMalloc");
    KCHK2(cudaMemsetAsync(d_bad, 0, 3 * sizeof(unsigned long long), h->stream), "memset");
    KCHK2(cudaMemsetAsync(d_degmax, 0, sizeof(int64_t), h->stream), "memset");
    {
        DeviceGraph g64;
        g64.n = n;
        g64.nnz = nnz;
        g64.off64 = true;
        g64.rowptr = rp64;
        g64.col = nullptr;
        KCHK2(launch_validate_csr(g64, d_bad, d_degmax, h->stream), "validate");
    }
    // relabel: stable counting sort by degree class, then the new offsets
    int64_t* counts = nullptr;
    uint64_t* class_start = nullptr;
    int64_t* deg_new = nullptr;
    int64_t* rp_new = nullptr;
    int64_t* sums = nullptr;
    KCHK2(dmalloc(h, &counts, (size_t)relabel_scratch(n)), "cudaMalloc counts");
    KCHK2(dmalloc(h, &class_start, NUM_CLASSES), "cudaMalloc");
    KCHK2(dmalloc(h, &g.perm, (size_t)n), "cudaMalloc perm");
    KCHK2(dmalloc(h, &g.inv, (size_t)n), "cudaMalloc inv");
    KCHK2(dmalloc(h, &deg_new, (size_t)n + 1), "cudaMalloc");
    KCHK2(dmalloc(h, &rp_new, (size_t)n + 1), "cudaMalloc");
    KCHK2(dmalloc(h, &sums, (size_t)scan_blocks(n + 1)), "cudaMalloc");
    KCHK2(dmalloc(h, &g.col, (size_t)nnz), "cudaMalloc col");
    KCHK2(relabel_by_degree_class(rp64, n, counts, g.perm, g.inv, class_start, h->stream), "relabel");
    KCHK2(relabel_offsets(rp64, g.perm, n, deg_new, rp_new, sums, h->stream), "relabel offsets");
    // small reads go through pinned memory: a pageable copy would queue
    // behind the column slices still in flight
    struct HostVals {
        unsigned long long bad, bad_col, max_chunks;
        int64_t degmax, chunks;
        uint64_t cs[NUM_CLASSES];
    };
    static_assert(sizeof(HostVals) <= H_SMALL, "pinned scratch");
    HostVals& hv = *(HostVals*)h->h_small;
    KCHK2(cudaMemcpyAsync(&hv.bad, d_bad, sizeof(hv.bad), cudaMemcpyDeviceToHost, h->stream), "copy");
    KCHK2(cudaMemcpyAsync(&hv.degmax, d_degmax, sizeof(hv.degmax), cudaMemcpyDeviceToHost, h->stream), "copy");
    KCHK2(cudaMemcpyAsync(hv.cs, class_start, sizeof(hv.cs), cudaMemcpyDeviceToHost, h->stream), "copy classes");
    KCHK2(cudaStreamSynchronize(h->stream), "validate sync");
    if (hv.bad) {
        drop_staging();
        katz_destroy(h);
        return KATZ_EINVAL;
    }
    h->deg_max = hv.degmax;
    h->D = std::max<int64_t>(h->opts.deg_bound, hv.degmax);
    for (int c = 0; c < NUM_CLASSES; ++c) h->cls_start[c] = hv.cs[c];
    h->classes_exact = true;
    // rows of degree > 2048 / > 128 / > 16 come first: classes >= 13 / >= 9 / >= 6
    const int64_t row_warp = (int64_t)hv.cs[12], row_octet = (int64_t)hv.cs[8], row_thread = (int64_t)hv.cs[5];
    // chunk table of the CHUNK rows, on the device (every CHUNK row holds more
    // than CHUNK_ARCS arcs, so the count stays below nnz / CHUNK_ARCS + row_warp)
    const int64_t chunks_cap = nnz / CHUNK_ARCS + row_warp + 1;
    KCHK2(dmalloc(h, &g.chunk_first, (size_t)row_warp + 1), "cudaMalloc");
    KCHK2(dmalloc(h, &g.chunk_row, (size_t)chunks_cap), "cudaMalloc");
    KCHK2(dmalloc(h, &g.chunk_part, 3 * (size_t)chunks_cap), "cudaMalloc");
    h->chunk_row_cap = chunks_cap;
    h->chunk_part_cap = chunks_cap;
    KCHK2(build_chunk_table(rp_new, row_warp, deg_new, sums, g.chunk_first, g.chunk_row, d_bad + 2, h->stream),
          "chunk table");
    // the column array, slice by slice as it arrives (entries range-checked),
    // renamed into degree-class order
    for (int i = 0; i < slices; ++i) {
        KCHK2(cudaStreamWaitEvent(h->stream, ev[i], 0), "event");
        KCHK2(remap_src_rows(rp64, col0, g.inv, rp_new, vcut[i], vcut[i + 1], n, row_warp, g.col, d_bad + 1,
                             h->stream), "relabel rows");
        KCHK2(remap_hub_chunks(rp64, col0, g.perm, g.inv, rp_new, g.chunk_row, g.chunk_first, row_warp, chunks_cap,
                               vcut[i], vcut[i + 1], n, g.col, d_bad + 1, h->stream), "relabel hub rows");
    }
    // then the low-degree rows reordered inside their classes by anchor
    // (katz_opts.locality); the rows of degree > 16 keep their places, the
    // staging column array holds the old tail
    const bool locality = (h->opts.locality > 0 || (h->opts.locality == 0 && n >= ((int64_t)1 << 25))) &&
                          n - row_thread > 1;
    if (locality) {
        const int64_t m = n - row_thread, cnt = 256 * radix_tiles(m);
        RadixBuffers rs;
        int64_t* rp_fin = nullptr;
        e = dmalloc(h, &rp_fin, (size_t)n + 1);
        for (int q = 0; q < 2 && e == cudaSuccess; ++q)
            if ((e = dmalloc(h, &rs.hi[q], (size_t)m)) == cudaSuccess && (e = dmalloc(h, &rs.lo[q], (size_t)m)) == cudaSuccess)
                e = dmalloc(h, &rs.val[q], (size_t)m);
        if (e == cudaSuccess && (e = dmalloc(h, &rs.counts, (size_t)cnt)) == cudaSuccess &&
            (e = dmalloc(h, &rs.offs, (size_t)cnt)) == cudaSuccess)
            e = dmalloc(h, &rs.sums, (size_t)scan_blocks(cnt));
        if (e == cudaSuccess)
            e = locality_order(n, nnz, row_thread, rp_new, g.col, g.perm, g.inv, deg_new, rp_fin, col0, sums, rs,
                               h->stream);
        for (int q = 0; q < 2; ++q) {
            dfree(h, rs.hi[q]);
            dfree(h, rs.lo[q]);
            dfree(h, rs.val[q]);
        }
        dfree(h, rs.counts);
        dfree(h, rs.offs);
        dfree(h, rs.sums);
        dfree(h, rp_new);
        rp_new = rp_fin;
        if (e != cudaSuccess) {
            dfree(h, rp_new);
            drop_staging();
            st = cuda_fail(h, e, "locality order");
            katz_destroy(h);
            return st;
        }
    }
    if (g.off64) {
        g.rowptr = rp_new;
        rp_new = nullptr;
    } else {
        int32_t* rp32 = nullptr;
        KCHK2(dmalloc(h, &rp32, (size_t)n + 1), "cudaMalloc rowptr32");
        KCHK2(launch_narrow_rowptr(rp_new, rp32, n + 1, h->stream), "narrow rowptr");
        g.rowptr = rp32;
    }
    KCHK2(cudaMemcpyAsync(&hv.bad_col, d_bad + 1, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream),
          "copy");
    KCHK2(cudaMemcpyAsync(&hv.chunks, g.chunk_first + row_warp, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream),
          "copy");
    KCHK2(cudaStreamSynchronize(h->stream), "relabel sync");
    g.layout = make_layout(n, row_warp, row_octet, row_thread, hv.chunks);
    h->sum_depth = max_sum_depth(g.layout, (int64_t)hv.max_chunks);
    dfree(h, d_bad);
    dfree(h, d_degmax);
    dfree(h, counts);
    dfree(h, class_start);
    dfree(h, deg_new);
    dfree(h, rp_new);
    dfree(h, sums);
    drop_staging();
    dfree(h, h->rp_new);  // the reverse graph of an inbound handle, now copied
    dfree(h, h->col_spare);
    h->rp_new = nullptr;
    h->col_spare = nullptr;
    h->col_spare_cap = 0;
    if (hv.bad_col) {  // a column entry outside [0, n)
        katz_destroy(h);
        return KATZ_EINVAL;
    }
#undef KCHK2
    if ((st = alloc_rank_scratch(h)) != KATZ_OK) {
        katz_destroy(h);
        return st;
    }
    KCHK(cudaStreamSynchronize(h->stream), "create sync");
#undef KCHK
    *out = h;
    return KATZ_OK;
}

static katz_status rank_static_once(katz_h h, double alpha, int64_t k, double eps, katz_info* info);

namespace katz {
// the handle's current top-k ranking recomputed from scratch with its alpha,
// k and eps (the FP32 escalation of an update)
katz_status rank_static_fp64(katz_handle* h, katz_info* info) {
    return rank_static_once(h, h->alpha, h->k_eff, h->eps, info);
}
}  // namespace katz

// KATZ_FP32_CERT_AUTO: a ranking whose FP32 rounding widening stalls the
// certificate is recomputed with FP64 levels on the same handle (the
// buffers of an FP32 handle hold FP64 levels too).
katz_status katz_rank_static(katz_h h, double alpha, int64_t k, double eps, katz_info* info) {
    if (!h) return KATZ_EINVAL;
    const L2FetchScope fetch(h);
    katz_status st = rank_static_once(h, alpha, k, eps, info);
    if (st != KATZ_EPRECISION || h->opts.precision != KATZ_FP32_CERT_AUTO) return st;
    const int64_t launches = h->launches;
    h->fp32 = false;
    st = rank_static_once(h, alpha, k, eps, info);
    h->fp32 = true;
    h->launches += launches;
    if (info) {
        info->escalated = 1;
        info->launches = h->launches;
    }
    return st;
}

static katz_status rank_static_once(katz_h h, double alpha, int64_t k, double eps, katz_info* info) {
    if (!h) return KATZ_EINVAL;
    h->err.clear();
    if (!(eps > 0.0) || !std::isfinite(eps) || k < 1 || !std::isfinite(alpha))
        return fail(h, KATZ_EINVAL, "need eps > 0, k >= 1, finite alpha");
    const int64_t k_eff = std::min<int64_t>(k, h->g.n);
    if (k_eff > KATZ_MAX_K) return fail(h, KATZ_EINVAL, "k exceeds KATZ_MAX_K");
    double a = 0.0, gamma = 0.0;
    katz_status st = setup_ranking(h, alpha, k_eff, eps, a, gamma);
    if (st != KATZ_OK) return st;
    IterParams& p = h->p;
    h->criterion = KATZ_CRIT_TOPK;
    h->b.use_cond = 0;
    h->ranked = false;
    h->launches = h->classes_exact ? 3 : 4;  // init_walk, cert_init, theta_0 (one or two kernels)
    cudaError_t e;
    if ((e = cudaEventRecord(h->ev0, h->stream)) != cudaSuccess) return cuda_fail(h, e, "event");
    if ((e = cudaMemsetAsync(h->b.ctrl, 0, sizeof(Ctrl), h->stream)) != cudaSuccess) return cuda_fail(h, e, "memset ctrl");
    if ((e = launch_init_walk(h->g, h->b, p, h->fp32, h->stream)) != cudaSuccess) return cuda_fail(h, e, "init");
    if ((e = launch_cert_init(h->b, p, h->stream)) != cudaSuccess) return cuda_fail(h, e, "init levels");
    const bool prof = h->opts.profile != 0;
    if (h->classes_exact) {
        // the degree class holding the k-th largest degree: classes are laid
        // out from the highest down, class c (>= 1) ends where class c-1 starts
        const int64_t n = h->g.n;
        auto end_of = [&](int c) -> int64_t { return c >= 1 ? (int64_t)h->cls_start[c - 1] : n; };
        int c = NUM_CLASSES - 1;
        while (c > 0 && end_of(c) < k_eff) --c;
        const int64_t a = (int64_t)h->cls_start[c];
        const int64_t lo = c == 0 ? -1 : (c == 1 ? 0 : (int64_t)1 << (c - 2));
        const int bits = c >= 2 ? c - 2 : 0;
        if ((e = launch_theta0_class(h->g, h->b, p, a, end_of(c), lo, bits, k_eff - a, h->stream)) != cudaSuccess)
            return cuda_fail(h, e, "theta0");
    } else if ((e = launch_theta0(h->g, h->b, p, h->d_deghist, deg_hist_top(h->D), h->stream)) != cudaSuccess) {
        return cuda_fail(h, e, "theta0");
    }
    if (prof && (st = ensure_prof_events(h)) != KATZ_OK) return st;
    if ((e = launch_first_iteration(h, prof ? &h->sp_ev[0] : nullptr)) != cudaSuccess)
        return cuda_fail(h, e, "first iteration");
    h->launches += 4;  // degree level, select, count, finalize
    st = run_loop(h, 1);
    if (st != KATZ_OK) return st;
    if ((e = cudaEventRecord(h->ev1, h->stream)) != cudaSuccess) return cuda_fail(h, e, "event");
    if ((e = cudaMemcpyAsync(h->h_ctrl, h->b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "copy ctrl");
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(h, e, "sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    const Ctrl& hc = *h->h_ctrl;
    h->r = hc.r;
    h->converged = hc.converged;
    h->k_eff = hc.k_eff;
    h->alpha = a;
    h->gamma = gamma;
    h->eps = eps;
    h->ranked = true;
    h->last_ms = ms;
    std::vector<int64_t> tr((size_t)h->opts.r_max + 2, 0);
    if ((e = cudaMemcpyAsync(tr.data(), h->b.trace, tr.size() * sizeof(int64_t), cudaMemcpyDeviceToHost,
                             h->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "copy trace");
    h->trace.assign(tr.begin() + 1, tr.begin() + 1 + std::max(0, h->r));
    if (h->opts.use_graph && !h->opts.profile)
        // loop bodies that did work: all finalize runs but the first iteration's
        h->launches += (h->g.layout.row_warp > 0 ? 5 : 4) * std::max<int64_t>(0, (int64_t)hc.body_runs - 1);
    double spmv_ms = 0.0;
    if (h->opts.profile) {  // levels 2..r: level 1 reads no walk values
        for (int q = 1; q < h->r && 2 * q + 1 < (int)h->sp_ev.size(); ++q) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, h->sp_ev[2 * q], h->sp_ev[2 * q + 1]) == cudaSuccess) spmv_ms += t;
        }
    }
    const int fp32_levels = (h->fp32 && hc.f32_from <= h->r) ? h->r - hc.f32_from + 1 : 0;
    h->f32_from = hc.f32_from;
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->fp32_levels = fp32_levels;
        info->spmv_ms = spmv_ms;
        info->spmv_launches = std::max(0, h->r - 1);
        info->launches = h->launches;
        info->r = h->r;
        info->converged = h->converged;
        info->active = h->trace.empty() ? h->g.n : h->trace.back();
        info->k = h->k_eff;
        info->alpha = a;
        info->gamma = gamma;
        info->time_ms = ms;
        info->nnz = h->g.nnz;
    }
    if (!h->converged && hc.stall)
        return fail(h, KATZ_EPRECISION, "FP32 rounding widening exceeds the remaining tail; rank in FP64");
    if (!h->converged) return fail(h, KATZ_ENOTCONV, "r_max reached before the top-k criterion held");
    return KATZ_OK;
}

katz_status katz_rank(katz_h h, double alpha, int32_t criterion, int64_t k, const int32_t* pair, double eps,
                      katz_info* info) {
    if (!h) return KATZ_EINVAL;
    if (criterion == KATZ_CRIT_TOPK) return katz_rank_static(h, alpha, k, eps, info);
    const L2FetchScope fetch(h);
    h->err.clear();
    if (criterion != KATZ_CRIT_RANKING && criterion != KATZ_CRIT_SCORE && criterion != KATZ_CRIT_PAIR)
        return fail(h, KATZ_EINVAL, "unknown criterion");
    if (h->fp32) return fail(h, KATZ_ESTATE, "the ranking, score and pair criteria run on FP64 handles");
    if (!(eps > 0.0) || !std::isfinite(eps) || !std::isfinite(alpha))
        return fail(h, KATZ_EINVAL, "need eps > 0 and a finite alpha");
    const int64_t n = h->g.n;
    int32_t oa = 0, ob = 0;
    if (criterion == KATZ_CRIT_PAIR) {
        if (!pair) return fail(h, KATZ_EINVAL, "the pair criterion needs two node ids");
        oa = pair[0];
        ob = pair[1];
        if (oa < 0 || ob < 0 || oa >= n || ob >= n || oa == ob)
            return fail(h, KATZ_EINVAL, "the pair must be two distinct nodes");
    }
    const int64_t k_eff = criterion == KATZ_CRIT_RANKING ? n : (criterion == KATZ_CRIT_PAIR ? 2 : 0);
    double a = 0.0, gamma = 0.0;
    katz_status st = setup_ranking(h, alpha, std::max<int64_t>(k_eff, 1), eps, a, gamma);
    if (st != KATZ_OK) return st;
    IterParams& p = h->p;
    cudaError_t e;
    if (criterion == KATZ_CRIT_RANKING && !h->rank_ids) {
        RadixBuffers& rs = h->rs;
        const int64_t cnt = 256 * radix_tiles(n);
        if ((e = dmalloc(h, &h->rank_ids, (size_t)n)) != cudaSuccess ||
            (e = dmalloc(h, &rs.hi[0], (size_t)n)) != cudaSuccess || (e = dmalloc(h, &rs.hi[1], (size_t)n)) != cudaSuccess ||
            (e = dmalloc(h, &rs.lo[0], (size_t)n)) != cudaSuccess || (e = dmalloc(h, &rs.lo[1], (size_t)n)) != cudaSuccess ||
            (e = dmalloc(h, &rs.val[0], (size_t)n)) != cudaSuccess ||
            (e = dmalloc(h, &rs.val[1], (size_t)n)) != cudaSuccess ||
            (e = dmalloc(h, &rs.counts, (size_t)cnt)) != cudaSuccess ||
            (e = dmalloc(h, &rs.offs, (size_t)cnt)) != cudaSuccess ||
            (e = dmalloc(h, &rs.sums, (size_t)scan_blocks(cnt))) != cudaSuccess)
            return cuda_fail(h, e, "cudaMalloc ranking buffers");
    }
    h->criterion = criterion;
    h->ranked = false;
    h->launches = 0;
    const int64_t spmv_kernels = h->g.layout.row_warp > 0 ? 2 : 1;
    const int64_t check_kernels = criterion == KATZ_CRIT_RANKING ? 2 + 12 * 5 : 1;  // keys, 12 x (hist, scan 3, scatter), check
    if ((e = cudaEventRecord(h->ev0, h->stream)) != cudaSuccess) return cuda_fail(h, e, "event");
    if ((e = cudaMemsetAsync(h->b.ctrl, 0, sizeof(Ctrl), h->stream)) != cudaSuccess ||
        (e = launch_init_walk(h->g, h->b, p, false, h->stream)) != cudaSuccess ||
        (e = launch_cert_init(h->b, p, h->stream)) != cudaSuccess ||
        (e = launch_crit_init(h->b, h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "init");
    h->launches += 3;
    for (int it = 0; it < p.r_max; ++it) {
        // level 1 is the degree vector (A 1 = deg), one O(n) pass
        e = it == 0 ? launch_degree_level(h->g, h->b, p, h->stream) : launch_spmv(h->g, h->b, p, false, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "spmv");
        if (criterion == KATZ_CRIT_RANKING)
            e = launch_ranking_check(h->g, h->b, p, h->rs, h->rank_ids, h->stream);
        else if (criterion == KATZ_CRIT_SCORE)
            e = launch_score_check(h->b, p, h->stream);
        else
            e = launch_pair_check(h->g, h->b, p, oa, ob, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "criterion");
        if ((e = launch_finalize_crit(h->b, p, h->stream)) != cudaSuccess) return cuda_fail(h, e, "finalize");
        h->launches += (it == 0 ? 1 : spmv_kernels) + check_kernels + 1;
        if ((e = cudaMemcpyAsync(h->h_ctrl, h->b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
            return cuda_fail(h, e, "sync");
        if (h->h_ctrl->stop) break;
    }
    if ((e = cudaEventRecord(h->ev1, h->stream)) != cudaSuccess ||
        (e = cudaEventSynchronize(h->ev1)) != cudaSuccess)
        return cuda_fail(h, e, "event");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    const Ctrl& hc = *h->h_ctrl;
    h->r = hc.r;
    h->converged = hc.converged;
    h->k_eff = k_eff;
    h->alpha = a;
    h->gamma = gamma;
    h->eps = eps;
    h->ranked = true;
    h->last_ms = ms;
    h->f32_from = 0x7fffffff;
    h->trace.assign((size_t)std::max(0, h->r), n);
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->r = h->r;
        info->converged = h->converged;
        info->active = n;
        info->k = k_eff;
        info->alpha = a;
        info->gamma = gamma;
        info->time_ms = ms;
        info->nnz = h->g.nnz;
        info->launches = h->launches;
        info->spmv_launches = std::max(0, h->r - 1);
    }
    if (!h->converged) return fail(h, KATZ_ENOTCONV, "r_max reached before the criterion held");
    return KATZ_OK;
}

katz_status katz_get_ranking(katz_h h, int32_t* ids, int64_t k) {
    if (!h || !ids) return KATZ_EINVAL;
    if (!h->ranked) return fail(h, KATZ_ESTATE, "no ranking yet");
    if (h->criterion == KATZ_CRIT_SCORE) return fail(h, KATZ_ESTATE, "the score criterion certifies scores, not an order");
    if (k < 0 || k > h->k_eff) return fail(h, KATZ_EINVAL, "k larger than the ranked k");
    if (k == 0) return KATZ_OK;
    const int32_t* src = h->criterion == KATZ_CRIT_RANKING ? h->rank_ids : h->b.topk_id;
    cudaError_t e = cudaMemcpyAsync(ids, src, (size_t)k * sizeof(int32_t), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? KATZ_OK : cuda_fail(h, e, "copy ranking");
}

katz_status katz_get_bounds(katz_h h, double* lower, double* upper, double* err) {
    if (!h) return KATZ_EINVAL;
    if (!h->ranked) return fail(h, KATZ_ESTATE, "no ranking yet");
    const int64_t n = h->g.n;
    cudaError_t e;
    const bool dev = (!lower || is_device_ptr(lower)) && (!upper || is_device_ptr(upper)) &&
                     (!err || is_device_ptr(err));
    double* dl = lower;
    double* du = upper;
    double* de = err;
    if (!dev) {
        if (!h->d_scratch) {
            if ((e = dmalloc(h, &h->d_scratch, 3 * (size_t)n)) != cudaSuccess) return cuda_fail(h, e, "cudaMalloc");
        }
        dl = lower ? h->d_scratch : nullptr;
        du = upper ? h->d_scratch + n : nullptr;
        de = err ? h->d_scratch + 2 * n : nullptr;
    }
    if ((e = launch_bounds_out(h->g, h->b, h->p, h->r, h->fp32, dl, du, de, h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "bounds");
    if (!dev) {
        if (lower && (e = cudaMemcpyAsync(lower, dl, (size_t)n * sizeof(double), cudaMemcpyDefault, h->stream)) != cudaSuccess)
            return cuda_fail(h, e, "copy lower");
        if (upper && (e = cudaMemcpyAsync(upper, du, (size_t)n * sizeof(double), cudaMemcpyDefault, h->stream)) != cudaSuccess)
            return cuda_fail(h, e, "copy upper");
        if (err && (e = cudaMemcpyAsync(err, de, (size_t)n * sizeof(double), cudaMemcpyDefault, h->stream)) != cudaSuccess)
            return cuda_fail(h, e, "copy err");
    }
    e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? KATZ_OK : cuda_fail(h, e, "sync");
}

katz_status katz_get_walk(katz_h h, int32_t i, double* s_out) {
    if (!h || !s_out) return KATZ_EINVAL;
    if (!h->ranked) return fail(h, KATZ_ESTATE, "no ranking yet");
    if (i < 0 || i > h->r || i <= h->r - h->walk_slots)
        return fail(h, KATZ_EINVAL, "walk level not retained (keep_history = 0 keeps the last two)");
    const int64_t n = h->g.n;
    cudaError_t e;
    double* dst = s_out;
    const bool dev = is_device_ptr(s_out);
    if (!dev) {
        if (!h->d_scratch && (e = dmalloc(h, &h->d_scratch, 3 * (size_t)n)) != cudaSuccess) return cuda_fail(h, e, "cudaMalloc");
        dst = h->d_scratch;
    }
    if ((e = launch_walk_out(h->g, h->b, h->p, i, h->fp32, dst, h->stream)) != cudaSuccess) return cuda_fail(h, e, "walk");
    if (!dev && (e = cudaMemcpyAsync(s_out, dst, (size_t)n * sizeof(double), cudaMemcpyDefault, h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "copy walk");
    e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? KATZ_OK : cuda_fail(h, e, "sync");
}

katz_status katz_get_trace(katz_h h, int64_t* active_per_iter, int32_t cap) {
    if (!h || !active_per_iter || cap < 0) return KATZ_EINVAL;
    if (!h->ranked) return fail(h, KATZ_ESTATE, "no ranking yet");
    const int32_t m = std::min<int32_t>(cap, (int32_t)h->trace.size());
    for (int32_t q = 0; q < m; ++q) active_per_iter[q] = h->trace[q];
    return KATZ_OK;
}

}  // extern "C"

namespace katz {

// Phase 1 of Algorithm 2 for one batch, on stream_a: the preconditions
// checked against the current graph, then the updated graph built into the
// spare buffers (col, row offsets, chunk table).  The current graph and
// everything the repair of an earlier batch reads stay untouched, so this can
// run while that repair is on the device.  The result waits in h->pend.
katz_status update_prepare(katz_handle* h, const int32_t* src, const int32_t* dst, const uint8_t* is_insert,
                           int64_t m, cudaEvent_t ready) {
    katz_handle::Pending& pd = h->pend;
    pd = katz_handle::Pending();
    pd.m = m;
    cudaError_t e;
    const DeviceGraph& g = h->g;
    const int64_t n = g.n;
    if (!h->stream_a) {  // the stream and events of the two phases, once
        if ((e = cudaStreamCreateWithFlags(&h->stream_a, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->ev_prepared, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->ev_committed, cudaEventDisableTiming)) != cudaSuccess) {
            pd.status = KATZ_ECUDA;
            pd.err = "update stream";
            pd.ready = true;
            return pd.status;
        }
    }
    cudaStream_t sa = h->stream_a;
    // every way out records ev_prepared on stream_a: the commit waits for it
    auto done = [&](katz_status st, const char* msg) {
        pd.status = st;
        if (msg) pd.err = msg;
        cudaEventRecord(h->ev_prepared, sa);
        pd.ready = true;
        return st;
    };
    auto cuda_done = [&](cudaError_t ce, const char* what) {
        return done(ce == cudaErrorMemoryAllocation ? KATZ_ENOMEM : KATZ_ECUDA,
                    (std::string(what) + ": " + cudaGetErrorString(ce)).c_str());
    };
    // the spare buffers held the graph before the current one: the repair
    // that read it is queued on the handle's stream before ev_committed
    if ((e = cudaStreamWaitEvent(sa, h->ev_committed, 0)) != cudaSuccess) return cuda_done(e, "event");
    if (ready && (e = cudaStreamWaitEvent(sa, ready, 0)) != cudaSuccess) return cuda_done(e, "event");  // the batch
    {
        const katz_status rs = dyn_reserve(h, m, 0, sa);
        if (rs != KATZ_OK) return done(rs, "cudaMalloc update scratch");
    }
    const int bs = h->next_bset;
    h->next_bset ^= 1;
    pd.bset = bs;
    DynBuffers d = h->dyn;  // this phase's view: its batch set
    d.src = h->bsrc[bs];
    d.dst = h->bdst[bs];
    d.ins = h->bins[bs];
    d.undirected = h->opts.undirected != 0;
    if (m == 0) return done(KATZ_OK, nullptr);
    if ((e = cudaMemcpyAsync(d.src, src, (size_t)m * sizeof(int32_t), cudaMemcpyDefault, sa)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d.dst, dst, (size_t)m * sizeof(int32_t), cudaMemcpyDefault, sa)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d.ins, is_insert, (size_t)m, cudaMemcpyDefault, sa)) != cudaSuccess)
        return cuda_done(e, "copy batch");
    // ---- validate (nothing changes unless the whole batch is valid) --------------
    int32_t* herr = (int32_t*)(h->h_small + H_SMALL - 64);  // pinned words of this phase
    if ((e = cudaMemsetAsync(d.err, 0, sizeof(int32_t), sa)) != cudaSuccess ||
        (e = dyn_validate(g, d, m, h->D, sa)) != cudaSuccess ||
        (e = cudaMemcpyAsync(herr, d.err, sizeof(int32_t), cudaMemcpyDeviceToHost, sa)) != cudaSuccess ||
        (e = cudaStreamSynchronize(sa)) != cudaSuccess)
        return cuda_done(e, "validate batch");
    pd.launches += 2;
    if (*herr) {
        const int32_t err = *herr;
        if ((e = dyn_clear(g, d, m, sa)) != cudaSuccess || (e = cudaStreamSynchronize(sa)) != cudaSuccess)
            return cuda_done(e, "clear batch");
        if (err & DYN_E_INVAL)
            return done(KATZ_EINVAL, "batch violates the preconditions (range, self-loop, duplicate pair, "
                                     "inserted edge present or deleted edge absent)");
        return done(KATZ_EALPHA, "a row would exceed the degree bound D");
    }
    // ---- apply: new offsets, rows rebuilt into the spare buffers ------------------
    if ((e = dyn_prepare(g, d, m, h->rp_new, h->deg_tmp, h->scan_sums, sa)) != cudaSuccess)
        return cuda_done(e, "prepare rebuild");
    pd.launches += 8;  // 5 bucket/degree kernels + 3 scan passes
    // FP32-certified levels: the rows the batch lengthens bound the chain of
    // FP32 additions of their repaired sums (the precision option is fixed at
    // creation; the repair reads the handle's current mode)
    const bool cert = h->opts.precision != KATZ_FP64;
    unsigned long long* hdmax = (unsigned long long*)(h->h_small + H_SMALL - 128);
    if (cert && ((e = dyn_mode_degree_max(g, d, m, h->rp_new, sa)) != cudaSuccess ||
                 (e = cudaMemcpyAsync(hdmax, d.mode_dmax, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                      sa)) != cudaSuccess))
        return cuda_done(e, "degree maxima");
    pd.launches += cert ? 1 : 0;
    int64_t* hnnz = (int64_t*)(h->h_small + H_SMALL - 56);
    if ((e = cudaMemcpyAsync(hnnz, h->rp_new + n, sizeof(int64_t), cudaMemcpyDeviceToHost, sa)) != cudaSuccess ||
        (e = cudaStreamSynchronize(sa)) != cudaSuccess)
        return cuda_done(e, "rebuild size");
    const unsigned long long dmax[3] = {cert ? hdmax[0] : 0ull, cert ? hdmax[1] : 0ull, cert ? hdmax[2] : 0ull};
    const int64_t nnz_new = *hnnz;
    // the updated graph outgrows 32-bit offsets: its offsets go to a new
    // int64 array, and a second one becomes the spare of later batches; the
    // swap installs both and releases the two int32 arrays
    const bool promote = !g.off64 && n + nnz_new >= 0x7fffffffLL;
    if (promote && !h->rp64_next) {
        if ((e = dmalloc_on(h, &h->rp64_next, (size_t)n + 1, sa)) != cudaSuccess ||
            (e = dmalloc_on(h, &h->rp64_spare_next, (size_t)n + 1, sa)) != cudaSuccess) {
            dfree_on(h->rp64_next, sa);
            dfree_on(h->rp64_spare_next, sa);
            h->rp64_next = nullptr;
            h->rp64_spare_next = nullptr;
            dyn_clear(g, d, m, sa);
            cudaStreamSynchronize(sa);
            return cuda_done(e, "cudaMalloc int64 rowptr");
        }
    }
    if (nnz_new > h->col_spare_cap) {
        dfree_on(h->col_spare, sa);
        h->col_spare = nullptr;
        h->col_spare_cap = 0;
        const int64_t cap = nnz_new + nnz_new / 16 + 1024;
        if ((e = dmalloc_on(h, &h->col_spare, (size_t)cap, sa)) != cudaSuccess) {
            dyn_clear(g, d, m, sa);
            cudaStreamSynchronize(sa);
            return cuda_done(e, "cudaMalloc col");
        }
        h->col_spare_cap = cap;
    }
    const bool hubs = g.layout.row_warp > 0;
    if (hubs && g.layout.chunks > d.hub_keep_cap) {
        dfree_on(h->dyn.hub_keep, sa);
        h->dyn.hub_keep = nullptr;
        h->dyn.hub_keep_cap = 0;
        const int64_t cap = g.layout.chunks + g.layout.chunks / 8 + 64;
        if ((e = dmalloc_on(h, &h->dyn.hub_keep, (size_t)cap, sa)) != cudaSuccess) {
            dyn_clear(g, d, m, sa);
            cudaStreamSynchronize(sa);
            return cuda_done(e, "cudaMalloc hub chunks");
        }
        h->dyn.hub_keep_cap = cap;
        d.hub_keep = h->dyn.hub_keep;
        d.hub_keep_cap = cap;
    }
    if ((e = dyn_rebuild(g, d, m, h->rp_new, h->col_spare, promote ? (void*)h->rp64_next : h->rowptr_spare, promote,
                         sa)) != cudaSuccess)
        return cuda_done(e, "rebuild rows");
    pd.launches += (g.n > g.layout.row_warp ? 2 : 0) + (g.layout.chunks > 0 ? 1 : 0) + (hubs ? 3 : 0) + 1;
    if ((e = dyn_clear(g, d, m, sa)) != cudaSuccess) return cuda_done(e, "clear batch");
    pd.launches += 1;
    // chunk table of the CHUNK rows from their new degrees, into the spares
    const int64_t rw = g.layout.row_warp;
    std::vector<int64_t> hrp((size_t)rw + 1);
    if ((e = cudaMemcpyAsync(hrp.data(), h->rp_new, hrp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, sa)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(sa)) != cudaSuccess)
        return cuda_done(e, "copy rowptr head");
    std::vector<int64_t> first((size_t)rw + 1, 0);
    int64_t max_chunks = 0;
    for (int64_t u = 0; u < rw; ++u) {
        const int64_t c = (hrp[u + 1] - hrp[u] + CHUNK_ARCS - 1) / CHUNK_ARCS;
        first[u + 1] = first[u] + c;
        max_chunks = std::max(max_chunks, c);
    }
    const int64_t chunks = first[rw];
    if (cert) {
        const SpmvLayout& L = g.layout;
        pd.depth = sum_depth_of((int64_t)dmax[0], (int64_t)dmax[1], (int64_t)dmax[2], L.row_thread > L.row_octet,
                                L.row_octet > L.row_warp, rw > 0 ? std::max<int64_t>(max_chunks, 1) : 0);
    }
    if (chunks > h->chunk_row_spare_cap) {
        dfree_on(h->chunk_row_spare, sa);
        h->chunk_row_spare = nullptr;
        h->chunk_row_spare_cap = 0;
        const int64_t cap = chunks + chunks / 8 + 16;
        if ((e = dmalloc_on(h, &h->chunk_row_spare, (size_t)cap, sa)) != cudaSuccess)
            return cuda_done(e, "cudaMalloc chunks");
        h->chunk_row_spare_cap = cap;
    }
    std::vector<int32_t> crow((size_t)std::max<int64_t>(chunks, 1));
    for (int64_t u = 0; u < rw; ++u)
        for (int64_t q = first[u]; q < first[u + 1]; ++q) crow[q] = (int32_t)u;
    if ((e = cudaMemcpyAsync(h->chunk_first_spare, first.data(), first.size() * sizeof(int64_t),
                             cudaMemcpyHostToDevice, sa)) != cudaSuccess ||
        (chunks > 0 && (e = cudaMemcpyAsync(h->chunk_row_spare, crow.data(), (size_t)chunks * sizeof(int32_t),
                                            cudaMemcpyHostToDevice, sa)) != cudaSuccess) ||
        (e = cudaStreamSynchronize(sa)) != cudaSuccess)
        return cuda_done(e, "copy chunks");
    pd.nnz = nnz_new;
    pd.chunks = chunks;
    pd.applied = true;
    pd.promote = promote;
    return done(KATZ_OK, nullptr);
}

// Phase 2a on the handle's stream: the prepared graph becomes the current
// one (host-side swaps; once this returns, the next batch may be prepared).
katz_status update_swap(katz_handle* h) {
    katz_handle::Pending& pd = h->pend;
    cudaError_t e;
    DeviceGraph& g = h->g;
    const int64_t n = g.n;
    h->err.clear();
    h->launches = pd.launches;
    if ((e = cudaStreamWaitEvent(h->stream, h->ev_prepared, 0)) != cudaSuccess) return cuda_fail(h, e, "event");
    if ((e = cudaEventRecord(h->ev0, h->stream)) != cudaSuccess) return cuda_fail(h, e, "event");
    h->rep = pd;  // the next prepare may overwrite pend once this returns
    if (pd.status != KATZ_OK || !pd.applied) {
        if ((e = cudaEventRecord(h->ev_committed, h->stream)) != cudaSuccess) return cuda_fail(h, e, "event");
        return pd.status != KATZ_OK ? fail(h, pd.status, pd.err) : KATZ_OK;
    }
    {
        std::swap(g.col, h->col_spare);
        std::swap(h->col_cap, h->col_spare_cap);
        if (pd.promote) {  // int32 -> int64 offsets; the old arrays are released after the work queued on them
            dfree(h, g.rowptr);
            dfree(h, h->rowptr_spare);
            g.rowptr = h->rp64_next;
            h->rowptr_spare = h->rp64_spare_next;
            h->rp64_next = nullptr;
            h->rp64_spare_next = nullptr;
            g.off64 = true;
        } else {
            std::swap(g.rowptr, h->rowptr_spare);
        }
        std::swap(g.chunk_first, h->chunk_first_spare);
        std::swap(g.chunk_row, h->chunk_row_spare);
        std::swap(h->chunk_row_cap, h->chunk_row_spare_cap);
        g.nnz = pd.nnz;
        if (pd.chunks > h->chunk_part_cap) {
            dfree(h, g.chunk_part);
            g.chunk_part = nullptr;
            h->chunk_part_cap = 0;
            const int64_t cap = pd.chunks + pd.chunks / 8 + 16;
            if ((e = dmalloc(h, &g.chunk_part, 3 * (size_t)cap)) != cudaSuccess)
                return cuda_fail(h, e, "cudaMalloc chunk sums");
            h->chunk_part_cap = cap;
        }
        g.layout = make_layout(n, g.layout.row_warp, g.layout.row_octet, g.layout.row_thread, pd.chunks);
        h->classes_exact = false;  // rows keep their place while their degrees change
        drop_graph(h);             // captured launches hold the old arrays and layout
        // the next prepare may overwrite the old graph once the work on it,
        // queued before this point, is done
        if ((e = cudaEventRecord(h->ev_committed, h->stream)) != cudaSuccess) return cuda_fail(h, e, "event");
    }
    return KATZ_OK;
}

// Phase 2b on the handle's stream: s_1..s_r repaired (Sec. 4), the bounds and
// the active set re-derived, and further iterations until converged() holds.
// The levels (repair_levels) and the rest (repair_finish) are separate steps:
// the two-state pass (update_pair_levels) computes the levels of two batches
// at once and then runs repair_finish for each.
static katz_status repair_levels(katz_handle* h, int64_t& full_levels, int64_t& affected, bool& all_rows);
static katz_status repair_finish(katz_handle* h, katz_info* info, int64_t full_levels, int64_t affected,
                                 bool all_rows);

katz_status update_repair(katz_handle* h, katz_info* info) {
    int64_t full_levels = 0, affected = 0;
    bool all_rows = false;
    const katz_status st = repair_levels(h, full_levels, affected, all_rows);
    return st != KATZ_OK ? st : repair_finish(h, info, full_levels, affected, all_rows);
}

static katz_status repair_levels(katz_handle* h, int64_t& full_levels, int64_t& affected, bool& all_rows) {
    const katz_handle::Pending& pd = h->rep;
    cudaError_t e;
    DeviceGraph& g = h->g;
    const int64_t n = g.n, m = pd.m;
    const int r = h->r;
    DynBuffers d = h->dyn;  // the repair's view: the batch set its prepare used
    d.src = h->bsrc[pd.bset];
    d.dst = h->bdst[pd.bset];
    d.ins = h->bins[pd.bset];
    d.undirected = h->opts.undirected != 0;
    const bool hubs = g.layout.row_warp > 0;
    full_levels = 0;
    affected = 0;
    all_rows = false;
    if (pd.applied) {
        // directed: the reverse BFS walks in-arcs, from the transposed CSR of
        // the updated graph
        if (!d.undirected) {
            if (!h->rrowptr && (e = dmalloc(h, &h->rrowptr, (size_t)n + 1)) != cudaSuccess)
                return cuda_fail(h, e, "cudaMalloc transposed offsets");
            if (!h->t_cnt && ((e = dmalloc(h, &h->t_cnt, (size_t)n + 1)) != cudaSuccess ||
                              (e = dmalloc(h, &h->t_sums, (size_t)scan_blocks(n + 1))) != cudaSuccess))
                return cuda_fail(h, e, "cudaMalloc transposition scratch");
            if (g.nnz > h->rcap) {
                dfree(h, h->rcol);
                h->rcol = nullptr;
                h->rcap = 0;
                const int64_t cap = g.nnz + g.nnz / 16 + 1024;
                if ((e = dmalloc(h, &h->rcol, (size_t)cap)) != cudaSuccess)
                    return cuda_fail(h, e, "cudaMalloc transposed arcs");
                h->rcap = cap;
            }
            d.rrowptr = h->rrowptr;
            d.rcol = h->rcol;
            d.rcap = h->rcap;
            if ((e = dyn_transpose(g, d, h->t_cnt, h->t_sums, h->stream)) != cudaSuccess)
                return cuda_fail(h, e, "transpose");
            h->launches += 3 + (g.nnz > 0 ? 1 + (g.n > g.layout.row_warp ? 1 : 0) + (g.layout.chunks > 0 ? 1 : 0) : 0);
        }
        // ---- repair s_1..s_r: affected rows only, or whole levels once the
        //      affected set is large (Sec. 4) ------------------------------------------
        if ((e = dyn_seed(g, d, m, h->stream)) != cudaSuccess) return cuda_fail(h, e, "seed frontier");
        h->launches += 1;
        unsigned long long* fs = (unsigned long long*)(h->h_small + H_SMALL - 32);  // frontier size, its arcs
        if ((e = cudaMemcpyAsync(fs, d.fsize, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
            return cuda_fail(h, e, "frontier size");
        const double tau = h->opts.frontier_abort_frac > 0 ? h->opts.frontier_abort_frac : 0.05;
        // a level goes full once the frontier holds more than tau of the nodes
        // or of the arcs (its rows' arcs are the work of a frontier level)
        auto too_big = [&](unsigned long long cnt, unsigned long long vol) {
            return (double)cnt > tau * (double)n || (double)vol > tau * (double)g.nnz;
        };
        // Expanding the nodes that joined at a level reads their arcs.  Past
        // tau/25 of all arcs (0.2% at the default tau) their neighbourhoods
        // hold hubs on graphs with skewed degrees, and the next frontier goes
        // full all the same; such an expansion is skipped and the remaining
        // levels are full.  Either way the repaired values are the same.
        const double expand_cap = tau / 25.0 * (double)g.nnz;
        int64_t lo = 0, hi = (int64_t)fs[0];
        unsigned long long vol_lo = 0;  // arcs of frontier[0, lo)
        bool full = too_big(fs[0], fs[1]);
        for (int i = 1; i <= r; ++i) {
            if (full) {
                e = i == 1 ? launch_degree_store(g, h->b, h->p, h->stream)
                           : launch_spmv_store(g, h->b, h->p, i, h->stream);
                if (e != cudaSuccess) return cuda_fail(h, e, "full level");
                ++full_levels;
                h->launches += i == 1 ? 1 : (hubs ? 2 : 1);
                continue;
            }
            if ((e = launch_rows_store(g, h->b, h->p, d.frontier, d.fsize, hi, d.vbits, i, h->stream)) != cudaSuccess)
                return cuda_fail(h, e, "repair rows");
            h->launches += (hi > 0 ? 1 : 0) + (hi > 0 && g.layout.chunks > 0 ? 2 : 0);
            if (i < r) {
                if ((double)(fs[1] - vol_lo) > expand_cap) {
                    full = true;
                    continue;
                }
                vol_lo = fs[1];
                if ((e = dyn_expand(g, d, lo, hi, i, h->stream)) != cudaSuccess) return cuda_fail(h, e, "expand");
                h->launches += hi > lo ? 1 + (d.undirected && g.layout.chunks > 0 ? 1 : 0) : 0;
                if ((e = cudaMemcpyAsync(fs, d.fsize, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                         h->stream)) != cudaSuccess ||
                    (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
                    return cuda_fail(h, e, "frontier size");
                lo = hi;
                hi = (int64_t)fs[0];
                full = too_big(fs[0], fs[1]);
            }
        }
        affected = full ? n : hi;
        all_rows = full;
    }
    return KATZ_OK;
}

static katz_status repair_finish(katz_handle* h, katz_info* info, int64_t full_levels, int64_t affected,
                                 bool all_rows) {
    const katz_handle::Pending& pd = h->rep;
    cudaError_t e;
    DeviceGraph& g = h->g;
    const int64_t n = g.n;
    const int r = h->r;
    DynBuffers d = h->dyn;
    if (pd.applied) {
        if ((e = dyn_recompute_c(g, h->b, d, h->p, r, all_rows, h->stream)) != cudaSuccess)
            return cuda_fail(h, e, "recompute c");
        h->launches += 1;
        // FP32-certified: a row sum longer than any before widens every
        // level's error bound; the bounds of level r are re-derived with it
        if (h->p.cert && pd.depth > h->p.depth) {
            h->p.depth = pd.depth;
            h->sum_depth = pd.depth;
            if ((e = launch_cert_replay(h->b, h->p, r, h->stream)) != cudaSuccess)
                return cuda_fail(h, e, "error bounds");
            h->launches += 1;
        }
    }
    // ---- bounds, reactivation, converged() at level r, then more iterations ------
    h->launches += 5;  // theta_lb, reactivate, select, count, finalize
    if ((e = dyn_reactivate(g, h->b, h->p, r, h->stream)) != cudaSuccess ||
        (e = launch_select(g, h->b, h->p, h->b.cand_l, h->b.cand_u, h->b.cand_id, h->fp32, h->stream)) != cudaSuccess ||
        (e = launch_count(g, h->b, h->p, h->fp32, h->stream)) != cudaSuccess ||
        (e = launch_finalize(h->b, h->p, h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "re-check");
    if ((e = cudaMemcpyAsync(h->h_ctrl, h->b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "re-check sync");
    katz_status st = KATZ_OK;
    if (!h->h_ctrl->stop) {
        st = run_loop(h, 0);
        if (st != KATZ_OK) return st;
    }
    if ((e = cudaEventRecord(h->ev1, h->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h->h_ctrl, h->b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    const Ctrl& hc = *h->h_ctrl;
    h->r = hc.r;
    h->converged = hc.converged;
    h->k_eff = hc.k_eff;
    h->last_ms = ms;
    h->f32_from = hc.f32_from;
    const bool stalled = !hc.converged && hc.stall;
    std::vector<int64_t> tr((size_t)h->opts.r_max + 2, 0);
    if ((e = cudaMemcpyAsync(tr.data(), h->b.trace, tr.size() * sizeof(int64_t), cudaMemcpyDeviceToHost,
                             h->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "copy trace");
    h->trace.assign(tr.begin() + 1, tr.begin() + 1 + std::max(0, h->r));
    if (stalled && h->opts.precision == KATZ_FP32_CERT_AUTO) {
        // the FP32 widening stalls the certificate on the updated graph: its
        // levels are recomputed in FP64 (the handle continues in FP64)
        const int64_t launches = h->launches;
        h->fp32 = false;
        const katz_status st2 = rank_static_fp64(h, info);
        h->fp32 = true;
        h->launches += launches;
        if (info) {
            info->escalated = 1;
            info->launches = h->launches;
            info->affected = n;
        }
        return st2;
    }
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->fp32_levels = (h->p.cert && hc.f32_from <= h->r) ? h->r - hc.f32_from + 1 : 0;
        info->r = h->r;
        info->converged = h->converged;
        info->active = h->trace.empty() ? n : h->trace.back();
        info->k = h->k_eff;
        info->alpha = h->alpha;
        info->gamma = h->gamma;
        info->time_ms = ms;
        info->nnz = g.nnz;
        info->affected = affected;
        info->full_levels = (int32_t)full_levels;
        info->launches = h->launches;
    }
    h->last_repair_whole = all_rows;
    if (stalled) return fail(h, KATZ_EPRECISION, "FP32 rounding widening exceeds the remaining tail; rank in FP64");
    if (!h->converged) return fail(h, KATZ_ENOTCONV, "r_max reached before the top-k criterion held");
    return KATZ_OK;
}

katz_status update_commit(katz_handle* h, katz_info* info) {
    const katz_status st = update_swap(h);
    return st != KATZ_OK ? st : update_repair(h, info);
}

// ---- two batches in one pass (katz_spmv.cu, "Two graph states in one pass") ----
bool pair_possible(katz_handle* h) {
    const katz_handle::Pending& a = h->rep;   // swapped in, not yet repaired
    const katz_handle::Pending& b = h->pend;  // prepared on top of it
    return h->opts.undirected && a.status == KATZ_OK && a.applied && b.ready && b.status == KATZ_OK && b.applied &&
           !b.promote && h->r >= 1 && h->ranked && h->criterion == KATZ_CRIT_TOPK;
}

katz_status update_pair_first(katz_handle* h, katz_info* info) {
    const katz_handle::Pending& pb = h->pend;
    DeviceGraph& g = h->g;
    const int64_t n = g.n;
    const int r = h->r;
    cudaError_t e;
    h->pair_r = -1;
    // the second state's graph: the spare buffers its prepare built
    DeviceGraph gb = g;
    gb.nnz = pb.nnz;
    gb.col = h->col_spare;
    gb.rowptr = h->rowptr_spare;
    gb.chunk_first = h->chunk_first_spare;
    gb.chunk_row = h->chunk_row_spare;
    gb.chunk_part = nullptr;
    gb.layout = make_layout(n, g.layout.row_warp, g.layout.row_octet, g.layout.row_thread, pb.chunks);
    const int64_t pstride = 2 * h->stride;
    const size_t need = (size_t)(r + 1) * (size_t)pstride;
    if (need > h->pair_P_cap) {
        dfree(h, h->pair_P);
        h->pair_P = nullptr;
        h->pair_P_cap = 0;
        if ((e = dmalloc(h, &h->pair_P, need)) != cudaSuccess) return cuda_fail(h, e, "cudaMalloc pair levels");
        h->pair_P_cap = need;
    }
    if (h->p.cert && !h->pair_t && (e = dmalloc(h, &h->pair_t, 2 * (size_t)n)) != cudaSuccess)
        return cuda_fail(h, e, "cudaMalloc pair roundings");
    const int64_t part_need = 6 * std::max<int64_t>(pb.chunks, 1);
    if (part_need > h->pair_part_cap) {
        dfree(h, h->pair_part);
        h->pair_part = nullptr;
        h->pair_part_cap = 0;
        if ((e = dmalloc(h, &h->pair_part, (size_t)part_need)) != cudaSuccess)
            return cuda_fail(h, e, "cudaMalloc pair chunk sums");
        h->pair_part_cap = part_need;
    }
    if ((e = cudaStreamWaitEvent(h->stream, h->ev_prepared, 0)) != cudaSuccess) return cuda_fail(h, e, "event");
    const int f32_from = h->f32_from;
    const int t_level = h->p.cert ? std::min(f32_from - 1, r) : 0;
    if ((e = launch_pair_levels(g, gb, h->bsrc[pb.bset], h->bdst[pb.bset], pb.m, h->p, r, f32_from, t_level,
                                h->pair_P, pstride, h->pair_t, h->pair_part, h->dyn.vbits, h->dyn.frontier,
                                h->dyn.fsize, h->stream)) != cudaSuccess ||
        (e = launch_pair_split(g, h->b, h->p, r, f32_from, 0, h->pair_P, pstride, h->pair_t, h->stream)) !=
            cudaSuccess)
        return cuda_fail(h, e, "pair levels");
    {  // launches: mark, degrees, per level SpMV (+ hub merge) and the fixes, split
        const int per_level = 1 + (gb.layout.row_warp > 0 ? 1 : 0) + (pb.m > 0 ? 1 + (g.layout.chunks > 0 ? 2 : 0) : 0);
        h->launches += (pb.m > 0 ? 1 : 0) + 1 + (int64_t)std::max(0, r - 1) * per_level + 1;
    }
    h->pair_r = r;
    h->pair_f32_from = f32_from;
    return repair_finish(h, info, r, n, true);
}

katz_status update_pair_second(katz_handle* h, katz_info* info) {
    const int r_pair = h->pair_r, f32_pair = h->pair_f32_from;
    h->pair_r = -1;
    h->pair_second_used = false;
    // the first batch's finish kept r and the precision: the second state's
    // levels of the same pass hold (else it is repaired alone)
    if (r_pair < 0 || !h->rep.applied || h->r != r_pair || h->f32_from != f32_pair) return update_repair(h, info);
    cudaError_t e;
    if ((e = launch_pair_split(h->g, h->b, h->p, r_pair, f32_pair, 1, h->pair_P, 2 * h->stride, h->pair_t,
                               h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "pair split");
    h->launches += 1;
    h->pair_second_used = true;
    return repair_finish(h, info, r_pair, h->g.n, true);
}

// the checks a handle must pass before it takes update batches
katz_status update_allowed(katz_handle* h) {
    if (!h->ranked) return fail(h, KATZ_ESTATE, "rank the graph before updating it");
    if (h->criterion != KATZ_CRIT_TOPK) return fail(h, KATZ_ESTATE, "dynamic updates continue the top-k criterion");
    if (!h->opts.keep_history) return fail(h, KATZ_ESTATE, "dynamic updates need keep_history = 1");
    return KATZ_OK;
}

}  // namespace katz

extern "C" {

// Algorithm 2 on the device: validate, apply, repair s_1..s_r, re-derive the
// active set and continue iterating until converged() holds again (the two
// phases back to back).
katz_status katz_apply_update_batch(katz_h h, const int32_t* src, const int32_t* dst, const uint8_t* is_insert,
                                    int64_t m, katz_info* info) {
    if (!h) return KATZ_EINVAL;
    const L2FetchScope fetch(h);
    h->err.clear();
    katz_status st = update_allowed(h);
    if (st != KATZ_OK) return st;
    if (m < 0 || (m > 0 && (!src || !dst || !is_insert))) return fail(h, KATZ_EINVAL, "bad batch arguments");
    // an inbound handle holds the reverse graph: the arc src -> dst of the
    // given graph is dst -> src there
    if (h->opts.inbound && !h->opts.undirected) std::swap(src, dst);
    update_prepare(h, src, dst, is_insert, m, nullptr);
    return update_commit(h, info);
}

}  // extern "C"
