// Checkpoint and restore of a ranked handle: the state the paper's dynamic
// algorithm keeps between batches (Sec. 4: omega_1..omega_r as the scaled
// walk history, c_r, the active set M, r) together with the graph, so that a
// restored handle continues exactly where the original stood.
//
// The image is the handle's device state in its internal layout (relabelled
// CSR, walk slots, bounds, control block) behind a fixed header; it is tied
// to this library version (magic + version + struct sizes are checked).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <vector>

#include "../../include/katz.h"
#include "katz_handle.h"

using namespace katz;

namespace {

constexpr uint64_t CKPT_MAGIC = 0x31504b435a54414bull;  // "KATZCKP1"
constexpr uint32_t CKPT_VERSION = 2;

struct CkptHeader {
    uint64_t magic;
    uint32_t version;
    uint32_t sizes;  // sizeof(Ctrl) | sizeof(IterParams) << 16, a layout check
    katz_opts opts;
    int64_t n, nnz, D, deg_max, stride, k_eff;
    int64_t row_warp, row_octet, row_thread, chunks;
    int32_t off64, fp32, sum_depth, f32_from, walk_slots, r, converged, criterion, ranked, has_rank_ids;
    double alpha, gamma, eps;
    float last_ms;
    int32_t trace_len;
    IterParams p;
    Ctrl ctrl;
};

// Walks the image in one fixed order: counts bytes, writes them, or reads them.
struct Image {
    enum Mode { COUNT, WRITE, READ } mode;
    katz_handle* h;
    unsigned char* buf;
    uint64_t cap, pos = 0;
    bool ok = true;

    void host(void* p, uint64_t bytes) {
        if (mode != COUNT && pos + bytes > cap) ok = false;
        if (ok && mode == WRITE) std::memcpy(buf + pos, p, bytes);
        if (ok && mode == READ) std::memcpy(p, buf + pos, bytes);
        pos += bytes;
    }
    void dev(void* d, uint64_t bytes) {
        if (mode != COUNT && pos + bytes > cap) ok = false;
        if (ok && bytes && mode == WRITE)
            ok = cudaMemcpyAsync(buf + pos, d, bytes, cudaMemcpyDeviceToHost, h->stream) == cudaSuccess;
        if (ok && bytes && mode == READ)
            ok = cudaMemcpyAsync(d, buf + pos, bytes, cudaMemcpyHostToDevice, h->stream) == cudaSuccess;
        pos += bytes;
    }
};

// the device arrays of a handle, in image order (sizes from the header)
void walk_arrays(Image& im, katz_handle* h, const CkptHeader& hd) {
    const uint64_t n = (uint64_t)hd.n;
    DeviceGraph& g = h->g;
    IterBuffers& b = h->b;
    im.dev(g.rowptr, (n + 1) * (hd.off64 ? 8 : 4));
    im.dev(g.col, (uint64_t)hd.nnz * 4);
    im.dev(g.perm, n * 4);
    im.dev(g.inv, n * 4);
    im.dev(g.chunk_first, ((uint64_t)hd.row_warp + 1) * 8);
    im.dev(g.chunk_row, (uint64_t)hd.chunks * 4);
    im.dev(b.walk, (uint64_t)hd.walk_slots * (uint64_t)hd.stride * 8);
    im.dev(b.c, n * 8);
    if (hd.fp32) im.dev(b.c32, n * 8);
    if (hd.fp32) im.dev(b.s32, n * 4);  // the first FP32 level's input (an update may recompute that level)
    im.dev(b.lb, n * 8);
    im.dev(b.ub, n * 8);
    im.dev(b.active, n);
    im.dev(b.topk_id, (uint64_t)KATZ_MAX_K * 4);
    im.dev(b.topk_l, (uint64_t)KATZ_MAX_K * 8);
    im.dev(b.topk_u, (uint64_t)KATZ_MAX_K * 8);
    im.dev(b.trace, ((uint64_t)hd.opts.r_max + 2) * 8);
    if (hd.has_rank_ids) im.dev(h->rank_ids, n * 4);
}

void fill_header(katz_handle* h, CkptHeader& hd) {
    std::memset(&hd, 0, sizeof(hd));
    hd.magic = CKPT_MAGIC;
    hd.version = CKPT_VERSION;
    hd.sizes = (uint32_t)sizeof(Ctrl) | (uint32_t)sizeof(IterParams) << 16;
    hd.opts = h->opts;
    hd.opts.cuda_stream = nullptr;
    const DeviceGraph& g = h->g;
    hd.n = g.n;
    hd.nnz = g.nnz;
    hd.D = h->D;
    hd.deg_max = h->deg_max;
    hd.stride = h->stride;
    hd.k_eff = h->k_eff;
    hd.row_warp = g.layout.row_warp;
    hd.row_octet = g.layout.row_octet;
    hd.row_thread = g.layout.row_thread;
    hd.chunks = g.layout.chunks;
    hd.off64 = g.off64;
    hd.fp32 = h->fp32;
    hd.sum_depth = h->sum_depth;
    hd.f32_from = h->f32_from;
    hd.walk_slots = h->walk_slots;
    hd.r = h->r;
    hd.converged = h->converged;
    hd.criterion = h->criterion;
    hd.ranked = h->ranked;
    hd.has_rank_ids = h->criterion == KATZ_CRIT_RANKING && h->rank_ids != nullptr;
    hd.alpha = h->alpha;
    hd.gamma = h->gamma;
    hd.eps = h->eps;
    hd.last_ms = h->last_ms;
    hd.trace_len = (int32_t)h->trace.size();
    hd.p = h->p;
}

katz_status image_of(katz_handle* h, Image& im) {
    CkptHeader hd;
    fill_header(h, hd);
    if (im.mode == Image::WRITE &&
        cudaMemcpyAsync(&hd.ctrl, h->b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return cuda_fail(h, cudaGetLastError(), "copy ctrl");
    if (im.mode == Image::WRITE && cudaStreamSynchronize(h->stream) != cudaSuccess)
        return cuda_fail(h, cudaGetLastError(), "sync");
    im.host(&hd, sizeof(hd));
    im.host(h->trace.data(), h->trace.size() * sizeof(int64_t));
    walk_arrays(im, h, hd);
    if (im.mode == Image::WRITE && cudaStreamSynchronize(h->stream) != cudaSuccess)
        return cuda_fail(h, cudaGetLastError(), "sync");
    return im.ok ? KATZ_OK : fail(h, KATZ_EINVAL, "checkpoint buffer too small");
}

}  // namespace

extern "C" {

katz_status katz_checkpoint_size(katz_h h, uint64_t* bytes) {
    if (!h || !bytes) return KATZ_EINVAL;
    if (!h->ranked) return fail(h, KATZ_ESTATE, "checkpoints hold a ranked handle");
    Image im{Image::COUNT, h, nullptr, 0};
    const katz_status st = image_of(h, im);
    *bytes = im.pos;
    return st;
}

katz_status katz_checkpoint(katz_h h, void* buf, uint64_t bytes) {
    if (!h || !buf) return KATZ_EINVAL;
    if (!h->ranked) return fail(h, KATZ_ESTATE, "checkpoints hold a ranked handle");
    Image im{Image::WRITE, h, (unsigned char*)buf, bytes};
    return image_of(h, im);
}

katz_status katz_restore(katz_h* out, const void* buf, uint64_t bytes, const katz_opts* opts) {
    if (!out || !buf) return KATZ_EINVAL;
    *out = nullptr;
    CkptHeader hd;
    if (bytes < sizeof(hd)) return KATZ_EINVAL;
    std::memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != CKPT_MAGIC || hd.version != CKPT_VERSION ||
        hd.sizes != ((uint32_t)sizeof(Ctrl) | (uint32_t)sizeof(IterParams) << 16) || hd.n < 1 || hd.nnz < 0 ||
        hd.walk_slots < 2 || hd.stride < hd.n + 1 || hd.row_warp < 0 || hd.row_warp > hd.n || hd.chunks < 0 ||
        hd.trace_len < 0 || hd.trace_len > hd.opts.r_max + 2 || !hd.ranked)
        return KATZ_EINVAL;
    katz_handle* h = new katz_handle();
    h->opts = hd.opts;
    h->opts.cuda_stream = opts ? opts->cuda_stream : nullptr;
    katz_status st = init_handle_runtime(h);
    if (st != KATZ_OK) {
        katz_destroy(h);
        return st;
    }
    DeviceGraph& g = h->g;
    IterBuffers& b = h->b;
    g.n = hd.n;
    g.nnz = hd.nnz;
    g.off64 = hd.off64 != 0;
    g.layout = make_layout(hd.n, hd.row_warp, hd.row_octet, hd.row_thread, hd.chunks);
    h->fp32 = hd.fp32 != 0;
    h->D = hd.D;
    h->deg_max = hd.deg_max;
    h->sum_depth = hd.sum_depth;
    const uint64_t n = (uint64_t)hd.n;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, uint64_t count) {
        if (e == cudaSuccess) e = dmalloc(h, p, (size_t)count);
    };
    if (g.off64) A((int64_t**)&g.rowptr, n + 1);
    else A((int32_t**)&g.rowptr, n + 1);
    A(&g.col, (uint64_t)hd.nnz);
    A(&g.perm, n);
    A(&g.inv, n);
    A(&g.chunk_first, (uint64_t)hd.row_warp + 1);
    A(&g.chunk_row, (uint64_t)hd.chunks + 1);
    A(&g.chunk_part, 3 * ((uint64_t)hd.chunks + 1));
    h->chunk_row_cap = hd.chunks + 1;
    h->chunk_part_cap = hd.chunks + 1;
    if (e != cudaSuccess) {
        st = cuda_fail(h, e, "cudaMalloc graph");
        katz_destroy(h);
        return st;
    }
    // iteration buffers as the handle's settings make them; the image must match
    if ((st = ensure_iter_buffers(h)) != KATZ_OK || h->walk_slots != hd.walk_slots || h->stride != hd.stride) {
        katz_destroy(h);
        return st != KATZ_OK ? st : KATZ_EINVAL;
    }
    if (hd.has_rank_ids) A(&h->rank_ids, n);
    if (e == cudaSuccess && (st = alloc_rank_scratch(h)) != KATZ_OK) {
        katz_destroy(h);
        return st;
    }
    if (e != cudaSuccess) {
        st = cuda_fail(h, e, "cudaMalloc");
        katz_destroy(h);
        return st;
    }
    hd.ctrl.list_ready = 0;  // the active list is not in the image: rebuilt from the flags
    hd.ctrl.n_list_next = 0;
    Image im{Image::READ, h, (unsigned char*)buf, bytes};
    im.pos = sizeof(hd);
    h->trace.resize((size_t)hd.trace_len);
    im.host(h->trace.data(), h->trace.size() * sizeof(int64_t));
    walk_arrays(im, h, hd);
    if (im.ok) im.ok = cudaMemcpyAsync(b.ctrl, &hd.ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream) == cudaSuccess;
    if (!im.ok || im.pos != bytes || cudaStreamSynchronize(h->stream) != cudaSuccess) {
        katz_destroy(h);
        return KATZ_EINVAL;
    }
    h->p = hd.p;
    h->k_eff = hd.k_eff;
    h->f32_from = hd.f32_from;
    h->r = hd.r;
    h->converged = hd.converged;
    h->criterion = hd.criterion;
    h->alpha = hd.alpha;
    h->gamma = hd.gamma;
    h->eps = hd.eps;
    h->last_ms = hd.last_ms;
    h->ranked = true;
    *out = h;
    return KATZ_OK;
}

}  // extern "C"
