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

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/katz.h"
#include "katz_handle.h"

using namespace katz;

namespace {

constexpr uint64_t CKPT_MAGIC = 0x31504b435a54414bull;  // "KATZCKP1"
constexpr uint32_t CKPT_VERSION = 3;

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

// Consistency of the restored device arrays that the kernels index with
// (the CSR itself is checked by launch_validate_csr):
//   bad[0] perm / inv not inverse permutations of [0, n)
//   bad[1] chunk table inconsistent (chunk_first monotone from 0 to `chunks`,
//          every chunk inside the range of its row)
//   bad[2] a top-k or ranking id outside [0, n)
__global__ void image_check_kernel(const int32_t* __restrict__ perm, const int32_t* __restrict__ inv, int64_t n,
                                   const int64_t* __restrict__ chunk_first, const int32_t* __restrict__ chunk_row,
                                   int64_t row_warp, int64_t chunks, const int32_t* __restrict__ topk_id,
                                   int64_t k_eff, const int32_t* __restrict__ rank_ids, unsigned long long* bad) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long b0 = 0, b1 = 0, b2 = 0;
    for (int64_t i = tid; i < n; i += stride) {
        const int32_t v = perm[i];
        if (v < 0 || (int64_t)v >= n || (int64_t)inv[v] != i) ++b0;
        if (rank_ids) {
            const int32_t w = rank_ids[i];
            if (w < 0 || (int64_t)w >= n) ++b2;
        }
    }
    for (int64_t u = tid; u < row_warp; u += stride)
        if (chunk_first[u + 1] < chunk_first[u]) ++b1;
    if (tid == 0 && (chunk_first[0] != 0 || chunk_first[row_warp] != chunks)) ++b1;
    for (int64_t q = tid; q < chunks; q += stride) {
        const int32_t u = chunk_row[q];
        if (u < 0 || (int64_t)u >= row_warp || chunk_first[u] > q || chunk_first[u + 1] <= q) ++b1;
    }
    for (int64_t q = tid; q < k_eff; q += stride)
        if (topk_id[q] < 0 || (int64_t)topk_id[q] >= n) ++b2;
    if (b0) atomicAdd(&bad[0], b0);
    if (b1) atomicAdd(&bad[1], b1);
    if (b2) atomicAdd(&bad[2], b2);
}

// The header fields a restored handle relies on, checked before any device
// work: sizes, row-mode boundaries, the iteration state against the buffers.
bool header_consistent(const CkptHeader& hd) {
    const int64_t n = hd.n;
    const bool f32_ok = hd.f32_from >= 2;  // INT32_MAX: no FP32 level
    return hd.magic == CKPT_MAGIC && hd.version == CKPT_VERSION &&
           hd.sizes == ((uint32_t)sizeof(Ctrl) | (uint32_t)sizeof(IterParams) << 16) && n >= 1 &&
           n < 0x7fffffffLL && hd.nnz >= 0 && hd.ranked && hd.opts.r_max >= 1 && hd.opts.r_max <= (1 << 20) &&
           hd.walk_slots >= 2 && hd.stride >= n + 1 && hd.row_warp >= 0 && hd.row_warp <= hd.row_octet &&
           hd.row_octet <= hd.row_thread && hd.row_thread <= n && hd.chunks >= 0 && hd.trace_len >= 0 &&
           hd.trace_len <= hd.opts.r_max + 2 && hd.r >= 0 && hd.r <= hd.opts.r_max && hd.k_eff >= 1 &&
           hd.k_eff <= n && f32_ok && hd.sum_depth >= 1 && hd.deg_max >= 0 &&
           hd.D >= hd.deg_max && hd.alpha > 0.0 && hd.alpha * (double)hd.D < 1.0 && hd.criterion >= KATZ_CRIT_TOPK &&
           hd.criterion <= KATZ_CRIT_PAIR && (hd.off64 == 0 || hd.off64 == 1) && (hd.fp32 == 0 || hd.fp32 == 1) &&
           (hd.off64 || n + hd.nnz < 0x7fffffffLL) && hd.ctrl.r == hd.r && hd.ctrl.k_eff >= 0 &&
           hd.ctrl.k_eff <= std::min<int64_t>(n, KATZ_MAX_K) &&
           (hd.ctrl.list_cur == 0 || hd.ctrl.list_cur == 1) && hd.ctrl.f32_from == hd.f32_from &&
           hd.p.n == n && hd.p.stride == hd.stride && hd.p.slots == hd.walk_slots &&
           hd.p.r_max == hd.opts.r_max;
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
    if (!header_consistent(hd)) return KATZ_EINVAL;
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
    // the image's arrays are checked as create checks its input: a CSR with
    // offsets and columns in range, degrees within D, consistent relabelling
    // and chunk table, ids in range; anything else is refused before any
    // kernel gathers through them
    {
        unsigned long long* d_bad = nullptr;
        int64_t* d_degmax = nullptr;
        struct Checks {
            unsigned long long csr[3];
            unsigned long long img[3];
            int64_t degmax;
        };
        static_assert(sizeof(Checks) <= H_SMALL, "pinned scratch");
        Checks& hc = *(Checks*)h->h_small;
        const int64_t span = std::max<int64_t>(std::max<int64_t>(hd.n, hd.nnz), hd.chunks);
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((span + 255) / 256, 152 * 8));
        if ((e = dmalloc(h, &d_bad, 6)) == cudaSuccess && (e = dmalloc(h, &d_degmax, 1)) == cudaSuccess &&
            (e = cudaMemsetAsync(d_bad, 0, 6 * sizeof(unsigned long long), h->stream)) == cudaSuccess &&
            (e = cudaMemsetAsync(d_degmax, 0, sizeof(int64_t), h->stream)) == cudaSuccess &&
            (e = launch_validate_csr(g, d_bad, d_degmax, h->stream)) == cudaSuccess) {
            image_check_kernel<<<blocks, 256, 0, h->stream>>>(g.perm, g.inv, g.n, g.chunk_first, g.chunk_row,
                                                              hd.row_warp, hd.chunks, b.topk_id, hd.ctrl.k_eff,
                                                              hd.has_rank_ids ? h->rank_ids : nullptr, d_bad + 3);
            e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hc.csr, d_bad, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&hc.degmax, d_degmax, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        }
        dfree(h, d_bad);
        dfree(h, d_degmax);
        if (e != cudaSuccess) {
            st = cuda_fail(h, e, "check image");
            katz_destroy(h);
            return st;
        }
        if (hc.csr[0] || hc.csr[1] || hc.img[0] || hc.img[1] || hc.img[2] || hc.degmax > hd.D) {
            katz_destroy(h);
            return KATZ_EINVAL;
        }
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
