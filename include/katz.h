/*
 * katz.h - C ABI of the GB300 (sm_103a) certified Katz ranking library.
 *
 * Method: van der Grinten, Bergamini, Green, Bader, Meyerhenke, "Scalable
 * Katz Ranking Computation in Large Static and Dynamic Graphs" (ESA 2018).
 *
 *   Katz centrality (Eq. 1): c(v) = sum_{i>=1} alpha^i omega_i(v), omega_i(v)
 *   the number of walks of length i that start at v.  The library never
 *   forms c exactly; it iterates the walk recurrence of Eq. (5),
 *   omega_i(v) = sum_{v->x} omega_{i-1}(x), and keeps per-node bounds
 *   l_r(v) <= c(v) <= u_r(v) (Sec. 3.1, Theorem 1) until the top-k
 *   criterion holds: the k nodes with the highest lower bounds are
 *   eps-separated (Eq. 3) from each other and from every other node
 *   (Algorithm 1 with its converged() procedure).
 *
 * Internally the walk vectors are stored scaled, s_i = alpha^i omega_i, so
 * that they stay in [0, 1] when alpha * deg_max < 1.
 *
 * Conventions shared by every entry point
 *   - Every function returns a katz_status; KATZ_OK is 0.  No function
 *     throws or aborts.  On failure the handle is left as it was before the
 *     call (an update batch is applied completely or not at all) and
 *     katz_last_error() describes the failure.
 *   - Pointers are plain host or device addresses; the library tells them
 *     apart with CUDA unified addressing unless a flag says otherwise.
 *     Output buffers are owned by the caller and must hold the stated
 *     number of elements.  Input arrays are read during the call only; the
 *     library keeps its own device copies.
 *   - Node ids are int32 in [0, n).  Graph arrays are CSR: rowptr (int64,
 *     n+1 entries, rowptr[0] = 0, non-decreasing) and col (int32, nnz =
 *     rowptr[n] entries).  An undirected graph is passed as its symmetric
 *     CSR (each edge as two arcs; Sec. 2.1).
 *   - A handle is used by one host thread at a time, except that
 *     katz_submit_update_batch and katz_poll may be called from any thread.
 *     All device work is ordered on the handle's CUDA stream
 *     (katz_opts.cuda_stream, or a stream the library creates).
 */
#ifndef KATZ_H_
#define KATZ_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct katz_handle* katz_h;

typedef enum {
    KATZ_OK = 0,
    KATZ_EINVAL = 1,      /* bad argument, malformed graph or batch */
    KATZ_EALPHA = 2,      /* alpha * deg_bound >= 1 (Theorem 1 needs alpha < 1/deg_max) */
    KATZ_ENOMEM = 3,      /* device or pinned host allocation failed */
    KATZ_ECUDA = 4,       /* a CUDA runtime call failed */
    KATZ_ENOTCONV = 5,    /* r_max iterations ran without meeting the criterion */
    KATZ_EPRECISION = 6,  /* FP32-certified mode cannot separate the remaining pairs */
    KATZ_ETIMEOUT = 7,    /* a bounded wait expired */
    KATZ_EBUSY = 8,       /* no free slot / request still running */
    KATZ_ESTATE = 9       /* call not valid in the handle's state (e.g. no ranking yet) */
} katz_status;

/* Arithmetic of the walk vectors. */
enum {
    KATZ_FP64 = 0,          /* s_i in FP64, as the paper (which implies FP64) */
    KATZ_FP32_CERT = 1,     /* s_i in FP32, bounds widened by a rigorous rounding term;
                               KATZ_EPRECISION when the widening stalls the certificate */
    KATZ_FP32_CERT_AUTO = 2 /* as KATZ_FP32_CERT, but a stalled ranking is recomputed with
                               FP64 levels (katz_info.escalated = 1) instead of failing */
};

typedef struct {
    int32_t precision;     /* KATZ_FP64 (default), KATZ_FP32_CERT or KATZ_FP32_CERT_AUTO */
    int32_t undirected;    /* 1 (default): the CSR is symmetric; use the undirected lower
                              bound l_r = c_r + alpha^{r+1} omega_r (Sec. 3.1) */
    int32_t keep_history;  /* 1: keep s_1..s_r (needed by katz_apply_update_batch and
                              katz_get_walk for i < r-1); 0 (default): two live levels */
    int32_t r_max;         /* iteration cap, default 128 */
    int64_t deg_bound;     /* D >= deg_max used in gamma = D/(1 - alpha D); 0 (default):
                              deg_max of the input graph */
    double frontier_abort_frac; /* dynamic update: fall back to a full level when the
                              affected set exceeds this fraction of n (Sec. 4; default 0.05) */
    void* cuda_stream;     /* cudaStream_t to run on; NULL: the library creates one */
    int32_t use_graph;     /* 1 (default): run the iteration as a CUDA graph with a
                              device-side while loop; 0: host-driven loop */
    int32_t inbound;       /* directed handles: 1 ranks by inbound Katz (walks that end at
                              v, Sec. 2.1), which is the outbound Katz of the reverse
                              graph: the library reverses the CSR on the device at create.
                              Update batches still name arcs src -> dst of the graph as
                              given.  0 (default): outbound.  Ignored when undirected. */
    int32_t profile;       /* 1: time every walk-count SpMV launch with CUDA events on the
                              handle's stream (katz_info.spmv_ms); forces the host-driven loop */
    int32_t fp32_from;     /* KATZ_FP32_CERT: first walk level computed in FP32 (>= 2);
                              0 (default): chosen on the device once the FP32 rounding
                              widening is predicted to stay below eps/16 */
    int32_t offsets64;     /* 1: keep the row offsets as int64 from the start.  0 (default):
                              int32 while n + nnz < 2^31 - 1, int64 above; an update batch
                              that takes a handle past that limit moves it to int64 offsets
                              (one extra (n+1)-entry array during that batch) */
    int32_t l2_fetch_bytes; /* > 0 (32, 64 or 128): during each katz_rank_static, katz_rank and
                              katz_apply_update_batch call on the handle, the current context's
                              maximum L2 fetch granularity (cudaLimitMaxL2FetchGranularity) is
                              set to this many bytes, and set back to the value
                              cudaDeviceGetLimit reported before the call when the call
                              returns.  The limit is context-wide: other work of the process
                              that runs during the call sees it too.  0 (default): the
                              library leaves the limit alone.  On two GB300 machines, 64 changed
                              a gather level with a 1 GB walk vector by -12% and by +4%;
                              walk vectors within a few times L2 ran fastest at the default */
    int32_t locality;      /* internal order of the rows of degree <= 16 (the low end of the
                              degree-class order): 1 orders them inside each degree class by
                              their anchor, the smallest internal id among their neighbours,
                              so that the walk values one hub row gathers from them sit
                              together and a line fetched from DRAM serves several gathers;
                              -1 keeps them in original-id order; 0 (default): 1 when
                              n >= 2^25 (walk vectors several times larger than L2), else -1.
                              Results are the same bits either way. */
    int32_t reserved;      /* set to 0 */
} katz_opts;

typedef struct {
    int32_t r;             /* iterations performed (walk length reached) */
    int32_t converged;     /* 1 if the top-k criterion holds at r */
    int64_t active;        /* |M| after the last convergence check */
    int64_t k;             /* effective k = min(k, n) */
    double alpha;          /* attenuation used */
    double gamma;          /* D / (1 - alpha D) */
    double time_ms;        /* device time of the call (CUDA events) */
    int64_t nnz;           /* arcs the walk recurrence visited per iteration */
    int32_t fp32_levels;   /* FP32-certified mode: levels carried in FP32 */
    int32_t full_levels;   /* dynamic update: levels recomputed for every node */
    int64_t affected;      /* dynamic update: nodes whose walk counts were recomputed */
    double spmv_ms;        /* profile = 1: summed device time of the SpMV launches of
                              levels 2..r (level 1 is the degree vector: A 1 = deg, no
                              walk values are gathered) */
    int64_t launches;      /* kernels this call launched */
    int32_t spmv_launches; /* SpMV launches of levels 2..r this call made */
    int32_t escalated;     /* KATZ_FP32_CERT_AUTO: 1 if the FP32-certified run stalled and the
                              ranking was recomputed with FP64 levels */
} katz_info;

/* Fill *opts with the defaults listed above. */
void katz_default_opts(katz_opts* opts);

/* Human-readable name of a status code (static string). */
const char* katz_status_string(katz_status s);

/*
 * Create a handle for the graph (n, rowptr, col) and copy it to device
 * memory the library owns.  rowptr/col may be host or device pointers.
 * Validates rowptr (monotone, rowptr[0] = 0, rowptr[n] = nnz) and every
 * col entry in [0, n); self-loops are accepted (a self-loop is a walk of
 * length 1).  opts may be NULL for the defaults.
 * Errors: KATZ_EINVAL (n < 1, nnz < 0, malformed CSR), KATZ_ENOMEM, KATZ_ECUDA.
 */
katz_status katz_create_csr(katz_h* out, int64_t n, int64_t nnz, const int64_t* rowptr,
                            const int32_t* col, const katz_opts* opts);

/* Release the handle and all device memory it owns (NULL is ignored). */
void katz_destroy(katz_h h);

/* Description of the last failure on this handle ("" if none). */
const char* katz_last_error(katz_h h);

/*
 * Algorithm 1 (Sec. 3.2) with the top-k criterion (Sec. 3.1).
 * alpha: attenuation; alpha <= 0 selects alpha = 1/(1 + D) (Sec. 3.1).
 * k: 1 <= k; clamped to n; at most KATZ_MAX_K.
 * eps > 0: absolute separation slack of Eq. (3).
 * Runs iterations r = 1, 2, ... (s_r = alpha A s_{r-1}, c_r = c_{r-1} + s_r,
 * l_r, u_r, then converged()) until the criterion holds or r_max is hit.
 * The ranking and bounds stay in the handle (katz_get_ranking/_bounds).
 * info may be NULL.
 * Errors: KATZ_EINVAL, KATZ_EALPHA, KATZ_ENOTCONV (the state at r_max is
 * still readable), KATZ_EPRECISION (FP32-certified mode), KATZ_ECUDA.
 */
#define KATZ_MAX_K 8192
katz_status katz_rank_static(katz_h h, double alpha, int64_t k, double eps, katz_info* info);

/* Stopping criteria (Sec. 3.1). */
enum {
    KATZ_CRIT_TOPK = 0,     /* the top-k nodes eps-separated from each other and from all others */
    KATZ_CRIT_RANKING = 1,  /* every pair of nodes eps-separated: the top-k criterion with k = n */
    KATZ_CRIT_SCORE = 2,    /* u_r(v) - l_r(v) < eps for every node */
    KATZ_CRIT_PAIR = 3      /* two given nodes eps-separated */
};

/*
 * Algorithm 1 (Sec. 3.2) with any stopping criterion of Sec. 3.1.
 * KATZ_CRIT_TOPK: the same as katz_rank_static(h, alpha, k, eps, info).
 * The others run on FP64 handles and keep every node active:
 *   KATZ_CRIT_RANKING: each iteration sorts all n nodes by (l desc, id asc)
 *     and checks every adjacent pair (Eq. 3); afterwards katz_get_ranking
 *     returns the full certified order (k up to n);
 *   KATZ_CRIT_SCORE: stops once u_r - l_r < eps at every node; the bounds
 *     (katz_get_bounds) then give every score to within eps, and there is
 *     no ranking (katz_get_ranking returns KATZ_ESTATE);
 *   KATZ_CRIT_PAIR: pair = host array of two distinct node ids; stops once
 *     they are eps-separated; katz_get_ranking(h, ids, 2) returns them in
 *     their certified order.
 * k is read by KATZ_CRIT_TOPK only, pair by KATZ_CRIT_PAIR only.
 * katz_apply_update_batch continues the top-k criterion only.
 * Errors: KATZ_EINVAL, KATZ_EALPHA, KATZ_ENOTCONV, KATZ_ESTATE (another
 * criterion on an FP32-certified handle), KATZ_ENOMEM, KATZ_ECUDA.
 */
katz_status katz_rank(katz_h h, double alpha, int32_t criterion, int64_t k, const int32_t* pair, double eps,
                      katz_info* info);

/*
 * The certified top-k after the last rank/update call: ids[0..k) in
 * decreasing order of lower bound (ties by smaller id).  k must equal the
 * effective k of that call or be smaller (a prefix).
 * Errors: KATZ_ESTATE (no ranking yet), KATZ_EINVAL.
 */
katz_status katz_get_ranking(katz_h h, int32_t* ids, int64_t k);

/*
 * Per-node bounds at the current r: lower[v] = l_r(v), upper[v] = u_r(v)
 * (Alg. 1), each n doubles, host or device.  err (nullable): in
 * KATZ_FP32_CERT mode the width of the rounding interval per node: lower[v]
 * and upper[v] each lie within err[v] of l_r(v) and u_r(v) evaluated in exact
 * arithmetic (lower[v] below, upper[v] above them); zeros in FP64 mode.  Any
 * pointer may be NULL to skip it.
 */
katz_status katz_get_bounds(katz_h h, double* lower, double* upper, double* err);

/*
 * The scaled walk vector s_i = alpha^i omega_i (n doubles, host or device)
 * for 1 <= i <= r; i < r-1 requires keep_history.
 */
katz_status katz_get_walk(katz_h h, int32_t i, double* s_out);

/* Number of active nodes |M| after each iteration 1..r (cap entries). */
katz_status katz_get_trace(katz_h h, int64_t* active_per_iter, int32_t cap);

/*
 * Algorithm 2 (Sec. 4): apply a batch of m edge updates (insert if
 * is_insert[e] != 0, else delete) to the graph of a handle that has ranked
 * with keep_history = 1 under the top-k criterion, repair the stored walk
 * vectors s_1..s_r, recompute the bounds, re-derive the active set and
 * continue iterating until the top-k criterion holds again.
 * FP32-certified handles repair each level in its own arithmetic (FP64 up
 * to the switch level, FP32 from it on) and summation order; a batch that
 * makes a row's sum longer than any before widens the rounding-error bound
 * of every level.  If that widening stalls the certificate the call returns
 * KATZ_EPRECISION (KATZ_FP32_CERT; the bounds stay valid) or, under
 * KATZ_FP32_CERT_AUTO, ranks the updated graph again with FP64 levels
 * (info->escalated = 1) and the handle continues in FP64.
 * On an undirected handle an update is the edge {src[e], dst[e]} (both arcs
 * change); on a directed one (opts.undirected = 0) it is the arc
 * src[e] -> dst[e] alone (Sec. 2.1), so a batch may name a -> b and b -> a.
 * Preconditions (checked, Sec. 4): inserted edges are absent, deleted
 * edges are present, no edge appears twice in the batch (unordered pairs
 * when undirected, ordered when directed), no self-loops, and no row
 * exceeds the degree bound D afterwards (out-degrees when directed).
 * Arrays may be host or device pointers.
 * Errors: KATZ_EINVAL (precondition), KATZ_EALPHA (a row would exceed D),
 * KATZ_ESTATE (no ranking / no history), KATZ_EPRECISION, KATZ_ENOTCONV,
 * KATZ_ENOMEM, KATZ_ECUDA.
 */
katz_status katz_apply_update_batch(katz_h h, const int32_t* src, const int32_t* dst,
                                    const uint8_t* is_insert, int64_t m, katz_info* info);

/*
 * Algorithm 2 without blocking the caller: queue a batch for h and return at
 * once with *ticket.  Batches submitted to one handle are applied in
 * submission order, each exactly as katz_apply_update_batch applies it (the
 * graph after the batches before it, re-certified top-k); the validation and
 * rebuild of one batch overlap the repair of the one before it.  src, dst and
 * is_insert are host arrays, copied before the call returns.  The first
 * submitted batch sets up a private serving queue for h (the serving loop
 * below, two workers) whose slots take batches of up to max(m, 10^4)
 * updates; a later batch above that size returns KATZ_EINVAL.
 * katz_submit_update_batch and katz_poll may be called from any thread.
 * Between a submit and the katz_poll that reports its batch finished, the
 * caller makes no other call on h; katz_destroy finishes the batch that is
 * running and drops the queued ones.
 * Errors: KATZ_EINVAL (arguments, batch size), KATZ_ESTATE (as
 * katz_apply_update_batch), KATZ_ENOMEM, KATZ_ECUDA.
 */
katz_status katz_submit_update_batch(katz_h h, const int32_t* src, const int32_t* dst,
                                     const uint8_t* is_insert, int64_t m, uint64_t* ticket);

/*
 * The outcome of a submitted batch.  KATZ_EBUSY: still queued or running.
 * Otherwise the batch has finished: *info (nullable) is what
 * katz_apply_update_batch would have written, and the return value is its
 * status (KATZ_EINVAL: the batch was rejected and changed nothing).  Each
 * ticket is reported finished once; an unknown or already collected ticket
 * gives KATZ_ESTATE.
 */
katz_status katz_poll(katz_h h, uint64_t ticket, katz_info* info);

/*
 * The number conversions of the FP32-certified levels, for tests and
 * diagnostics: out[i] = in[i] rounded to binary32 (to nearest, ties to even;
 * subnormal results kept, 0 below half the smallest subnormal) and
 * back[i] = out[i] widened exactly to binary64, computed on the device with
 * the integer routines the SpMV epilogue uses.  in holds n non-negative finite
 * values; in, out and back are device pointers (n elements each).  Runs on
 * the default stream and returns when done.
 * Errors: KATZ_EINVAL (NULL or host pointer, n < 0), KATZ_ECUDA.
 */
katz_status katz_convert_f64_f32(const double* in, int64_t n, float* out, double* back);

/*
 * Checkpoint and restore of a ranked handle (the state Sec. 4 keeps between
 * batches: the walk history s_1..s_r, c_r, the active set M and r, with the
 * graph and the last ranking).  katz_checkpoint_size gives the bytes of the
 * image, katz_checkpoint writes it into a host buffer of that size, and
 * katz_restore creates a handle on the current device from such a buffer
 * (opts: only cuda_stream is read; NULL: a stream of its own).  The restored
 * handle continues where the original stood: the same ranking, bounds and
 * walks, and later calls give the same results.  The image is this library
 * version's internal layout, not an exchange format.  katz_restore checks it
 * before any kernel reads it, as katz_create_csr checks its input: the header
 * fields against each other, the CSR (offsets monotone from 0 to nnz, column
 * ids in range, degrees within the degree bound), the relabelling (an inverse
 * pair of permutations), the hub-row chunk table and the stored ids.
 * Errors: KATZ_EINVAL (NULL pointer, buffer too small, not an image of this
 * version, or an inconsistent image), KATZ_ESTATE (handle not ranked),
 * KATZ_ENOMEM, KATZ_ECUDA.
 */
katz_status katz_checkpoint_size(katz_h h, uint64_t* bytes);
katz_status katz_checkpoint(katz_h h, void* buf, uint64_t bytes);
katz_status katz_restore(katz_h* out, const void* buf, uint64_t bytes, const katz_opts* opts);

/*
 * Serving loop for dynamic graphs (Sec. 4 applied to a stream of batches).
 *
 * A server takes update batches for one or more attached handles as they
 * arrive and answers each with the certified top-k of its graph after that
 * batch.  Requests on one handle run in arrival order, each on the graph the
 * previous ones left; requests on different handles run at the same time on
 * their handles' streams.  Submitted batches wait in arrival order until one
 * of `slots` staging slots is free and the admitted requests stay within
 * `admit_updates` updates and `admit_bytes` bytes of staging memory;
 * admission copies the batch to the device on the slot's own
 * stream, overlapping the work in flight.  `workers` host threads drive the
 * admitted requests through the two phases of katz_apply_update_batch and
 * katz_get_ranking.  The first phase validates a batch and builds the updated
 * graph into the handle's spare buffers on a second stream of the handle;
 * the second swaps that graph in and repairs the walk vectors on the
 * handle's stream.  On one handle the first phase of a request overlaps the
 * second phase of the one before it, so with two or more workers the batches
 * of one graph are pipelined.
 * Attaching a handle reserves its device buffers for batches of up to
 * slot_updates updates (and adjacency headroom), so a request allocates
 * nothing on the device unless its graph grows past that headroom.
 */
typedef struct katz_server* katz_server_h;

typedef struct {
    int32_t workers;        /* host threads driving requests (default 4) */
    int32_t slots;          /* requests admitted at once (default 8) */
    int64_t slot_updates;   /* largest batch accepted, in updates (default 10000) */
    int64_t admit_updates;  /* admitted updates in total at most (0: slots * slot_updates) */
    int64_t admit_bytes;    /* staging memory of the admitted requests in bytes at most: a
                               request of m updates holds 18 m bytes (its batch in pinned host
                               memory and on the device) from admission to completion
                               (0: no limit beyond admit_updates) */
    int32_t pair_batches;   /* two queued batches of one undirected graph in one pass: the walk
                               levels of both graph states are computed together (one gathered
                               line serves both), and each batch is answered with its own
                               certified ranking, bit for bit that of applying the batches one
                               by one.  1 (default): when the graph's last repair recomputed
                               whole levels (the case where one pass for two pays off);
                               2: whenever two batches are queued; 0: never */
    int32_t reserved;       /* set to 0 */
} katz_server_opts;

typedef struct {
    int32_t status;         /* katz_status of the request (KATZ_EINVAL: batch rejected,
                               graph and ranking unchanged) */
    int32_t paired;         /* 1: its walk levels came from one two-state pass with the
                               request before or after it on the same handle */
    int64_t k;              /* ids written to ids_out */
    katz_info info;         /* katz_apply_update_batch's info */
    double queue_ms;        /* submit -> admitted into a slot */
    double wait_ms;         /* admitted -> a worker started it */
    double service_ms;      /* started -> ranking copied to the host (with pipelined batches
                               this includes waiting for the earlier request's repair) */
    double latency_ms;      /* submit -> ranking copied to the host */
} katz_request_result;

void katz_server_default_opts(katz_server_opts* opts);

/* Create a server on the current device (opts NULL: defaults).
 * Errors: KATZ_EINVAL, KATZ_ENOMEM. */
katz_status katz_server_create(katz_server_h* out, const katz_server_opts* opts);

/*
 * Serve handle h, answering with its top k (1 <= k <= the ranked k).  h must
 * have ranked with keep_history = 1 (any precision, directed or undirected) and
 * should own its stream (katz_opts.cuda_stream = NULL), so that its work can
 * overlap other handles'.  While attached, h belongs to the server: the caller
 * makes no other call on it until the server is destroyed.
 * Errors: KATZ_EINVAL, KATZ_ESTATE, KATZ_ENOMEM, KATZ_ECUDA.
 */
katz_status katz_server_attach(katz_server_h s, katz_h h, int64_t k);

/*
 * Queue a batch of m updates for h, read as katz_apply_update_batch reads
 * them (host arrays, copied before the call returns; m <= slot_updates).
 * *ticket identifies the request.
 * Errors: KATZ_EINVAL, KATZ_ESTATE (h not attached).
 */
katz_status katz_server_submit(katz_server_h s, katz_h h, const int32_t* src, const int32_t* dst,
                               const uint8_t* is_insert, int64_t m, uint64_t* ticket);

/*
 * Wait up to timeout_ms (0: just look) for a request.  Once it has finished,
 * writes its ranking to ids_out (host, k entries; NULL skips it) and its
 * result to res (nullable), forgets the ticket and returns KATZ_OK; the
 * request's own outcome is res->status.  Each ticket is collected by one
 * call.  Errors: KATZ_ETIMEOUT (not finished yet), KATZ_EINVAL (unknown
 * ticket).
 */
katz_status katz_server_wait(katz_server_h s, uint64_t ticket, int64_t timeout_ms, int32_t* ids_out,
                             katz_request_result* res);

/* Finish the requests that are running, drop the queued ones, release the
 * server (NULL is ignored).  Attached handles stay valid. */
void katz_server_destroy(katz_server_h s);

/*
 * katz_certify_topk_noalloc - the paper has no counterpart to this entry
 * point.  It is for callers that must not have a library allocate device
 * memory: a process whose own caching allocator holds all device memory, a
 * latency-bound loop that cannot take the device-wide wait of cudaFree, a
 * host that forbids device allocation by the code it loads.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *
 * Given per-node bounds lower[v] <= c(v) <= upper[v] for v in [0, n) (two
 * arrays of n doubles in device memory, e.g. from katz_get_bounds; no NaN),
 * writes ids_out[0..k) = the k nodes with the largest lower bounds in
 * decreasing order (ties by smaller id) and *certified_out = 1 if the top-k
 * criterion that katz_rank_static stops on holds for these bounds (each
 * adjacent top-k pair and the k-th node against every other node
 * eps-separated), else 0.  ids_out (k int32) and certified_out (one int32)
 * are device memory owned by the caller.
 *
 * Working memory: one fixed array of at most 420 KiB in the library's device image,
 * present on every device that loads the library until the process exits.
 * It holds at most KATZ_MAX_K candidates, so the limits are
 * 1 <= k <= KATZ_MAX_K, k <= n <= 2^31 - 2, eps > 0: anything beyond them
 * returns KATZ_EINVAL before any work is queued.
 *
 * The work is queued on cuda_stream (NULL: the default stream) and the call
 * returns without waiting for it.  The first call on a device, with that
 * device current, looks up the array's device address and raises the sort
 * kernel's shared-memory limit; make that first call before any stream
 * capture begins on that device.  Every call on a device uses the same
 * array, which keeps the contents of the last call; each call clears what
 * must start at zero.  Calls whose work overlaps on the GPU (streams with no
 * ordering between them) race on the array and give wrong results.
 * No handle: errors are reported by the return value alone.
 * Errors: KATZ_EINVAL (NULL pointer, sizes above the limits), KATZ_ECUDA
 * (device lookup or a launch failed).
 */
katz_status katz_certify_topk_noalloc(const double* lower, const double* upper, int64_t n, int64_t k,
                                      double eps, int32_t* ids_out, int32_t* certified_out,
                                      void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* KATZ_H_ */
