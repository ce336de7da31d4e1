// Serving loop for dynamic graphs: update batches arrive over time, each one
// is applied to its graph with Algorithm 2 (Sec. 4) and answered with the
// certified top-k of the graph after it.
//
// The state a request works on (the CSR, the stored walk vectors s_1..s_r,
// the bounds) stays on the device in its handle.  The host side is a small
// scheduler:
//   - submit() copies the batch into host memory the server owns and queues
//     it in arrival order;
//   - admission moves queued requests, oldest first, into one of `slots`
//     staging slots while a slot is free and the admitted updates stay within
//     the update budget; admission starts the host-to-device copy of the batch
//     on the slot's copy stream, so it overlaps whatever runs on the device;
//   - `workers` threads take admitted requests, oldest first.  A request runs
//     in two phases (katz_api.cu): its prepare validates the batch and builds
//     the updated graph into the handle's spare buffers on a second stream,
//     its commit swaps that graph in and repairs the walk vectors on the
//     handle's stream.  On one handle the phases follow arrival order, and the
//     prepare of a request overlaps the repair of the one before it (it may
//     start once that one has swapped its graph in); requests on different
//     handles run at the same time;
//   - a finished request releases its slot, which admits the next one, and
//     its result (status, info, ranking, timestamps) waits for wait().
// Every request sees exactly the graph that the requests on its handle before
// it produced, so its answer does not depend on what else is in flight.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/katz.h"
#include "katz_handle.h"

namespace {

using Clock = std::chrono::steady_clock;

// staging memory of one admitted update: src, dst (int32) and the insert flag,
// in pinned host memory and on the device
constexpr int64_t kStagingBytesPerUpdate = 2 * (2 * (int64_t)sizeof(int32_t) + 1);

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

enum RequestState { WAITING, ADMITTED, RUNNING, DONE };

struct Request {
    uint64_t ticket = 0;
    uint64_t seq = 0;  // arrival order on its handle
    katz_handle* h = nullptr;
    int64_t m = 0;
    std::vector<int32_t> src, dst;
    std::vector<uint8_t> ins;
    RequestState state = WAITING;
    int slot = -1;
    Clock::time_point t_submit, t_admit, t_start, t_done;
    katz_status status = KATZ_OK;
    bool paired = false;  // levels from a two-state pass with the neighbouring request
    katz_info info{};
    std::vector<int32_t> ids;
};

struct Slot {
    int32_t* d_src = nullptr;
    int32_t* d_dst = nullptr;
    uint8_t* d_ins = nullptr;
    int32_t* h_src = nullptr;   // pinned staging
    int32_t* h_dst = nullptr;
    uint8_t* h_ins = nullptr;
    int32_t* h_ids = nullptr;   // pinned, KATZ_MAX_K
    cudaStream_t copy = nullptr;
    cudaEvent_t h2d_done = nullptr;
};

struct Lane {
    int64_t k = 0;
    uint64_t next_seq = 0;      // sequence number of the next submitted request
    uint64_t prep_seq = 0;      // the next request to prepare
    bool preparing = false;     // a prepare is running
    bool swap_pending = false;  // a prepared request has not swapped its graph in yet
    bool repairing = false;     // a swap or repair is running
};

}  // namespace

struct katz_server {
    katz_server_opts opts{};
    int dev = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> waiting;    // submitted, not yet admitted (arrival order)
    std::deque<Request*> admitted;   // admitted, not yet started (admission order)
    std::unordered_map<uint64_t, Request*> requests;  // until wait() collects them
    std::unordered_map<katz_handle*, Lane> lanes;
    std::vector<Slot> slots;
    std::vector<int> free_slots;
    int64_t admitted_updates = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

void free_slot_memory(Slot& s) {
    cudaFree(s.d_src);
    cudaFree(s.d_dst);
    cudaFree(s.d_ins);
    cudaFreeHost(s.h_src);
    cudaFreeHost(s.h_dst);
    cudaFreeHost(s.h_ins);
    cudaFreeHost(s.h_ids);
    if (s.h2d_done) cudaEventDestroy(s.h2d_done);
    if (s.copy) cudaStreamDestroy(s.copy);
    s = Slot{};
}

// Move queued requests into free slots, oldest first (caller holds mu).
void admit_locked(katz_server* s) {
    while (!s->waiting.empty() && !s->free_slots.empty()) {
        Request* q = s->waiting.front();
        if (s->admitted_updates > 0 && s->admitted_updates + q->m > s->opts.admit_updates) break;
        if (s->opts.admit_bytes > 0 && s->admitted_updates > 0 &&
            (s->admitted_updates + q->m) * kStagingBytesPerUpdate > s->opts.admit_bytes)
            break;
        s->waiting.pop_front();
        const int si = s->free_slots.back();
        s->free_slots.pop_back();
        Slot& sl = s->slots[(size_t)si];
        q->slot = si;
        q->state = ADMITTED;
        q->t_admit = Clock::now();
        s->admitted_updates += q->m;
        if (q->m > 0) {
            std::memcpy(sl.h_src, q->src.data(), (size_t)q->m * sizeof(int32_t));
            std::memcpy(sl.h_dst, q->dst.data(), (size_t)q->m * sizeof(int32_t));
            std::memcpy(sl.h_ins, q->ins.data(), (size_t)q->m);
            cudaMemcpyAsync(sl.d_src, sl.h_src, (size_t)q->m * sizeof(int32_t), cudaMemcpyHostToDevice, sl.copy);
            cudaMemcpyAsync(sl.d_dst, sl.h_dst, (size_t)q->m * sizeof(int32_t), cudaMemcpyHostToDevice, sl.copy);
            cudaMemcpyAsync(sl.d_ins, sl.h_ins, (size_t)q->m, cudaMemcpyHostToDevice, sl.copy);
        }
        cudaEventRecord(sl.h2d_done, sl.copy);
        q->src.clear();
        q->src.shrink_to_fit();
        q->dst.clear();
        q->dst.shrink_to_fit();
        q->ins.clear();
        q->ins.shrink_to_fit();
        s->admitted.push_back(q);
        s->cv_work.notify_one();
    }
}

// Phase 1 (the caller holds no lock): the batch, once on the device, is
// validated and the next graph built into the handle's spare buffers.
void prepare_request(katz_server* s, Request* q) {
    Slot& sl = s->slots[(size_t)q->slot];
    katz_handle* h = q->h;
    const int32_t* src = sl.d_src;
    const int32_t* dst = sl.d_dst;
    if (h->opts.inbound && !h->opts.undirected) std::swap(src, dst);  // the handle holds the reverse graph
    katz::update_prepare(h, src, dst, sl.d_ins, q->m, sl.h2d_done);
}

// The ranking of the graph the handle now holds (after a rejected batch the
// graph is unchanged and so is the ranking).
void read_ranking(katz_server* s, Request* q, int64_t k) {
    katz_handle* h = q->h;
    Slot& sl = s->slots[(size_t)q->slot];
    if (q->status == KATZ_OK || q->status == KATZ_EINVAL || q->status == KATZ_EALPHA) {
        const int64_t kk = std::min<int64_t>(k, h->k_eff);
        if (kk > 0 && katz_get_ranking(h, sl.h_ids, kk) == KATZ_OK) q->ids.assign(sl.h_ids, sl.h_ids + kk);
    }
}

// A finished request releases its slot and admits the next (caller holds mu).
void complete_locked(katz_server* s, Request* q) {
    q->t_done = Clock::now();
    q->state = DONE;
    s->free_slots.push_back(q->slot);
    s->admitted_updates -= q->m;
    admit_locked(s);
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

// Phase 2 (the caller holds mu, released while the device works): wait for
// the earlier request's repair, swap the prepared graph in, let the next
// prepare start, then repair and read the ranking.  With pairing, the next
// request of the handle, when it is already admitted, is prepared here on top
// of this one and both are repaired in one two-state pass; this request's
// answer is ready before the second one's graph is swapped in.  Completes the
// request(s) it ran.
void commit_request(katz_server* s, Request* q, int64_t k, std::unique_lock<std::mutex>& lock) {
    Lane& lane = s->lanes[q->h];
    while (lane.repairing) s->cv_done.wait(lock);
    lane.repairing = true;
    katz_handle* h = q->h;
    const bool want_pair = s->opts.pair_batches == 2 || (s->opts.pair_batches == 1 && h->last_repair_whole);
    lock.unlock();
    const katz_status sw = katz::update_swap(h);
    lock.lock();
    lane.swap_pending = false;  // the next prepare reads the graph now current
    Request* q2 = nullptr;
    if (sw == KATZ_OK && want_pair && h->rep.applied && h->opts.undirected && !lane.preparing) {
        for (auto it = s->admitted.begin(); it != s->admitted.end(); ++it)
            if ((*it)->h == h && (*it)->seq == lane.prep_seq) {
                q2 = *it;
                s->admitted.erase(it);
                break;
            }
    }
    if (q2) {  // its prepare runs here; no other worker prepares for this handle meanwhile
        lane.preparing = true;
        q2->state = RUNNING;
        q2->t_start = Clock::now();
    }
    s->cv_work.notify_all();
    lock.unlock();
    bool paired = false;
    if (q2) {
        prepare_request(s, q2);
        lock.lock();
        lane.preparing = false;
        lane.swap_pending = true;
        lane.prep_seq += 1;
        lock.unlock();
        if (katz::pair_possible(h)) {
            paired = true;
            q->paired = true;
            q->status = katz::update_pair_first(h, &q->info);
        }
    }
    if (!paired) q->status = sw != KATZ_OK ? sw : katz::update_repair(h, &q->info);
    read_ranking(s, q, k);
    lock.lock();
    complete_locked(s, q);
    if (!q2) {
        lane.repairing = false;
        s->cv_done.notify_all();
        return;
    }
    lock.unlock();
    const katz_status sw2 = katz::update_swap(h);
    lock.lock();
    lane.swap_pending = false;
    s->cv_work.notify_all();
    lock.unlock();
    q2->status = sw2 != KATZ_OK ? sw2 : (paired ? katz::update_pair_second(h, &q2->info) : katz::update_repair(h, &q2->info));
    q2->paired = paired && h->pair_second_used;
    read_ranking(s, q2, k);
    lock.lock();
    complete_locked(s, q2);
    lane.repairing = false;
    s->cv_done.notify_all();
}

void worker_main(katz_server* s) {
    cudaSetDevice(s->dev);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        Request* q = nullptr;
        for (;;) {
            if (s->stop) return;
            // the oldest admitted request whose handle can start its prepare:
            // its turn in arrival order, no prepare running, no prepared
            // request still waiting to swap its graph in
            for (auto it = s->admitted.begin(); it != s->admitted.end(); ++it) {
                Lane& L = s->lanes[(*it)->h];
                if ((*it)->seq == L.prep_seq && !L.preparing && !L.swap_pending) {
                    q = *it;
                    s->admitted.erase(it);
                    break;
                }
            }
            if (q) break;
            s->cv_work.wait(lock);
        }
        Lane& lane = s->lanes[q->h];
        lane.preparing = true;
        q->state = RUNNING;
        q->t_start = Clock::now();
        const int64_t k = lane.k;
        lock.unlock();
        prepare_request(s, q);
        lock.lock();
        lane.preparing = false;
        lane.swap_pending = true;
        lane.prep_seq += 1;
        commit_request(s, q, k, lock);
    }
}

}  // namespace

extern "C" {

void katz_server_default_opts(katz_server_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->workers = 4;
    o->slots = 8;
    o->slot_updates = 10000;
    o->admit_updates = 0;
    o->admit_bytes = 0;
    o->pair_batches = 1;
    o->reserved = 0;
}

katz_status katz_server_create(katz_server_h* out, const katz_server_opts* opts) {
    if (!out) return KATZ_EINVAL;
    *out = nullptr;
    katz_server_opts o;
    katz_server_default_opts(&o);
    if (opts) o = *opts;
    if (o.workers < 1 || o.workers > 64 || o.slots < 1 || o.slots > 1024 || o.slot_updates < 1 || o.admit_bytes < 0 ||
        o.pair_batches < 0 || o.pair_batches > 2)
        return KATZ_EINVAL;
    if (o.admit_updates <= 0) o.admit_updates = (int64_t)o.slots * o.slot_updates;
    katz_server* s = new katz_server();
    s->opts = o;
    cudaGetDevice(&s->dev);
    s->slots.resize((size_t)o.slots);
    bool ok = true;
    for (int i = 0; i < o.slots && ok; ++i) {
        Slot& sl = s->slots[(size_t)i];
        const size_t m = (size_t)o.slot_updates;
        ok = cudaMalloc((void**)&sl.d_src, m * sizeof(int32_t)) == cudaSuccess &&
             cudaMalloc((void**)&sl.d_dst, m * sizeof(int32_t)) == cudaSuccess &&
             cudaMalloc((void**)&sl.d_ins, m) == cudaSuccess &&
             cudaMallocHost((void**)&sl.h_src, m * sizeof(int32_t)) == cudaSuccess &&
             cudaMallocHost((void**)&sl.h_dst, m * sizeof(int32_t)) == cudaSuccess &&
             cudaMallocHost((void**)&sl.h_ins, m) == cudaSuccess &&
             cudaMallocHost((void**)&sl.h_ids, (size_t)KATZ_MAX_K * sizeof(int32_t)) == cudaSuccess &&
             cudaStreamCreateWithFlags(&sl.copy, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&sl.h2d_done, cudaEventDisableTiming) == cudaSuccess;
        s->free_slots.push_back(o.slots - 1 - i);
    }
    if (!ok) {
        for (Slot& sl : s->slots) free_slot_memory(sl);
        delete s;
        return KATZ_ENOMEM;
    }
    for (int i = 0; i < o.workers; ++i) s->workers.emplace_back(worker_main, s);
    *out = s;
    return KATZ_OK;
}

katz_status katz_server_attach(katz_server_h s, katz_h h, int64_t k) {
    if (!s || !h) return KATZ_EINVAL;
    if (!h->ranked) return katz::fail(h, KATZ_ESTATE, "rank the graph before attaching it");
    if (!h->opts.keep_history) return katz::fail(h, KATZ_ESTATE, "served handles need keep_history = 1");
    if (k < 1 || k > h->k_eff) return katz::fail(h, KATZ_EINVAL, "k must lie in [1, ranked k]");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->lanes.count(h)) return katz::fail(h, KATZ_EINVAL, "handle already attached");
    }
    // device buffers for the largest batch and a rebuilt adjacency with headroom,
    // so that serving allocates nothing per request
    const int64_t nnz_cap = h->g.nnz + h->g.nnz / 16 + 2 * s->opts.slot_updates + 1024;
    const katz_status st = katz::dyn_reserve(h, s->opts.slot_updates, nnz_cap, h->stream);
    if (st != KATZ_OK) return st;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return katz::fail(h, KATZ_ECUDA, "attach sync");
    std::lock_guard<std::mutex> lock(s->mu);
    Lane lane;
    lane.k = k;
    s->lanes[h] = lane;
    return KATZ_OK;
}

katz_status katz_server_submit(katz_server_h s, katz_h h, const int32_t* src, const int32_t* dst,
                               const uint8_t* is_insert, int64_t m, uint64_t* ticket) {
    if (!s || !h || !ticket || m < 0 || m > s->opts.slot_updates) return KATZ_EINVAL;
    if (m > 0 && (!src || !dst || !is_insert)) return KATZ_EINVAL;
    Request* q = new Request();
    q->h = h;
    q->m = m;
    q->src.assign(src, src + m);
    q->dst.assign(dst, dst + m);
    q->ins.assign(is_insert, is_insert + m);
    q->t_submit = Clock::now();
    std::lock_guard<std::mutex> lock(s->mu);
    if (!s->lanes.count(h)) {
        delete q;
        return KATZ_ESTATE;
    }
    q->ticket = s->next_ticket++;
    q->seq = s->lanes[h].next_seq++;
    s->requests[q->ticket] = q;
    s->waiting.push_back(q);
    admit_locked(s);
    *ticket = q->ticket;
    return KATZ_OK;
}

katz_status katz_server_wait(katz_server_h s, uint64_t ticket, int64_t timeout_ms, int32_t* ids_out,
                             katz_request_result* res) {
    if (!s) return KATZ_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->requests.find(ticket);
    if (it == s->requests.end()) return KATZ_EINVAL;
    Request* q = it->second;
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (q->state != DONE) {
        if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && q->state != DONE)
            return KATZ_ETIMEOUT;
    }
    if (res) {
        std::memset(res, 0, sizeof(*res));
        res->status = q->status;
        res->paired = q->paired ? 1 : 0;
        res->k = (int64_t)q->ids.size();
        res->info = q->info;
        res->queue_ms = ms_between(q->t_submit, q->t_admit);
        res->wait_ms = ms_between(q->t_admit, q->t_start);
        res->service_ms = ms_between(q->t_start, q->t_done);
        res->latency_ms = ms_between(q->t_submit, q->t_done);
    }
    if (ids_out && !q->ids.empty()) std::memcpy(ids_out, q->ids.data(), q->ids.size() * sizeof(int32_t));
    s->requests.erase(it);
    delete q;
    return KATZ_OK;
}

// Algorithm 2 without blocking the caller: the handle's private server (two
// workers, so the prepare of a batch overlaps the repair of the one before it)
katz_status katz_submit_update_batch(katz_h h, const int32_t* src, const int32_t* dst, const uint8_t* is_insert,
                                     int64_t m, uint64_t* ticket) {
    if (!h || !ticket || m < 0 || (m > 0 && (!src || !dst || !is_insert))) return KATZ_EINVAL;
    std::lock_guard<std::mutex> lock(h->async_mu);
    if (!h->async) {
        katz_status st = katz::update_allowed(h);
        if (st != KATZ_OK) return st;
        katz_server_opts o;
        katz_server_default_opts(&o);
        o.workers = 2;
        o.slots = 4;
        o.slot_updates = std::max<int64_t>(m, o.slot_updates);
        katz_server* s = nullptr;
        if ((st = katz_server_create(&s, &o)) != KATZ_OK) return st;
        if ((st = katz_server_attach(s, h, h->k_eff)) != KATZ_OK) {
            katz_server_destroy(s);
            return st;
        }
        h->async = s;
    }
    if (m > h->async->opts.slot_updates) return KATZ_EINVAL;
    return katz_server_submit(h->async, h, src, dst, is_insert, m, ticket);
}

katz_status katz_poll(katz_h h, uint64_t ticket, katz_info* info) {
    if (!h) return KATZ_EINVAL;
    katz_server* s = nullptr;
    {
        std::lock_guard<std::mutex> lock(h->async_mu);
        s = h->async;
    }
    if (!s) return KATZ_ESTATE;  // nothing was submitted
    katz_request_result res;
    const katz_status st = katz_server_wait(s, ticket, 0, nullptr, &res);
    if (st == KATZ_ETIMEOUT) return KATZ_EBUSY;
    if (st != KATZ_OK) return KATZ_ESTATE;  // unknown or collected ticket
    if (info) *info = res.info;
    return (katz_status)res.status;
}

void katz_server_destroy(katz_server_h s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (std::thread& t : s->workers) t.join();
    for (auto& kv : s->requests) delete kv.second;
    for (auto& kv : s->lanes) cudaStreamSynchronize(kv.first->stream);
    for (Slot& sl : s->slots) {
        if (sl.copy) cudaStreamSynchronize(sl.copy);
        free_slot_memory(sl);
    }
    delete s;
}

}  // extern "C"
