// lscan_server.cu -- continuous-batching scan service on one GPU.
//
// Not in the paper (which times one scan at a time, Section 5): this is the
// serving pattern built on the same single-pass kernel.
//
//  * HBM budget.  At creation the server takes one device allocation of the
//    whole budget: a pool from which request outputs (and client buffers,
//    lscan_server_alloc) are carved, plus a small reserve for per-stream
//    scratch (status words, array descriptors).  No cudaMalloc happens while
//    serving.
//  * Admission.  A request whose output the server must allocate is
//    admitted at submission when the pool can hold its output and nothing
//    of its lane waits before it; otherwise it waits in its lane's FIFO queue
//    and is admitted in arrival order as earlier outputs are released.
//  * Continuous batching.  One scheduler thread per stream keeps that
//    stream's two launch slots busy (the second batch of a stream is queued
//    behind the first, so the GPU never waits for the host between
//    batches).  Whenever a slot is idle it takes the oldest admitted request
//    of its lane, gathers every admitted request of the same (op, dtype,
//    inclusive) up to a tile budget, and issues ONE persistent MODE_LIST
//    launch over them (each array keeps its own carry chain).  Batches are
//    chosen under the server lock and launched after it is released (one
//    copy of the array list, the kernel, two events), so the streams'
//    schedulers issue in parallel.  Different kinds run on different streams
//    and overlap on the device; requests arriving while batches run join the
//    next launch.
//  * Size-class lanes.  Requests of at most small_max elements (2^14 by
//    default) of the kinds the resident kernel scans take the resident lane
//    (resident_kernel.cu): the submitting thread writes each into a ring in
//    host memory mapped for the device, where a persistent kernel on
//    reserve_sms SMs (4 by default) claims it, scans it with one CTA and
//    writes its done word; a resident worker thread relaunches the kernel
//    when it has ended (idle) and retires finished requests.  Other
//    requests form bulk batches capped at bulk_cap tiles (32768 by
//    default), launched for the SMs the resident lane leaves.  FIFO order
//    holds within each lane.
//  * Completion.  Each scheduler polls the end event of its stream's older
//    in-flight batch (cudaEventQuery; batches on a stream finish in issue
//    order); nothing host-side sits in the stream, so the batch queued
//    behind it starts the moment the kernel before it ends.  Launch and
//    completion times are read from CUDA events and mapped onto the host
//    clock, so latencies are device-accurate.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/lscan.h"
#include "kernel_table.h"
#include "lscan_internal.h"
#include "resident.h"
#include "scan_common.h"

namespace lscan {
namespace {

constexpr size_t kPoolAlign = 256;
constexpr int64_t kMaxBatchTiles = 65536;   // ~1 GiB of 16 KiB tiles per launch
constexpr int kSlotsPerStream = 2;          // a second batch queues behind the first
constexpr int64_t kMinTileBytes = 8192;     // smallest input tile of any config
constexpr int64_t kMaxBatchRequests = 4096;
constexpr int64_t kDefaultSmallMax = int64_t{1} << 14;  // elements
constexpr int64_t kDefaultBulkCap = 32768;              // tiles per bulk batch
constexpr int kDefaultReserveSms = 4;                   // SMs for the resident lane
constexpr int kResCtasPerSm = 2;                        // resident CTAs per reserved SM
constexpr int64_t kResRing = 4096;                      // resident ring entries
constexpr uint64_t kResIdleNs = 20000000;               // resident CTAs leave after 20 ms idle
constexpr int kLanes = 2;                               // 0 bulk, 1 resident (small)
// A stream whose other slot is still running forms its next batch only once
// that batch would be worth a launch (half the tile cap) or its oldest
// request has waited this long: the batch would queue behind the running
// one anyway, and waiting lets it grow.
constexpr double kQueuedBatchDelayUs = 30.0;

// Takes m, trying for a short while before blocking: the threads on a small
// request's path (submitters, the resident worker) would otherwise sleep in
// the kernel for microseconds whenever another thread holds the lock for a
// moment.  Plain try_lock polling, no processor-specific pause.
std::unique_lock<std::mutex> spin_lock(std::mutex &m) {
    for (int i = 0; i < 2048; ++i)
        if (m.try_lock()) return std::unique_lock<std::mutex>(m, std::adopt_lock);
    return std::unique_lock<std::mutex>(m);
}

double now_us(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0)
        .count();
}

// First-fit allocator over [0, size) with coalescing.
class PoolAllocator {
   public:
    void init(size_t size) {
        free_.clear();
        free_[0] = size;
        used_ = 0;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = (bytes + kPoolAlign - 1) / kPoolAlign * kPoolAlign;
        if (bytes == 0) bytes = kPoolAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                sizes_[*off] = bytes;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    bool release(size_t off) {
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return false;
        size_t bytes = s->second;
        sizes_.erase(s);
        used_ -= bytes;
        size_t start = off;
        auto nx = free_.lower_bound(start);
        if (nx != free_.end() && nx->first == start + bytes) {
            bytes += nx->second;
            free_.erase(nx);
        }
        auto pv = free_.lower_bound(start);
        if (pv != free_.begin()) {
            --pv;
            if (pv->first + pv->second == start) {
                start = pv->first;
                bytes += pv->second;
                free_.erase(pv);
            }
        }
        free_[start] = bytes;
        return true;
    }
    size_t used() const { return used_; }

   private:
    std::map<size_t, size_t> free_;   // offset -> bytes
    std::map<size_t, size_t> sizes_;  // allocated offset -> bytes
    size_t used_ = 0;
};

struct Request {
    uint64_t id = 0;
    int op = 0, dtype = 0, inclusive = 1;
    const void *x = nullptr;
    void *y = nullptr;
    bool y_owned = false;  // output allocated by the server
    int64_t n = 0;
    lscan_req_stats st{};
    bool done = false;
    int64_t tag = -1;  // index in a replayed trace, -1 otherwise
    int lane = 0;      // 0 bulk, 1 resident (small)
    int kind = -1;     // resident lane: the kernel's kind id
    int64_t res_idx = -1;  // resident lane: its ring entry number
};

struct Batch {
    std::vector<Request *> reqs;
};

// A batch chosen under the lock, launched after it is released.
struct Pending {
    int slot = -1;
    LaunchSpec ls;
    size_t list_bytes = 0;  // first-tile indices + descriptors to copy
    bool empty = false;     // only empty requests: no kernel
};

struct Slot {
    cudaStream_t stream = nullptr;
    uint32_t *ctl = nullptr;
    uint64_t *status = nullptr;
    // one batch's array list: first-tile indices (n_seg + 1 int64) followed
    // by the descriptors, filled in pinned host memory and moved to the
    // device by ONE copy
    uint8_t *d_list = nullptr;
    uint8_t *h_list = nullptr;   // pinned
    uint32_t *h_err = nullptr;   // pinned, mapped: the kernel's last CTA
                                 // moves the batch's error word here
    uint32_t *d_err = nullptr;   // its device address
    Batch *inflight = nullptr;
    uint64_t launches = 0;
    bool owns_stream = false;
    int lane = 0;  // which lane's requests this slot launches
    cudaEvent_t ev_start = nullptr, ev_done = nullptr;
};

}  // namespace
}  // namespace lscan

using namespace lscan;

struct lscan_server {
    int device = 0;
    size_t budget = 0;
    uint8_t *mem = nullptr;  // the one device allocation
    uint8_t *pool = nullptr;
    size_t pool_size = 0;
    PoolAllocator alloc;
    std::vector<Slot> slots;
    std::deque<Request *> waiting[kLanes];   // not admitted (output not allocated)
    std::deque<Request *> admitted[kLanes];  // ready to launch
    int64_t small_max = kDefaultSmallMax;    // lane 1: n <= small_max (mu)
    int64_t bulk_cap = kDefaultBulkCap;      // tiles per lane-0 batch (mu)
    int64_t slot_words = 0;                  // status words per tile, reserved
    // resident lane: ring and control words in host memory mapped for the
    // device, the claim counter in device memory
    ResReq *res_ring = nullptr;       // kResRing entries
    uint64_t *res_ctl = nullptr;      // [0] published, [8] stop (as uint32)
    uint64_t *res_done = nullptr;     // kResRing done words
    unsigned long long *res_claim = nullptr;
    uint64_t res_published = 0;       // entries written (mu)
    cudaStream_t res_stream = nullptr;
    cudaEvent_t res_end = nullptr;    // after the running resident kernel
    std::vector<Request *> res_out;   // published, not yet done (resident worker)
    std::vector<Request *> res_new;   // published by a submitter, not yet in res_out (mu)
    std::unordered_map<uint64_t, Request *> reqs;
    std::mutex mu;     // requests, pool, slots
    std::mutex cb_mu;  // wake-up counter only
    std::condition_variable cv_sched, cv_done;
    uint64_t kicks = 0;                // bumped by every kick (cb_mu)
    int sleepers = 0;                  // schedulers waiting on cv_sched (cb_mu)
    std::vector<std::thread> workers;  // one scheduler per stream
    int n_str = 0;                     // streams (bulk + small lane)
    int reserve_sms = kDefaultReserveSms;  // SMs kept for the resident lane (mu)
    bool stop = false;
    bool hold = false;  // admit and queue, launch nothing (mu)
    uint64_t next_id = 1;
    std::chrono::steady_clock::time_point t0;
    cudaEvent_t ref_ev = nullptr;
    double ref_us = 0;
    bool collecting = false;          // a replay is running (mu)
    std::vector<Request *> finished;  // replayed requests done, not yet collected (mu)
};

namespace lscan {
namespace {

// Widest status slot (64-bit words per tile) of any batched-list kernel: the
// status words a launch slot reserves per tile.
int64_t list_slot_words() {
    ensure_kernels_registered();
    int64_t w = 1;
    for (int k = 0; k < kNumKinds; ++k)
        for (int v = 0; v < kNumVariants; ++v)
            if (g_kernels[k][MODE_LIST][v].fn && g_kernels[k][MODE_LIST][v].car_words > w)
                w = g_kernels[k][MODE_LIST][v].car_words;
    return w;
}

// Mark a request done.  Caller holds mu.
void finish_locked(lscan_server *srv, Request *r) {
    r->done = true;
    if (srv->collecting && r->tag >= 0) srv->finished.push_back(r);
}

int out_dtype_of(int op, int dtype) {
    return (op == LSCAN_ADD && dtype == LSCAN_BF16) ? LSCAN_F32 : dtype;
}

bool same_kind(const Request *a, const Request *b) {
    return a->op == b->op && a->dtype == b->dtype && a->inclusive == b->inclusive;
}

// Try to admit waiting requests (FIFO within a lane; the small lane first)
// into the pool.  Caller holds mu.
void admit_locked(lscan_server *srv) {
    for (int lane = kLanes - 1; lane >= 0; --lane) {
        auto &q = srv->waiting[lane];
        while (!q.empty()) {
            Request *r = q.front();
            size_t off = 0;
            const size_t bytes =
                static_cast<size_t>(r->n) * dtype_size(out_dtype_of(r->op, r->dtype));
            if (!srv->alloc.alloc(bytes, &off)) break;  // head-of-line waits
            r->y = srv->pool + off;
            r->y_owned = true;
            r->st.y = r->y;
            q.pop_front();
            r->st.admit_us = now_us(srv->t0);
            srv->admitted[lane].push_back(r);
        }
    }
}

double event_us(lscan_server *srv, cudaEvent_t ev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, srv->ref_ev, ev) != cudaSuccess) return now_us(srv->t0);
    return srv->ref_us + 1000.0 * ms;
}

// Finish a slot's batch.  Caller holds mu.
void retire_locked(lscan_server *srv, int si, bool cuda_ok) {
    Slot &sl = srv->slots[si];
    Batch *b = sl.inflight;
    if (!b) return;
    const double t_start = event_us(srv, sl.ev_start);
    const double t_done = event_us(srv, sl.ev_done);
    const uint32_t err = *reinterpret_cast<volatile uint32_t *>(sl.h_err);
    for (Request *r : b->reqs) {
        r->st.launch_us = t_start;
        r->st.done_us = t_done;
        if (r->st.status == LSCAN_OK)
            r->st.status = !cuda_ok ? LSCAN_ERR_CUDA : err ? LSCAN_ERR_TIMEOUT : LSCAN_OK;
        r->st.batch_requests = static_cast<int32_t>(b->reqs.size());
        finish_locked(srv, r);
    }
    delete b;
    sl.inflight = nullptr;
    srv->cv_done.notify_all();
}

// Choose one batch for an idle slot and fill the slot's pinned array list.
// Caller holds mu; the CUDA calls happen later in issue_batch, outside it.
bool prepare_batch_locked(lscan_server *srv, int si, Pending *pd, bool queued,
                          bool *deferred) {
    Slot &sl = srv->slots[si];
    auto &admitted = srv->admitted[sl.lane];
    const int64_t cap = sl.lane == 0 ? srv->bulk_cap : kMaxBatchTiles;
    *deferred = false;
    // plan with the head's kind (dummy disjoint aligned pointers, n = 1); a
    // head whose kind is not built fails and the next one is tried
    LaunchSpec ls;
    Request *head = nullptr;
    while (!admitted.empty()) {
        head = admitted.front();
        if (plan_scan(head->op, head->dtype, head->inclusive, reinterpret_cast<void *>(256),
                      reinterpret_cast<void *>(4096), 1, nullptr, MODE_LIST, nullptr, 0,
                      &ls) == LSCAN_OK)
            break;
        head->st.status = LSCAN_ERR_UNSUPPORTED;
        admitted.pop_front();
        finish_locked(srv, head);
        srv->cv_done.notify_all();
        head = nullptr;
    }
    if (head == nullptr) return false;
    const int tile = planned_tile(ls);
    if (queued) {
        // behind a running batch: wait until this one is worth a launch
        const double t = now_us(srv->t0);
        if (t - head->st.admit_us < kQueuedBatchDelayUs) {
            int64_t want = 0;
            for (const Request *r : admitted) {
                if (same_kind(r, head)) want += (r->n + tile - 1) / tile;
                if (2 * want >= cap) break;
            }
            if (2 * want < cap) {
                *deferred = true;
                return false;
            }
        }
    }
    Batch *b = new Batch();
    int64_t tiles = 0;
    bool aligned = true;
    // the list: first-tile indices [0, n_seg] then the descriptors; both
    // regions are written once n_seg is known (indices first, so the
    // descriptors go to a staging area at the end and move down)
    SegDesc *desc_tmp = reinterpret_cast<SegDesc *>(
        sl.h_list + (kMaxBatchRequests + 1) * sizeof(int64_t));
    int64_t *first = reinterpret_cast<int64_t *>(sl.h_list);
    for (auto it = admitted.begin(); it != admitted.end();) {
        Request *r = *it;
        if (!same_kind(r, head)) {
            ++it;
            continue;
        }
        const int64_t rt = (r->n + tile - 1) / tile;
        if (!b->reqs.empty() && (tiles + rt > cap ||
                                 static_cast<int64_t>(b->reqs.size()) >= kMaxBatchRequests))
            break;
        desc_tmp[b->reqs.size()] = SegDesc{r->x, r->y, r->n};
        first[b->reqs.size()] = tiles;
        tiles += rt;
        aligned = aligned && (reinterpret_cast<uintptr_t>(r->x) % 16 == 0) &&
                  (reinterpret_cast<uintptr_t>(r->y) % 16 == 0);
        b->reqs.push_back(r);
        it = admitted.erase(it);
    }
    const int64_t nseg = static_cast<int64_t>(b->reqs.size());
    first[nseg] = tiles;
    const size_t first_b = static_cast<size_t>(nseg + 1) * sizeof(int64_t);
    memmove(sl.h_list + first_b, desc_tmp, static_cast<size_t>(nseg) * sizeof(SegDesc));
    if (!aligned) ls.variant = 0;
    ls.mode = MODE_LIST;
    ls.offsets = reinterpret_cast<const int64_t *>(sl.d_list);
    ls.segs = sl.d_list + first_b;
    ls.n_seg = nseg;
    ls.list_tiles = tiles;
    ls.n = 0;
    ls.err_host = sl.d_err;
    // bulk batches leave CTA slots of reserve_sms SMs free for small ones
    if (srv->small_max > 0) ls.reserve_sms = srv->reserve_sms;
    const double t = now_us(srv->t0);
    for (Request *r : b->reqs) {
        r->st.launch_us = t;
        ls.n += r->n;
    }
    sl.inflight = b;
    pd->slot = si;
    pd->ls = ls;
    pd->list_bytes = first_b + static_cast<size_t>(nseg) * sizeof(SegDesc);
    pd->empty = tiles == 0;
    return true;
}

// Launch a prepared batch: one copy of its array list, the kernel between
// two events (the second is the one the scheduler polls).  Only the slot's
// stream scheduler touches a slot, so no lock is held.
void issue_batch(lscan_server *srv, const Pending &pd) {
    Slot &sl = srv->slots[pd.slot];
    Batch *b = sl.inflight;
    *reinterpret_cast<volatile uint32_t *>(sl.h_err) = 0u;
    if (pd.empty) {  // only empty requests
        cudaEventRecord(sl.ev_start, sl.stream);
        cudaEventRecord(sl.ev_done, sl.stream);
        return;
    }
    cudaMemcpyAsync(sl.d_list, sl.h_list, pd.list_bytes, cudaMemcpyHostToDevice, sl.stream);
    if (++sl.launches >= (1ull << 30) - 1) {  // keep the epoch tag from wrapping
        cudaMemsetAsync(sl.ctl, 0, CTL_WORDS * sizeof(uint32_t), sl.stream);
        cudaMemsetAsync(sl.status, 0, kMaxBatchTiles * srv->slot_words * sizeof(uint64_t),
                        sl.stream);
        sl.launches = 0;
    }
    cudaEventRecord(sl.ev_start, sl.stream);
    DevBuffers db{sl.ctl, sl.status};
    const lscan_status st = launch_scan(pd.ls, db, sl.stream);
    cudaEventRecord(sl.ev_done, sl.stream);
    if (st != LSCAN_OK)
        for (Request *r : b->reqs) r->st.status = st;
}

void kick(lscan_server *srv);

// One scheduler thread per stream: it owns that stream's two launch slots
// (the second batch queues behind the first, so the stream never waits for
// the host between batches), sleeps while neither is in flight and its lane
// has nothing to launch, and otherwise polls the older in-flight batch's end
// event.  It takes the lock only to retire a batch, admit waiting requests
// and choose the next batch; the CUDA calls are made after releasing it, so
// the streams' schedulers issue in parallel and never block submissions.
void worker_main(lscan_server *srv, int stream_idx) {
    cudaSetDevice(srv->device);
    const int si[2] = {stream_idx, stream_idx + srv->n_str};
    const int lane = srv->slots[si[0]].lane;
    uint64_t seen = 0;
    std::vector<Pending> todo;
    std::deque<int> order;  // in-flight slots in issue order (they finish in it)
    bool deferred = false;  // a batch was held back: look again without a kick
    double last_look = 0.0;
    while (true) {
        bool kicked;
        {
            std::unique_lock<std::mutex> lk(srv->cb_mu);
            if (order.empty() && srv->kicks == seen) {
                ++srv->sleepers;
                srv->cv_sched.wait(lk, [&] { return srv->kicks != seen; });
                --srv->sleepers;
            }
            kicked = srv->kicks != seen;
            seen = srv->kicks;
        }
        int done_slot = -1;
        bool cuda_ok = true;
        if (!order.empty()) {
            const cudaError_t q = cudaEventQuery(srv->slots[order.front()].ev_done);
            if (q != cudaErrorNotReady) {
                done_slot = order.front();
                cuda_ok = q == cudaSuccess;
                order.pop_front();
            }
        }
        // a held-back batch is looked at again every few microseconds
        const bool recheck = deferred && now_us(srv->t0) - last_look > 4.0;
        if (!kicked && done_slot < 0 && !recheck) {
            std::this_thread::yield();
            continue;
        }
        last_look = now_us(srv->t0);
        todo.clear();
        bool leave = false, more = false;
        deferred = false;
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            if (done_slot >= 0) retire_locked(srv, done_slot, cuda_ok);
            admit_locked(srv);
            if (!srv->hold || srv->stop)
                for (int s : si) {
                    if (srv->slots[s].inflight) continue;
                    Pending pd;
                    bool dfr = false;
                    const bool queued = !order.empty() || !todo.empty();
                    if (prepare_batch_locked(srv, s, &pd, queued && !srv->stop, &dfr))
                        todo.push_back(pd);
                    deferred = deferred || dfr;
                }
            leave = srv->stop && order.empty() && todo.empty() && srv->admitted[lane].empty();
            // requests this stream did not take: wake the others only if one
            // of them has a free slot (or the resident lane is asleep)
            bool idle_slot = false;
            for (const Slot &o : srv->slots) idle_slot = idle_slot || !o.inflight;
            more = (!srv->admitted[0].empty() && idle_slot) ||
                   (!srv->admitted[1].empty() && srv->res_out.empty());
        }
        for (const Pending &pd : todo) {
            issue_batch(srv, pd);
            order.push_back(pd.slot);
        }
        if (more) kick(srv);
        if (leave) break;
    }
}

// Release/acquire accesses of the resident lane's words in mapped host
// memory (the device reads and writes them with .sys-scope accesses).
void store_release(uint64_t *p, uint64_t v) { __atomic_store_n(p, v, __ATOMIC_RELEASE); }
uint64_t load_acquire(const uint64_t *p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }

// Writes admitted small requests into the resident lane's ring and makes
// them visible to the device kernel (srv->mu held, so the published counter
// only grows): called by the resident worker and by the submitting thread
// itself, so that a small request reaches the device without a hand-off
// between host threads.  The resident worker adopts them from res_new.
void publish_resident_locked(lscan_server *srv, double t) {
    auto &q = srv->admitted[1];
    bool any = false;
    while (!q.empty() && (!srv->hold || srv->stop)) {
        const uint64_t idx = srv->res_published;
        if (idx >= static_cast<uint64_t>(kResRing) &&
            load_acquire(srv->res_done + (idx % kResRing)) != idx - kResRing + 1)
            break;  // that entry's earlier request is still running
        Request *r = q.front();
        q.pop_front();
        ResReq &e = srv->res_ring[idx % kResRing];
        e.x = r->x;
        e.y = r->y;
        e.n = r->n;
        e.kind = r->kind;
        e.inclusive = r->inclusive;
        r->res_idx = static_cast<int64_t>(idx);
        r->st.launch_us = t;
        srv->res_published = idx + 1;
        srv->res_new.push_back(r);
        any = true;
    }
    if (any) store_release(srv->res_ctl, srv->res_published);  // entries first
}

// The resident lane's scheduler: publishes admitted small requests to the
// ring as the submitting threads do (an entry is reused only after the
// request that held it is done), keeps the resident kernel running while
// work is outstanding (it leaves by itself after kResIdleNs without work; a
// request published as it left is picked up by the next launch), and
// retires requests whose done word has been written.  Their launch time is
// the publication, their completion the first poll that saw the done word
// (host clock).
void resident_main(lscan_server *srv) {
    cudaSetDevice(srv->device);
    uint64_t seen = 0;
    bool running = false;
    double last_query = 0.0;
    auto &out = srv->res_out;
    while (true) {
        bool kicked;
        {
            std::unique_lock<std::mutex> lk(srv->cb_mu);
            if (out.empty() && srv->kicks == seen) {
                ++srv->sleepers;
                srv->cv_sched.wait(lk, [&] { return srv->kicks != seen; });
                --srv->sleepers;
            }
            kicked = srv->kicks != seen;
            seen = srv->kicks;
        }
        // the kernel ended (idle): it is launched again below if needed (the
        // driver is asked at most every 50 us)
        const double tq = now_us(srv->t0);
        if (running && tq - last_query > 50.0) {
            last_query = tq;
            if (cudaEventQuery(srv->res_end) != cudaErrorNotReady) running = false;
        }
        // done words need no lock (only this thread changes res_out)
        bool any_done = false;
        for (const Request *r : out)
            if (load_acquire(srv->res_done + (r->res_idx % kResRing)) ==
                static_cast<uint64_t>(r->res_idx) + 1) {
                any_done = true;
                break;
            }
        if (!kicked && !any_done && (running || out.empty())) {
            std::this_thread::yield();
            continue;
        }
        bool leave = false;
        size_t n_done = 0;
        {
            auto lk = spin_lock(srv->mu);
            // retire
            const double t = now_us(srv->t0);
            for (size_t i = 0; i < out.size();) {
                Request *r = out[i];
                const uint64_t d = load_acquire(srv->res_done + (r->res_idx % kResRing));
                if (d == static_cast<uint64_t>(r->res_idx) + 1) {
                    r->st.done_us = t;
                    r->st.batch_requests = 1;
                    finish_locked(srv, r);
                    out[i] = out.back();
                    out.pop_back();
                    ++n_done;
                } else {
                    ++i;
                }
            }
            if (n_done) srv->cv_done.notify_all();
            admit_locked(srv);
            publish_resident_locked(srv, t);
            // take over what this thread and the submitters published
            out.insert(out.end(), srv->res_new.begin(), srv->res_new.end());
            srv->res_new.clear();
            leave = srv->stop && out.empty() && srv->admitted[1].empty();
        }
        if (!out.empty() && !running) {
            ResParams rp;
            rp.ring = srv->res_ring;
            rp.published = srv->res_ctl;
            rp.stop = reinterpret_cast<const uint32_t *>(srv->res_ctl + 1);
            rp.claim = srv->res_claim;
            rp.done = srv->res_done;
            rp.ring_size = kResRing;
            rp.idle_ns = kResIdleNs;
            int sms = 1;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, srv->device);
            int reserve = srv->reserve_sms > 0 ? srv->reserve_sms : 1;
            if (reserve > sms) reserve = sms;
            if (launch_resident(rp, reserve * kResCtasPerSm, srv->res_stream) == LSCAN_OK &&
                cudaEventRecord(srv->res_end, srv->res_stream) == cudaSuccess)
                running = true;
        }
        if (leave) break;
    }
    // tell a still-running kernel to leave, and wait for it
    __atomic_store_n(reinterpret_cast<uint32_t *>(srv->res_ctl + 1), 1u, __ATOMIC_RELEASE);
    cudaStreamSynchronize(srv->res_stream);
}

// Wake every scheduler (never blocks on srv->mu).
void kick(lscan_server *srv) {
    bool wake;
    {
        std::lock_guard<std::mutex> lk(srv->cb_mu);
        ++srv->kicks;
        wake = srv->sleepers > 0;  // the others poll the counter
    }
    if (wake) srv->cv_sched.notify_all();
}

void release_request_locked(lscan_server *srv, Request *r) {
    if (r->y_owned) srv->alloc.release(static_cast<uint8_t *>(r->y) - srv->pool);
    srv->reqs.erase(r->id);
    delete r;
}

}  // namespace
}  // namespace lscan

extern "C" {

lscan_server *lscan_server_create(size_t hbm_budget_bytes, int n_streams) {
    if (n_streams < 1 || n_streams > 64) return nullptr;
    lscan_server *srv = new lscan_server();
    srv->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        delete srv;
        return nullptr;
    }
    auto up = [](size_t b) { return (b + kPoolAlign - 1) / kPoolAlign * kPoolAlign; };
    const size_t ctl_b = up(CTL_WORDS * sizeof(uint32_t));
    srv->slot_words = list_slot_words();
    const size_t st_b = up(kMaxBatchTiles * srv->slot_words * sizeof(uint64_t));
    const size_t list_b = up((kMaxBatchRequests + 1) * sizeof(int64_t) +
                             kMaxBatchRequests * sizeof(SegDesc));
    const size_t slot_b = ctl_b + st_b + list_b;
    // n_streams streams, two slots each; then the resident lane's claim
    // counter
    const size_t reserve = slot_b * n_streams * kSlotsPerStream + kPoolAlign;
    if (hbm_budget_bytes < reserve + (size_t{1} << 20)) {
        delete srv;
        return nullptr;
    }
    srv->budget = hbm_budget_bytes;
    if (cudaMalloc(&srv->mem, hbm_budget_bytes) != cudaSuccess) {
        delete srv;
        return nullptr;
    }
    cudaMemset(srv->mem, 0, reserve);
    srv->pool = srv->mem + reserve;
    srv->pool_size = hbm_budget_bytes - reserve;
    srv->alloc.init(srv->pool_size);
    // slots: [0, n) one per stream, then a second slot for each stream
    const int n_str = n_streams;
    const int n_slots = n_str * kSlotsPerStream;
    int prio_least = 0, prio_greatest = 0;
    cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    srv->slots.resize(n_slots);
    for (int i = 0; i < n_slots; ++i) {
        Slot &sl = srv->slots[i];
        uint8_t *base = srv->mem + i * slot_b;
        sl.ctl = reinterpret_cast<uint32_t *>(base);
        sl.status = reinterpret_cast<uint64_t *>(base + ctl_b);
        sl.d_list = base + ctl_b + st_b;
        sl.lane = 0;
        if (i < n_str)
            cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, prio_least);
        else
            sl.stream = srv->slots[i - n_str].stream;  // shares the stream
        sl.owns_stream = i < n_str;
        // the list is built in place: indices, then a staging area for the
        // descriptors at the end (one list's worth of each)
        cudaMallocHost(&sl.h_list, (kMaxBatchRequests + 1) * sizeof(int64_t) +
                                       2 * kMaxBatchRequests * sizeof(SegDesc));
        cudaHostAlloc(&sl.h_err, sizeof(uint32_t), cudaHostAllocMapped);
        if (sl.h_err) {
            *sl.h_err = 0;
            cudaHostGetDevicePointer(reinterpret_cast<void **>(&sl.d_err), sl.h_err, 0);
        }
        cudaEventCreate(&sl.ev_start);
        cudaEventCreate(&sl.ev_done);
    }
    // resident lane: ring, control and done words in mapped host memory
    srv->res_claim = reinterpret_cast<unsigned long long *>(
        srv->mem + slot_b * n_streams * kSlotsPerStream);
    cudaHostAlloc(&srv->res_ring, kResRing * sizeof(ResReq), cudaHostAllocMapped);
    cudaHostAlloc(&srv->res_ctl, 128, cudaHostAllocMapped);
    cudaHostAlloc(&srv->res_done, kResRing * sizeof(uint64_t), cudaHostAllocMapped);
    if (srv->res_ctl) memset(srv->res_ctl, 0, 128);
    if (srv->res_done) memset(srv->res_done, 0, kResRing * sizeof(uint64_t));
    cudaStreamCreateWithPriority(&srv->res_stream, cudaStreamNonBlocking, prio_greatest);
    cudaEventCreateWithFlags(&srv->res_end, cudaEventDisableTiming);
    cudaEventCreate(&srv->ref_ev);
    cudaEventRecord(srv->ref_ev, srv->slots[0].stream);
    cudaEventSynchronize(srv->ref_ev);
    srv->ref_us = now_us(srv->t0);
    if (cudaGetLastError() != cudaSuccess) {
        lscan_server_destroy(srv);
        return nullptr;
    }
    if (!srv->res_ring || !srv->res_ctl || !srv->res_done) {
        lscan_server_destroy(srv);
        return nullptr;
    }
    srv->n_str = n_str;
    for (int i = 0; i < n_str; ++i) srv->workers.emplace_back(worker_main, srv, i);
    srv->workers.emplace_back(resident_main, srv);
    return srv;
}

void lscan_server_destroy(lscan_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        // requests that were never admitted cannot run any more
        for (auto &q : srv->waiting) {
            for (Request *r : q) {
                r->st.status = LSCAN_ERR_NOMEM;
                finish_locked(srv, r);
            }
            q.clear();
        }
    }
    kick(srv);
    for (auto &w : srv->workers)
        if (w.joinable()) w.join();
    cudaSetDevice(srv->device);
    for (Slot &sl : srv->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.h_list) cudaFreeHost(sl.h_list);
        if (sl.h_err) cudaFreeHost(sl.h_err);
        if (sl.ev_start) cudaEventDestroy(sl.ev_start);
        if (sl.ev_done) cudaEventDestroy(sl.ev_done);
        delete sl.inflight;
    }
    for (Slot &sl : srv->slots)
        if (sl.owns_stream && sl.stream) cudaStreamDestroy(sl.stream);
    if (srv->ref_ev) cudaEventDestroy(srv->ref_ev);
    if (srv->res_stream) {
        cudaStreamSynchronize(srv->res_stream);
        cudaStreamDestroy(srv->res_stream);
    }
    if (srv->res_end) cudaEventDestroy(srv->res_end);
    if (srv->res_ring) cudaFreeHost(srv->res_ring);
    if (srv->res_ctl) cudaFreeHost(srv->res_ctl);
    if (srv->res_done) cudaFreeHost(srv->res_done);
    for (auto &kv : srv->reqs) delete kv.second;
    if (srv->mem) cudaFree(srv->mem);
    delete srv;
}

lscan_status lscan_server_hold(lscan_server *srv, int hold) {
    if (!srv) return LSCAN_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->hold = hold != 0;
    }
    kick(srv);
    return LSCAN_OK;
}

lscan_status lscan_server_set_lanes(lscan_server *srv, int64_t small_max_elems,
                                   int64_t bulk_batch_tiles, int32_t reserve_sms) {
    if (!srv || small_max_elems < 0 || bulk_batch_tiles < 1 ||
        bulk_batch_tiles > kMaxBatchTiles || reserve_sms < 0 || reserve_sms > 64)
        return LSCAN_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->small_max = small_max_elems;
        srv->bulk_cap = bulk_batch_tiles;
        srv->reserve_sms = reserve_sms;
    }
    kick(srv);
    return LSCAN_OK;
}

lscan_status lscan_server_alloc(lscan_server *srv, size_t bytes, void **dptr) {
    if (!srv || !dptr) return LSCAN_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    size_t off = 0;
    if (!srv->alloc.alloc(bytes, &off)) return LSCAN_ERR_NOMEM;
    *dptr = srv->pool + off;
    return LSCAN_OK;
}

lscan_status lscan_server_free(lscan_server *srv, void *dptr) {
    if (!srv || !dptr) return LSCAN_ERR_INVALID;
    lscan_status st;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        const uint8_t *p = static_cast<uint8_t *>(dptr);
        if (p < srv->pool || p >= srv->pool + srv->pool_size) return LSCAN_ERR_INVALID;
        st = srv->alloc.release(p - srv->pool) ? LSCAN_OK : LSCAN_ERR_INVALID;
    }
    kick(srv);  // waiting requests may now fit
    return st;
}

}  // extern "C"

// Submission.  A replayed request carries its trace index (tag >= 0) and its
// scheduled arrival time, both set under the same lock that makes it visible
// to the scheduler.
// A checked request (not yet visible to the schedulers), or an error.
static lscan_status make_request(lscan_op op, lscan_dtype dtype, int inclusive,
                                 const void *x, void *y, int64_t n, Request **out) {
    if (n < 0) return LSCAN_ERR_INVALID;
    if (op != LSCAN_ADD && op != LSCAN_MAX) return LSCAN_ERR_INVALID;
    const int isz = dtype_size(dtype);
    if (isz == 0) return LSCAN_ERR_INVALID;
    const int osz = dtype_size(out_dtype_of(op, dtype));
    if (n > 0 && (x == nullptr || reinterpret_cast<uintptr_t>(x) % isz != 0))
        return LSCAN_ERR_INVALID;
    if (y && reinterpret_cast<uintptr_t>(y) % osz != 0) return LSCAN_ERR_INVALID;
    if (y && n > 0) {
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(x), a1 = a0 + n * isz;
        const uintptr_t b0 = reinterpret_cast<uintptr_t>(y), b1 = b0 + n * osz;
        const bool disjoint = a1 <= b0 || b1 <= a0;
        if (!disjoint && !(a0 == b0 && isz == osz)) return LSCAN_ERR_INVALID;
    }
    // one request must fit one launch's status words
    const int64_t min_tile = kMinTileBytes / isz;  // elements
    if ((n + min_tile - 1) / min_tile > kMaxBatchTiles) return LSCAN_ERR_INVALID;
    Request *r = new Request();
    r->op = op;
    r->dtype = dtype;
    r->inclusive = inclusive ? 1 : 0;
    r->x = x;
    r->y = y;
    r->n = n;
    r->st.n = n;
    r->st.y = y;
    *out = r;
    return LSCAN_OK;
}

// Makes a checked request visible: ticket, lane, admission (at once when the
// pool has room and nothing of its lane waits before it).  Caller holds mu;
// the caller kicks the schedulers afterwards.  On error r is deleted.
static lscan_status enqueue_locked(lscan_server *srv, Request *r, int64_t tag,
                                   double arrival_us, uint64_t *ticket) {
    if (srv->stop) {
        delete r;
        return LSCAN_ERR_INVALID;
    }
    const size_t need =
        r->y ? 0 : static_cast<size_t>(r->n) * dtype_size(out_dtype_of(r->op, r->dtype));
    if (need > srv->pool_size) {
        delete r;
        return LSCAN_ERR_NOMEM;  // can never be admitted
    }
    r->id = srv->next_id++;
    r->tag = tag;
    // the resident lane takes small requests of the kinds it scans
    int kind = -1;
    if (r->n > 0 && r->n <= srv->small_max &&
        resolve_kind(r->op, r->dtype, nullptr, &kind, nullptr) == LSCAN_OK &&
        resident_kind_supported(kind)) {
        r->lane = 1;
        r->kind = kind;
    }
    r->st.submit_us = tag >= 0 ? arrival_us : now_us(srv->t0);
    srv->reqs[r->id] = r;
    if (r->y) {
        r->st.admit_us = r->st.submit_us;
        srv->admitted[r->lane].push_back(r);
    } else {
        srv->waiting[r->lane].push_back(r);
        admit_locked(srv);
    }
    // a small request goes to the device from here (the resident worker
    // only relaunches the kernel when it has ended, and retires requests)
    if (r->lane == 1) publish_resident_locked(srv, now_us(srv->t0));
    *ticket = r->id;
    return LSCAN_OK;
}

static lscan_status submit_impl(lscan_server *srv, lscan_op op, lscan_dtype dtype,
                                int inclusive, const void *x, void *y, int64_t n,
                                uint64_t *ticket) {
    if (!srv || !ticket) return LSCAN_ERR_INVALID;
    Request *r = nullptr;
    lscan_status st = make_request(op, dtype, inclusive, x, y, n, &r);
    if (st != LSCAN_OK) return st;
    {
        auto lk = spin_lock(srv->mu);
        st = enqueue_locked(srv, r, -1, 0.0, ticket);
    }
    if (st == LSCAN_OK) kick(srv);
    return st;
}

extern "C" {

lscan_status lscan_server_submit(lscan_server *srv, lscan_op op, lscan_dtype dtype,
                                 int inclusive, const void *x, void *y, int64_t n,
                                 uint64_t *ticket) {
    return submit_impl(srv, op, dtype, inclusive, x, y, n, ticket);
}

static lscan_status server_get(lscan_server *srv, uint64_t ticket, lscan_req_stats *out,
                               bool block) {
    if (!srv) return LSCAN_ERR_INVALID;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return LSCAN_ERR_INVALID;
    Request *r = it->second;
    if (!r->done) {
        if (!block) return LSCAN_ERR_BUSY;
        srv->cv_done.wait(lk, [&] { return r->done; });
    }
    if (out) *out = r->st;
    return static_cast<lscan_status>(r->st.status);
}

lscan_status lscan_server_wait(lscan_server *srv, uint64_t ticket, lscan_req_stats *out) {
    return server_get(srv, ticket, out, true);
}

lscan_status lscan_server_poll(lscan_server *srv, uint64_t ticket, lscan_req_stats *out) {
    return server_get(srv, ticket, out, false);
}

lscan_status lscan_server_release(lscan_server *srv, uint64_t ticket) {
    if (!srv) return LSCAN_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->reqs.find(ticket);
        if (it == srv->reqs.end()) return LSCAN_ERR_INVALID;
        if (!it->second->done) return LSCAN_ERR_BUSY;
        release_request_locked(srv, it->second);
    }
    kick(srv);
    return LSCAN_OK;
}

lscan_status lscan_server_replay(lscan_server *srv, const lscan_trace_req *trace,
                                 int64_t n_req, lscan_req_stats *out, double *wall_us) {
    if (!srv || (n_req > 0 && (!trace || !out))) return LSCAN_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->collecting || srv->stop) return LSCAN_ERR_BUSY;  // one replay at a time
        srv->collecting = true;
        srv->finished.clear();
    }
    std::atomic<int64_t> n_sub{0};
    const double base = now_us(srv->t0);
    std::atomic<int> sub_err{LSCAN_OK};
    // open-loop submitter: each request enters at its arrival time; the
    // requests already due enter together, under one lock
    std::thread submitter([&] {
        std::vector<Request *> group;
        int64_t i = 0;
        while (i < n_req && sub_err.load() == LSCAN_OK) {
            const double due = base + trace[i].arrival_us;
            while (now_us(srv->t0) < due) {
                const double left = due - now_us(srv->t0);
                if (left > 200) std::this_thread::sleep_for(std::chrono::microseconds(100));
            }
            const double now = now_us(srv->t0);
            const int64_t i0 = i;
            group.clear();
            for (; i < n_req && base + trace[i].arrival_us <= now; ++i) {
                Request *r = nullptr;
                const lscan_status st = make_request(
                    static_cast<lscan_op>(trace[i].op), static_cast<lscan_dtype>(trace[i].dtype),
                    trace[i].inclusive, trace[i].x, nullptr, trace[i].n, &r);
                if (st != LSCAN_OK) {
                    sub_err.store(st);
                    break;
                }
                group.push_back(r);
            }
            {
                auto lk = spin_lock(srv->mu);
                for (size_t g = 0; g < group.size(); ++g) {
                    uint64_t tk = 0;
                    const int64_t idx = i0 + static_cast<int64_t>(g);
                    const lscan_status st =
                        enqueue_locked(srv, group[g], idx, base + trace[idx].arrival_us, &tk);
                    if (st != LSCAN_OK) {
                        sub_err.store(st);
                        for (size_t h = g + 1; h < group.size(); ++h) delete group[h];
                        break;
                    }
                    n_sub.fetch_add(1);
                }
            }
            kick(srv);
        }
        kick(srv);  // lets the collector see the end of submission
        srv->cv_done.notify_all();
    });
    // collector: release outputs in completion order so admission never stalls
    int64_t collected = 0;
    double last_done = base;
    std::vector<Request *> fin;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        while (collected < n_req) {
            if (srv->finished.empty()) {
                if (sub_err.load() != LSCAN_OK && collected == n_sub.load()) break;
                srv->cv_done.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            fin.swap(srv->finished);
            for (Request *r : fin) {
                const int64_t i = r->tag;
                out[i] = r->st;
                out[i].y = nullptr;  // released below
                last_done = std::max(last_done, out[i].done_us);
                release_request_locked(srv, r);
                ++collected;
            }
            fin.clear();
            kick(srv);  // freed outputs may admit waiting requests
        }
        srv->collecting = false;
    }
    submitter.join();
    if (wall_us) *wall_us = last_done - base;
    return static_cast<lscan_status>(sub_err.load());
}

}  // extern "C"
