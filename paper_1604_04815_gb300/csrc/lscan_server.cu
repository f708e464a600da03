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
//  * Admission.  A request whose output the server must allocate waits in a
//    FIFO queue until the pool can hold it; requests are admitted in arrival
//    order as earlier ones release their outputs.
//  * Continuous batching.  A scheduler thread keeps two launch slots per
//    stream (the second batch of a stream is queued behind the first, so the
//    GPU never waits for the host between batches).  Whenever a slot is idle
//    it takes the oldest admitted request, gathers
//    every admitted request of the same (op, dtype, inclusive) up to a tile
//    budget, and issues ONE persistent MODE_LIST launch over them (each array
//    keeps its own carry chain).  Different kinds run on different streams
//    and overlap on the device; requests arriving while batches run are
//    admitted and launched as slots free up.
//  * Size-class lanes.  Requests of at most small_max elements (2^16 by
//    default) form their own lane: their own admission queue and two launch
//    slots on a stream created at the device's greatest priority, batched
//    only with each other.  Bulk batches are capped at bulk_cap tiles (8192
//    by default, ~128 MiB of 16 KiB tiles), so a small batch waits at most
//    about one capped bulk launch for SM slots: when a bulk kernel's
//    persistent CTAs retire, the block scheduler dispatches the
//    higher-priority small batch before the bulk batch queued behind it.
//    FIFO order holds within each lane.
//  * Completion.  The scheduler polls each in-flight slot's last event
//    (cudaEventQuery); nothing host-side sits in the stream, so the batch
//    queued behind it starts the moment the kernel before it ends.  Launch
//    and completion times are read from CUDA events and mapped onto the host
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
#include "scan_common.h"

namespace lscan {
namespace {

constexpr size_t kPoolAlign = 256;
constexpr int64_t kMaxBatchTiles = 65536;   // ~1 GiB of 16 KiB tiles per launch
constexpr int kSlotsPerStream = 2;          // a second batch queues behind the first
constexpr int64_t kMinTileBytes = 8192;     // smallest input tile of any config
constexpr int64_t kMaxBatchRequests = 4096;
constexpr int64_t kDefaultSmallMax = int64_t{1} << 16;  // elements
constexpr int64_t kDefaultBulkCap = 8192;               // tiles per bulk batch
constexpr int kLanes = 2;                               // 0 bulk, 1 small

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
    int lane = 0;      // 0 bulk, 1 small
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
    std::unordered_map<uint64_t, Request *> reqs;
    std::mutex mu;     // requests, pool, slots
    std::mutex cb_mu;  // wake-up flag only
    std::condition_variable cv_sched, cv_done;
    bool kick = false;
    std::thread sched;
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
bool prepare_batch_locked(lscan_server *srv, int si, Pending *pd) {
    Slot &sl = srv->slots[si];
    auto &admitted = srv->admitted[sl.lane];
    const int64_t cap = sl.lane == 0 ? srv->bulk_cap : kMaxBatchTiles;
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
// two events (the second is the one the scheduler polls).  Only the
// scheduler thread touches a slot, so no lock is held.
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

// The scheduler sleeps while no batch is in flight; otherwise it polls the
// in-flight slots' last events (only this thread launches or retires
// batches, so it reads the slots without the lock) and takes the lock only
// when a batch has finished or a client has kicked it.
void scheduler_main(lscan_server *srv) {
    cudaSetDevice(srv->device);
    std::vector<std::pair<int, bool>> done;  // (slot, CUDA ok)
    std::vector<Pending> todo;               // batches to launch
    bool busy = false;
    while (true) {
        bool kicked;
        {
            std::unique_lock<std::mutex> lk(srv->cb_mu);
            if (!busy) srv->cv_sched.wait(lk, [&] { return srv->kick; });
            kicked = srv->kick;
            srv->kick = false;
        }
        done.clear();
        for (size_t si = 0; si < srv->slots.size(); ++si) {
            const Slot &sl = srv->slots[si];
            if (!sl.inflight) continue;
            const cudaError_t q = cudaEventQuery(sl.ev_done);
            if (q != cudaErrorNotReady) done.emplace_back(static_cast<int>(si), q == cudaSuccess);
        }
        if (!kicked && done.empty()) {
            std::this_thread::yield();
            continue;
        }
        todo.clear();
        bool leave = false;
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            for (auto &d : done) retire_locked(srv, d.first, d.second);
            admit_locked(srv);
            if (!srv->hold || srv->stop)
                for (size_t si = 0; si < srv->slots.size(); ++si) {
                    if (srv->slots[si].inflight) continue;
                    Pending pd;
                    if (prepare_batch_locked(srv, static_cast<int>(si), &pd)) todo.push_back(pd);
                }
            busy = false;
            for (auto &sl : srv->slots) busy = busy || sl.inflight;
            leave = srv->stop && !busy && srv->admitted[0].empty() && srv->admitted[1].empty();
        }
        for (const Pending &pd : todo) issue_batch(srv, pd);
        if (leave) break;
    }
}

// Wake the scheduler (never blocks on srv->mu).
void kick(lscan_server *srv) {
    {
        std::lock_guard<std::mutex> lk(srv->cb_mu);
        srv->kick = true;
    }
    srv->cv_sched.notify_one();
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
    // n_streams bulk streams and one small-lane stream, two slots each
    const size_t reserve = slot_b * (n_streams + 1) * kSlotsPerStream;
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
    // slots: [0, n) bulk streams, n the small-lane stream; then a second
    // slot for each of them on the same stream
    const int n_str = n_streams + 1;
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
        sl.lane = (i % n_str) == n_streams ? 1 : 0;
        if (i < n_str)
            cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking,
                                         sl.lane == 1 ? prio_greatest : prio_least);
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
    cudaEventCreate(&srv->ref_ev);
    cudaEventRecord(srv->ref_ev, srv->slots[0].stream);
    cudaEventSynchronize(srv->ref_ev);
    srv->ref_us = now_us(srv->t0);
    if (cudaGetLastError() != cudaSuccess) {
        lscan_server_destroy(srv);
        return nullptr;
    }
    srv->sched = std::thread(scheduler_main, srv);
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
    if (srv->sched.joinable()) srv->sched.join();
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
                                   int64_t bulk_batch_tiles) {
    if (!srv || small_max_elems < 0 || bulk_batch_tiles < 1 ||
        bulk_batch_tiles > kMaxBatchTiles)
        return LSCAN_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->small_max = small_max_elems;
        srv->bulk_cap = bulk_batch_tiles;
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
static lscan_status submit_impl(lscan_server *srv, lscan_op op, lscan_dtype dtype,
                                int inclusive, const void *x, void *y, int64_t n,
                                uint64_t *ticket, int64_t tag, double arrival_us) {
    if (!srv || !ticket || n < 0) return LSCAN_ERR_INVALID;
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
    Request *r = new Request();
    r->op = op;
    r->dtype = dtype;
    r->inclusive = inclusive ? 1 : 0;
    r->x = x;
    r->y = y;
    r->n = n;
    r->st.n = n;
    r->st.y = y;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) {
            delete r;
            return LSCAN_ERR_INVALID;
        }
        const size_t need = y ? 0 : static_cast<size_t>(n) * osz;
        // one request must fit one launch's status words
        const int64_t min_tile = kMinTileBytes / isz;  // elements
        if ((n + min_tile - 1) / min_tile > kMaxBatchTiles) {
            delete r;
            return LSCAN_ERR_INVALID;
        }
        if (need > srv->pool_size) {
            delete r;
            return LSCAN_ERR_NOMEM;  // can never be admitted
        }
        r->id = srv->next_id++;
        r->tag = tag;
        r->lane = n <= srv->small_max ? 1 : 0;
        r->st.submit_us = tag >= 0 ? arrival_us : now_us(srv->t0);
        srv->reqs[r->id] = r;
        if (y) {
            r->st.admit_us = r->st.submit_us;
            srv->admitted[r->lane].push_back(r);
        } else {
            srv->waiting[r->lane].push_back(r);
        }
        *ticket = r->id;
    }
    kick(srv);
    return LSCAN_OK;
}

extern "C" {

lscan_status lscan_server_submit(lscan_server *srv, lscan_op op, lscan_dtype dtype,
                                 int inclusive, const void *x, void *y, int64_t n,
                                 uint64_t *ticket) {
    return submit_impl(srv, op, dtype, inclusive, x, y, n, ticket, -1, 0.0);
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
    // open-loop submitter: each request enters at its arrival time
    std::thread submitter([&] {
        for (int64_t i = 0; i < n_req; ++i) {
            const double due = base + trace[i].arrival_us;
            while (now_us(srv->t0) < due) {
                const double left = due - now_us(srv->t0);
                if (left > 200) std::this_thread::sleep_for(std::chrono::microseconds(100));
            }
            uint64_t tk = 0;
            const lscan_status st = submit_impl(
                srv, static_cast<lscan_op>(trace[i].op), static_cast<lscan_dtype>(trace[i].dtype),
                trace[i].inclusive, trace[i].x, nullptr, trace[i].n, &tk, i, due);
            if (st != LSCAN_OK) {
                sub_err.store(st);
                break;
            }
            n_sub.fetch_add(1);
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
