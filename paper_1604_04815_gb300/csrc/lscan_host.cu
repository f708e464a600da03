// lscan_host.cu -- single-array scans of arrays that live in host memory.
//
// Not in the paper, whose arrays are already on the device.  The array is
// cut into chunks that pass through a ring of device slots: chunk k is copied
// in on one stream while chunk k-1 is scanned on the caller's stream and
// chunk k-2 is copied out on a third, so both copy directions and the scans
// overlap.  Each chunk's scan writes its inclusive total in the kind's carry
// type (FP64 for the float adds with an FP64 carry), and the next chunk takes
// that as its carry-in: the carry chain of Section 4.3 continued from one
// launch to the next with no rounding to the output type in between, so a
// chunked scan meets the same error bound as one launch over the whole array.
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "../../include/lscan.h"
#include "lscan_internal.h"
#include "scan_common.h"

namespace lscan {
namespace {

constexpr int kSlots = 3;  // in flight: copy-in, scan, copy-out
constexpr int64_t kDefaultChunk = int64_t{1} << 23;
constexpr int64_t kRampChunk = int64_t{1} << 20;  // first and last chunks

// Length of chunk k when `remaining` elements are left.  Fixed chunks of C,
// or (ramp) chunks that double from kRampChunk up to C and halve again over
// the last 2 C elements: the first copy-in and the last copy-out overlap
// nothing, so they are kept short.
int64_t chunk_len(int64_t k, int64_t remaining, int64_t C, bool ramp) {
    if (!ramp || C <= kRampChunk) return remaining < C ? remaining : C;
    int64_t up = kRampChunk << (k < 16 ? k : 16);
    if (up > C) up = C;
    const int64_t half = (remaining + 1) / 2;
    const int64_t down = remaining <= kRampChunk ? remaining
                                                 : (half > kRampChunk ? half : kRampChunk);
    const int64_t m = up < down ? up : down;
    return m < remaining ? m : remaining;
}

struct HostPipe {
    int device = -1;
    std::mutex mu;  // one call at a time per (device, stream)
    cudaStream_t h2d = nullptr;
    cudaStream_t d2h = nullptr;
    cudaEvent_t fork = nullptr;
    cudaEvent_t in_done[kSlots] = {};
    cudaEvent_t scanned[kSlots] = {};
    cudaEvent_t out_done[kSlots] = {};
    void *din[kSlots] = {};
    void *dout[kSlots] = {};
    size_t in_cap = 0, out_cap = 0;  // bytes per slot
    void *car = nullptr;             // two 16-byte chunk totals
};

std::mutex g_host_mu;
std::map<std::pair<int, void *>, HostPipe *> g_pipes;

lscan_status create_pipe(int dev, HostPipe *p) {
    p->device = dev;
    const unsigned fl = cudaStreamNonBlocking;
    if (cudaStreamCreateWithFlags(&p->h2d, fl) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->d2h, fl) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) != cudaSuccess)
        return LSCAN_ERR_CUDA;
    for (int s = 0; s < kSlots; ++s)
        if (cudaEventCreateWithFlags(&p->in_done[s], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->scanned[s], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->out_done[s], cudaEventDisableTiming) != cudaSuccess)
            return LSCAN_ERR_CUDA;
    if (cudaMalloc(&p->car, 32) != cudaSuccess) return LSCAN_ERR_NOMEM;
    return LSCAN_OK;
}

void free_slots(HostPipe *p) {
    for (int s = 0; s < kSlots; ++s) {
        if (p->din[s]) cudaFree(p->din[s]);
        if (p->dout[s]) cudaFree(p->dout[s]);
        p->din[s] = p->dout[s] = nullptr;
    }
    p->in_cap = p->out_cap = 0;
}

// Slots of at least in_b / out_b bytes.  Earlier calls may still copy from
// or scan into the old slots: their last copy-outs are waited for first.
lscan_status ensure_slots(HostPipe *p, size_t in_b, size_t out_b) {
    if (p->in_cap >= in_b && p->out_cap >= out_b) return LSCAN_OK;
    for (int s = 0; s < kSlots; ++s)
        if (cudaEventSynchronize(p->out_done[s]) != cudaSuccess) return LSCAN_ERR_CUDA;
    free_slots(p);
    for (int s = 0; s < kSlots; ++s) {
        // 16-byte aligned slot bases keep every chunk on the bulk-copy kernels
        if (cudaMalloc(&p->din[s], in_b) != cudaSuccess ||
            cudaMalloc(&p->dout[s], out_b) != cudaSuccess) {
            free_slots(p);
            return LSCAN_ERR_NOMEM;
        }
    }
    p->in_cap = in_b;
    p->out_cap = out_b;
    return LSCAN_OK;
}

void destroy_pipe(HostPipe *p) {
    if (p->device >= 0) cudaSetDevice(p->device);
    if (p->h2d) cudaStreamSynchronize(p->h2d);
    if (p->d2h) cudaStreamSynchronize(p->d2h);
    free_slots(p);
    if (p->car) cudaFree(p->car);
    for (int s = 0; s < kSlots; ++s) {
        if (p->in_done[s]) cudaEventDestroy(p->in_done[s]);
        if (p->scanned[s]) cudaEventDestroy(p->scanned[s]);
        if (p->out_done[s]) cudaEventDestroy(p->out_done[s]);
    }
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->h2d) cudaStreamDestroy(p->h2d);
    if (p->d2h) cudaStreamDestroy(p->d2h);
    delete p;
}

bool host_ranges_partially_overlap(const void *x, size_t xb, const void *y, size_t yb) {
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(x), a1 = a0 + xb;
    const uintptr_t b0 = reinterpret_cast<uintptr_t>(y), b1 = b0 + yb;
    if (a1 <= b0 || b1 <= a0) return false;
    return !(a0 == b0 && xb == yb);
}

}  // namespace

void shutdown_host_pipes() {
    std::lock_guard<std::mutex> lk(g_host_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_pipes) destroy_pipe(kv.second);
    g_pipes.clear();
    cudaSetDevice(cur);
}

}  // namespace lscan

using namespace lscan;

extern "C" lscan_status lscan_scan_host(lscan_op op, lscan_dtype dtype, int inclusive,
                                        const void *hx, void *hy, int64_t n,
                                        const lscan_options *opts, int64_t chunk,
                                        void *stream) {
    if (n < 0 || chunk < 0) return LSCAN_ERR_INVALID;
    // the kind, output type and every option are checked by planning one
    // chunk; the host-side rules are checked here
    LaunchSpec probe;
    const lscan_options *popts = opts;
    lscan_options no_carry{};
    if (opts) {
        no_carry = *opts;
        no_carry.carry_in = nullptr;
        popts = &no_carry;
    }
    lscan_status st =
        plan_scan(op, dtype, inclusive, nullptr, nullptr, 0, popts, MODE_SINGLE, nullptr, 0,
                  &probe);
    if (st != LSCAN_OK) return st;
    if (n == 0) return LSCAN_OK;
    const int isz = dtype_size(dtype);
    int out_dt = dtype;
    if (op == LSCAN_ADD && dtype == LSCAN_BF16) out_dt = LSCAN_F32;
    if (opts && opts->out_dtype > 0 && opts->out_dtype <= LSCAN_F64) out_dt = opts->out_dtype;
    const int osz = dtype_size(out_dt);
    if (hx == nullptr || hy == nullptr) return LSCAN_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(hx) % isz != 0 ||
        reinterpret_cast<uintptr_t>(hy) % osz != 0)
        return LSCAN_ERR_INVALID;
    if (host_ranges_partially_overlap(hx, static_cast<size_t>(n) * isz, hy,
                                      static_cast<size_t>(n) * osz))
        return LSCAN_ERR_INVALID;
    if (opts && opts->carry_in && reinterpret_cast<uintptr_t>(opts->carry_in) % osz != 0)
        return LSCAN_ERR_INVALID;

    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(cs, &cap) != cudaSuccess) return LSCAN_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return LSCAN_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LSCAN_ERR_CUDA;

    HostPipe *p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        HostPipe *&slot = g_pipes[{dev, stream}];
        if (slot == nullptr) {
            slot = new HostPipe();
            st = create_pipe(dev, slot);
            if (st != LSCAN_OK) {
                destroy_pipe(slot);
                slot = nullptr;
                return st;
            }
        }
        p = slot;
    }
    std::lock_guard<std::mutex> plk(p->mu);

    const int64_t C = chunk > 0 ? (chunk < n ? chunk : n) : (kDefaultChunk < n ? kDefaultChunk : n);
    st = ensure_slots(p, static_cast<size_t>(C) * isz, static_cast<size_t>(C) * osz);
    if (st != LSCAN_OK) return st;

    // fork: the copies start after the work already queued on the stream
    if (cudaEventRecord(p->fork, cs) != cudaSuccess ||
        cudaStreamWaitEvent(p->h2d, p->fork, 0) != cudaSuccess ||
        cudaStreamWaitEvent(p->d2h, p->fork, 0) != cudaSuccess)
        return LSCAN_ERR_CUDA;

    const char *bx = static_cast<const char *>(hx);
    char *by = static_cast<char *>(hy);
    char *car = static_cast<char *>(p->car);
    int last = 0;
    int64_t off = 0;
    for (int64_t k = 0; off < n; ++k) {
        const int s = static_cast<int>(k % kSlots);
        const int64_t m = chunk_len(k, n - off, C, chunk == 0);
        // copy in once the slot's previous chunk has been copied out (which
        // also orders it after that chunk's scan)
        if (cudaStreamWaitEvent(p->h2d, p->out_done[s], 0) != cudaSuccess ||
            cudaMemcpyAsync(p->din[s], bx + off * isz, static_cast<size_t>(m) * isz,
                            cudaMemcpyHostToDevice, p->h2d) != cudaSuccess ||
            cudaEventRecord(p->in_done[s], p->h2d) != cudaSuccess)
            return LSCAN_ERR_CUDA;
        // scan on the caller's stream: chunk 0 takes the caller's carry-in,
        // chunk k > 0 the total chunk k-1 wrote (the two totals alternate)
        if (cudaStreamWaitEvent(cs, p->in_done[s], 0) != cudaSuccess) return LSCAN_ERR_CUDA;
        LaunchSpec ls;
        lscan_options o = opts ? *opts : lscan_options{};
        if (k > 0) o.carry_in = nullptr;
        st = plan_scan(op, dtype, inclusive, p->din[s], p->dout[s], m, &o, MODE_SINGLE,
                       nullptr, 0, &ls);
        if (st != LSCAN_OK) return st;
        if (k > 0) {
            ls.carry_in = car + 16 * ((k - 1) & 1);
            ls.carry_in_car = true;
        }
        ls.total_out = off + m < n ? car + 16 * (k & 1) : nullptr;
        st = run_planned(ls, stream);
        if (st != LSCAN_OK) return st;
        // copy out after the scan
        if (cudaEventRecord(p->scanned[s], cs) != cudaSuccess ||
            cudaStreamWaitEvent(p->d2h, p->scanned[s], 0) != cudaSuccess ||
            cudaMemcpyAsync(by + off * osz, p->dout[s], static_cast<size_t>(m) * osz,
                            cudaMemcpyDeviceToHost, p->d2h) != cudaSuccess ||
            cudaEventRecord(p->out_done[s], p->d2h) != cudaSuccess)
            return LSCAN_ERR_CUDA;
        last = s;
        off += m;
    }
    // join: work queued on the stream later runs after the last copy-out
    // (the copy-outs run in order on one stream)
    if (cudaStreamWaitEvent(cs, p->out_done[last], 0) != cudaSuccess) return LSCAN_ERR_CUDA;
    return LSCAN_OK;
}
