// lscan_noalloc.cu -- a single-array scan entry point that never allocates.
//
// Who needs it: code that may not call cudaMalloc at the point where it wants
// to scan -- for example a custom allocator or memory-pool implementation
// that is itself in the middle of servicing an allocation, code running under
// a framework that forbids device allocations outside its own pool, or a
// real-time path where an allocation (which can synchronise the device or
// fail when memory is tight) is not acceptable.  The regular entry points
// allocate their per-stream scratch lazily with cudaMalloc; this one uses a
// fixed scratch area compiled into the library instead.
//
// The scratch is the same thing the regular path allocates: a control block
// (tile ticket, finished-CTA count, epoch, error word) and a status slot of 2
// or 4 words per tile.  It lives in a file-scope __device__ array, so every
// GPU that loads the library holds its 2 MiB + 512 B until the process
// exits.
//
// Rules for callers (also stated in include/lscan.h):
//  - The first call on each device is a set-up call: it looks up the array's
//    device address (under lazy module loading this loads the library's
//    module, which is when the driver places the array) and clears it with
//    cudaMemsetAsync on the caller's stream.  Make it at initialisation,
//    outside any context that must not allocate.
//  - All calls share the one array.  Each launch re-arms the ticket and
//    advances the epoch itself at its end, so consecutive calls need no
//    clearing, but calls that overlap on the GPU (different streams without
//    synchronisation between them) race on the array and give wrong results.
//  - The tile configuration is fixed (configuration 2: 16 KiB input tiles,
//    status slots of 2 words for 32-bit carries), so the size limit does not
//    move with the autotuner's table.  Sizes whose status words do not fit
//    return LSCAN_ERR_INVALID without launching anything.  Arrays of at most
//    4096 elements take the single-CTA kernel, which uses no scratch.
//  - A device-side wait that ran out of time (every wait is bounded, so a
//    call cannot hang) latches the array's error word; lscan_noalloc_status
//    reads and clears it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lscan.h"
#include "lscan_internal.h"
#include "scan_common.h"

namespace lscan {
namespace {

// 512 B control block + 262144 status words: 2 MiB + 512 B per device.
constexpr size_t kNoAllocStatusWords = size_t{1} << 18;
constexpr size_t kNoAllocScratchWords = CTL_WORDS / 2 + kNoAllocStatusWords;

static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocScratchWords];

// tile configuration of every launch that needs scratch
constexpr int kNoAllocConfig = 2;

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
uint64_t *g_na_ptr[kMaxDevices] = {};
uint64_t g_na_launches[kMaxDevices] = {};

// Device address of this device's copy of the array; first use clears it.
lscan_status noalloc_scratch(int dev, cudaStream_t cs, uint64_t **out) {
    if (dev < 0 || dev >= kMaxDevices) return LSCAN_ERR_UNSUPPORTED;
    if (g_na_ptr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
            return LSCAN_ERR_CUDA;
        if (cudaMemsetAsync(p, 0, sizeof(g_noalloc_scratch), cs) != cudaSuccess)
            return LSCAN_ERR_CUDA;
        g_na_ptr[dev] = static_cast<uint64_t *>(p);
    }
    *out = g_na_ptr[dev];
    return LSCAN_OK;
}

}  // namespace
}  // namespace lscan

using namespace lscan;

extern "C" lscan_status lscan_scan_noalloc(lscan_op op, lscan_dtype dtype,
                                          int inclusive, const void *x, void *y,
                                          int64_t n, void *stream) {
    LaunchSpec ls;
    lscan_status st = plan_scan(op, dtype, inclusive, x, y, n, nullptr, MODE_SINGLE,
                                nullptr, 0, &ls);
    if (st != LSCAN_OK) return st;
    if (n == 0) return LSCAN_OK;
    if (!ls.tiny) {
        // a fixed configuration, so that the limit does not depend on tuning
        lscan_options o{};
        o.config = kNoAllocConfig;
        o.carry = LSCAN_CARRY_LOOKBACK;
        st = plan_scan(op, dtype, inclusive, x, y, n, &o, MODE_SINGLE, nullptr, 0, &ls);
        if (st != LSCAN_OK) return st;
    }
    if (ls.status_words > kNoAllocStatusWords) return LSCAN_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LSCAN_ERR_CUDA;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(g_na_mu);
    uint64_t *base = nullptr;
    st = noalloc_scratch(dev, cs, &base);
    if (st != LSCAN_OK) return st;
    uint32_t *ctl = reinterpret_cast<uint32_t *>(base);
    uint64_t *status = base + CTL_WORDS / 2;
    // keep the 30-bit epoch tag from wrapping (same rule as the regular path)
    if (++g_na_launches[dev] >= (uint64_t{1} << 30) - 1) {
        if (cudaMemsetAsync(base, 0, sizeof(g_noalloc_scratch), cs) != cudaSuccess)
            return LSCAN_ERR_CUDA;
        g_na_launches[dev] = 0;
    }
    DevBuffers b{ctl, status};
    return launch_scan(ls, b, cs);
}

extern "C" lscan_status lscan_noalloc_status(void *stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LSCAN_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LSCAN_ERR_UNSUPPORTED;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return LSCAN_ERR_CUDA;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (g_na_ptr[dev] == nullptr) return LSCAN_OK;  // no launch on this device yet
    }
    // the error word of this device's control block, read and cleared by
    // symbol (plain copies through host memory; nothing is allocated)
    const size_t off = CTL_ERROR * sizeof(uint32_t);
    uint32_t err = 0;
    if (cudaMemcpyFromSymbol(&err, g_noalloc_scratch, sizeof(err), off) != cudaSuccess)
        return LSCAN_ERR_CUDA;
    if (err == 0) return LSCAN_OK;
    const uint32_t zero = 0;
    if (cudaMemcpyToSymbol(g_noalloc_scratch, &zero, sizeof(zero), off) != cudaSuccess)
        return LSCAN_ERR_CUDA;
    if (err & (DEV_ERR_CARRY_WAIT | DEV_ERR_BARRIER_WAIT)) return LSCAN_ERR_TIMEOUT;
    return LSCAN_ERR_DEVICE;
}
