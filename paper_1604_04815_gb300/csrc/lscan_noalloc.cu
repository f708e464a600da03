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
//  - The first call on each device looks up the array's device address and
//    clears it with cudaMemsetAsync on the caller's stream; make that first
//    call before any stream capture.
//  - All calls share the one array.  Each launch re-arms the ticket and
//    advances the epoch itself at its end, so consecutive calls need no
//    clearing, but calls that overlap on the GPU (different streams without
//    synchronisation between them) race on the array and give wrong results.
//  - Sizes whose status words do not fit return LSCAN_ERR_INVALID without
//    launching anything.
//  - Device-side wait timeouts of these launches are not reported (no status
//    entry point reads this array); every wait is still bounded, so a call
//    can never hang the GPU.
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
    if (ls.status_words > kNoAllocStatusWords) return LSCAN_ERR_INVALID;
    if (n == 0) return LSCAN_OK;
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
