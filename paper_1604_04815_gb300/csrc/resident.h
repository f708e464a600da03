// resident.h -- ring layout and launch of the server's resident lane
// (resident_kernel.cu); shared by the kernel and lscan_server.cu.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/lscan.h"

namespace lscan {

// One published request (host memory mapped for the device; 32 bytes,
// read by the device as two 16-byte loads).
struct alignas(16) ResReq {
    const void *x;
    void *y;
    int64_t n;
    int32_t kind;
    int32_t inclusive;
};
static_assert(sizeof(ResReq) == 32, "two 16-byte loads");

struct ResParams {
    const ResReq *ring;          // ring_size entries, host-written
    const uint64_t *published;   // host: entries written so far (release)
    const uint32_t *stop;        // host: nonzero = CTAs leave
    unsigned long long *claim;   // device memory: next entry to claim
    uint64_t *done;              // ring_size words: entry i done <=> i + 1
    int64_t ring_size;
    uint64_t idle_ns;            // a CTA with nothing to claim this long leaves
};

// kinds the resident kernel scans (the server's default precision)
bool resident_kind_supported(int kind);
// ctas CTAs of 256 threads on stream s
lscan_status launch_resident(const ResParams &p, int ctas, cudaStream_t s);

}  // namespace lscan
