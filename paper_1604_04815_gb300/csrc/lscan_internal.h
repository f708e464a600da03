// lscan_internal.h -- declarations shared by the host-side translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "../../include/lscan.h"

namespace lscan {

// A fully checked launch request.
struct LaunchSpec {
    int kind = -1;
    int mode = 0;
    int variant = 0;
    const void *x = nullptr;
    void *y = nullptr;
    int64_t n = 0;
    const int64_t *offsets = nullptr;  // SEGMENTED offsets / LIST first tiles
    int64_t n_seg = 0;
    const void *segs = nullptr;        // LIST: device SegDesc[n_seg]
    int64_t list_tiles = 0;            // LIST: total tiles over all arrays
    bool inclusive = true;
    int carry_mode = 0;  // CarryMode
    int max_ctas = 0;
    size_t status_words = 0;
    const void *carry_in = nullptr;  // MODE_SINGLE only
    bool carry_in_car = false;       // carry_in holds the kind's carry type
    void *total_out = nullptr;       // MODE_SINGLE: inclusive total, carry type
    bool tiny = false;               // single-CTA kernel, no scratch
    const void *values = nullptr;    // stream compaction: values, count
    unsigned long long *count_out = nullptr;
    uint32_t *err_host = nullptr;    // mapped host word for the error word
    int reserve_sms = 0;             // launch for (SMs - reserve_sms) x CTAs/SM
};

// Device scratch a launch uses (control block + status words).
struct DevBuffers {
    uint32_t *ctl;
    uint64_t *status;
};

// kind id (and output dtype) of (op, dtype, opts: out_dtype, precision)
lscan_status resolve_kind(int op, int dtype, const lscan_options *opts, int *kind,
                          int *out_dtype);
lscan_status plan_scan(int op, int dtype, int inclusive, const void *x, void *y,
                       int64_t n, const lscan_options *opts, int mode,
                       const int64_t *offsets, int64_t n_seg, LaunchSpec *ls);
lscan_status launch_scan(const LaunchSpec &ls, const DevBuffers &buf,
                         cudaStream_t cs);
lscan_status run_planned(const LaunchSpec &ls, void *stream);
// tile length of the kernel a plan selected
int planned_tile(const LaunchSpec &ls);
// number of 64-bit status words per tile of a kind
int carry_words(int kind);

// tile configuration the tuning table picks for (kind, mode, n), and the
// carry protocol recorded with it (an lscan_carry; 0 = auto)
int tuned_variant(int kind, int mode, int64_t n, int *carry);
// tiles of a planned launch
int64_t planned_tiles(const LaunchSpec &ls);
// registers every compiled kernel (once)
void ensure_kernels_registered();

std::mutex &api_mutex();
// the (device, stream) scratch of the scan (grown to `words` status words,
// epoch kept from wrapping), for other chained kernels on the stream
lscan_status acquire_stream_scratch(void *stream, size_t words, DevBuffers *out);
// the device wait limit, and the fault-injection tile of the next launch
uint64_t current_wait_limit_ns();
int64_t take_skip_tile();
void shutdown_graphs_locked();
void shutdown_host_pipes();  // frees the staging of lscan_scan_host
void shutdown_radix();       // frees the counters of lscan_radix_offsets
int dtype_size(int dt);
void note_launch();  // counts one kernel launch of this library

// cudaLaunchKernel with programmatic stream serialization: the kernel's CTAs
// may be scheduled while the previous kernel of the stream finishes.  Only
// for kernels that wait for their predecessor (griddepcontrol.wait) before
// they touch global memory.
cudaError_t launch_serialized(const void *fn, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, void **args);
// entry = configuration | carry << 8
void set_tuned_variant(int kind, int mode, int size_cls, int entry);

}  // namespace lscan
