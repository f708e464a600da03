// scan_common.h -- definitions shared by the kernels and the host library.
#pragma once
#include <cuda.h>  // CUtensorMap

#include <cstdint>

namespace lscan {

// Control block of one scratch set (device memory, 512 bytes).  Each field
// sits on its own 128-byte line.  ticket/done/epoch are reset or advanced by
// the last CTA of every launch, so consecutive launches on a stream (and CUDA
// graph replays) need no host-side memset.
enum CtlWord : int {
    CTL_TICKET = 0,   // next tile to hand out (atomic ticket, Section 4 intro)
    CTL_DONE = 32,    // CTAs finished in the current launch
    CTL_EPOCH = 64,   // launch counter that tags status words
    CTL_ERROR = 96,   // sticky device error bits (read + cleared by the host)
    CTL_ERR_EPOCH = 100,  // epoch + 1 of the launch that last gave up a wait
    CTL_WORDS = 128
};

enum DevError : uint32_t {
    DEV_ERR_CARRY_WAIT = 1u,    // a predecessor's status never arrived in time
    DEV_ERR_BARRIER_WAIT = 2u,  // a tile-ring barrier never completed in time
    DEV_ERR_SMEM_ALIGN = 4u,    // dynamic shared memory not 1024-byte aligned
                                // (swizzled tile copies need it; nothing ran)
};

// Status word: (payload32 << 32) | tag32, tag = (epoch mod 2^30) << 2 | state.
// A payload wider than 32 bits uses several words, each with the full tag.
enum TileState : uint32_t { ST_INVALID = 0, ST_AGGREGATE = 1, ST_INCLUSIVE = 2 };
constexpr uint32_t kEpochMask = 0x3fffffffu;

// MODE_SINGLE: one array.  MODE_SEGMENTED: arrays back to back, delimited by
// offsets; tiles span segment boundaries.  MODE_LIST: arrays anywhere in
// memory, given as (x, y, n) descriptors; every array starts a new tile.
enum ScanMode : int {
    MODE_SINGLE = 0,
    MODE_SEGMENTED = 1,
    MODE_LIST = 2,
    MODE_COUNT = 3
};

// One array of a MODE_LIST launch.
struct SegDesc {
    const void *x;
    void *y;
    int64_t n;
};

// How a tile obtains the prefix of everything before it (Section 4.3).
enum CarryMode : int {
    CARRY_LOOKBACK = 0,  // decoupled look-back over predecessors' statuses
    CARRY_CHAINED = 1    // wait for the left neighbour's inclusive prefix
};

struct ScanParams {
    const void *x;
    void *y;
    int64_t n;        // elements
    int64_t n_tiles;  // ceil(n / TILE)
    const int64_t *offsets;  // MODE_SEGMENTED: n_seg + 1 element offsets;
                             // MODE_LIST: n_seg + 1 first-tile indices
    int64_t n_seg;
    const SegDesc *segs;     // MODE_LIST: n_seg descriptors
    uint32_t *ctl;    // CTL_WORDS uint32
    uint64_t *status; // n_tiles * carry words
    uint64_t wait_limit_ns;
    int64_t skip_tile;  // fault injection: never publish this tile (-1: off)
    int32_t inclusive;
    int32_t carry_mode;  // CarryMode
    const void *carry_in;  // MODE_SINGLE: one element (type: carry_in_car) or null
    int32_t carry_in_car;  // 1: carry_in holds the kind's carry type, 0: output type
    int32_t reserved;
    void *total_out;       // MODE_SINGLE: gets x_0 (+) ... (+) x_{n-1} (+ carry-in),
                           // in the carry type, or null
    // stream compaction (x = flags): the values, and where the count goes
    const void *values;
    unsigned long long *count_out;
    // if set: the last CTA moves the launch's device error word here (host
    // memory mapped for the device) and clears it, so a caller polling for
    // completion reads it without a device-to-host copy
    uint32_t *err_host;
    // Single arrays, bulk-copy variants whose thread rows are 32, 64 or 128
    // bytes: x and y viewed as [1024-byte blocks][8][128 bytes] (complete
    // blocks only), through which full tiles are copied with the 128-byte
    // swizzle (encoded by the host at launch; unused otherwise)
    CUtensorMap tm_x;
    CUtensorMap tm_y;
};

// Single-CTA kernel for arrays of at most one tile (no inter-tile carry).
constexpr int kTinyThreads = 256;
constexpr int kTinyItems = 16;
constexpr int kTinyMax = kTinyThreads * kTinyItems;  // 4096 elements

struct TinyParams {
    const void *x;
    void *y;
    int32_t n;  // 1 .. kTinyMax
    int32_t inclusive;
    const void *carry_in;  // one element (type: carry_in_car) or null
    int32_t carry_in_car;  // 1: carry_in holds the kind's carry type, 0: output type
    int32_t reserved;
    void *total_out;       // gets the inclusive total in the carry type, or null
};

// Per-launch constants the wait loops need.
struct WaitCtx {
    uint32_t *ctl;
    uint64_t limit_ns;
    uint32_t epoch;
};

}  // namespace lscan
