// kernel_table.h -- registry of compiled scan kernels (host side).
#pragma once
#include <cstdint>

#include "scan_common.h"

namespace lscan {

// Variant 0 is the plain-load path for pointers that are not 16-byte
// aligned; variants 1..kNumTmaCfg are bulk-copy (TMA) tile configurations
// of single-array scans, of which batched scans have the first kMultiCfg.
constexpr int kNumTmaCfg = 17;
constexpr int kMultiCfg = 6;
constexpr int kNumVariants = 1 + kNumTmaCfg;
constexpr int kNumKinds = 23;
// most status words any kernel uses per tile (fixed-size scratch is sized
// with it)
constexpr int kMaxSlotWords = 16;

struct KernelEntry {
    const void *fn = nullptr;
    int threads = 0;   // CTA size (consumer warps + 1 producer warp)
    int smem = 0;      // dynamic shared memory bytes
    int tile = 0;      // elements per tile
    int items = 0;     // elements per consumer thread
    int cwarps = 0;    // consumer warps
    int stages = 0;    // tile-ring depth
    int run = 1;       // consecutive tiles per ticket
    int car_words = 0; // 64-bit status words per tile slot
    int in_size = 0;
    int out_size = 0;
    // thread row bytes (32, 64 or 128) where full tiles of x (into the
    // ring) and of y (out of the staging) move as 128-byte-swizzled tensor
    // copies, 0 where the variant uses plain bulk copies; the launch encodes
    // ScanParams::tm_x / tm_y when they are set
    int swz_in = 0;
    int swz_out = 0;
};

// [kind][mode][variant]
extern KernelEntry g_kernels[kNumKinds][MODE_COUNT][kNumVariants];
// [kind]: the single-CTA kernel for n <= kTinyMax
extern const void *g_tiny_kernels[kNumKinds];
// [kind]: the reduction to the kind's carry type (sharded scans), and the
// carry type's size in bytes
extern const void *g_reduce_kernels[kNumKinds];
extern int g_carry_bytes[kNumKinds];

void register_all_kernels();

}  // namespace lscan
