// scan_kernel.cuh -- persistent single-pass scan kernel for sm_103a.
//
// Structure (LightScan Section 4, re-designed for GB300):
//  * Work decomposition (Section 4 intro, Algorithm 1).  x is cut into tiles
//    of L = ITEMS * CTHREADS elements.  A persistent grid of CTAs takes tiles
//    in ascending order from an atomic ticket (the paper deals them
//    cyclically to exactly #SM blocks, which deadlocks when not every block
//    is resident; the ticket keeps the "earlier tiles are owned by running
//    blocks" property under any residency, e.g. beside concurrent kernels).
//  * Loads (Section 4.1 step 1, Section 4.5).  One producer warp per CTA
//    copies whole tiles (tensor copies with the 128-byte swizzle, or plain
//    bulk copies) into a STAGES-deep shared-memory ring, STAGES-1 tiles
//    ahead, so HBM reads stay in flight while the consumer warps wait on a
//    carry (a ragged last tile: a bulk copy of its 16-byte-aligned prefix,
//    the last few bytes copied by the producer lanes).  x is read once.
//  * Intra-warp local scan (Section 4.1, Algorithm 2).  Each thread holds
//    ITEMS consecutive elements (16-byte shared-memory reads that cover all
//    32 banks per quarter-warp: swizzled tiles, or XOR-rotated reads), scans
//    them sequentially (the matrix-scan row of Section 2.3), then the warp
//    runs the Hillis-Steele shuffle scan of Section 2.1 on the 32 thread
//    totals (5 rounds of shfl.up).
//  * Intra-block local scan (Section 4.2, Algorithm 3).  Lane 31 of each warp
//    writes the warp total to a <=32-entry shared array; every warp scans that
//    array with shuffles (redundantly, which saves the second barrier of
//    Algorithm 3) and takes its own offset and the tile aggregate.
//  * Inter-block communication (Section 4.3, Algorithm 4).  One status word
//    per tile in L2 carries payload and flag in a single 64-bit relaxed
//    gpu-scope access (the paper's single-transaction (u, v) pair).  Two
//    protocols: CHAINED waits for tile t-1's inclusive prefix only
//    (Algorithm 4); LOOK-BACK publishes the tile aggregate first and lets a
//    warp combine predecessors' aggregates 32 at a time until it meets an
//    inclusive prefix.  Every wait is bounded by a %globaltimer limit and
//    reports DEV_ERR_CARRY_WAIT instead of hanging.
//  * Intra-block global scan (Section 4.4, Algorithm 5).  Each element gets
//    carry (+) block offset (+) lane offset (+) own prefix, and y is written
//    exactly once: staged per warp in shared memory and stored with a tensor
//    or bulk copy (full tiles) or coalesced plain stores from the staging
//    (the ragged last tile); unaligned pointers take plain stores straight
//    from registers.
//  * Batched mode (MODE_SEGMENTED, not in the paper).  The producer warp
//    marks segment heads of its tile in a bitmap (warp-parallel lower_bound
//    on the offsets); the scan operator is lifted to (head flag, value); a
//    tile that contains a head publishes its inclusive status immediately.
#pragma once
#include <cstdint>
#include <type_traits>

#include "kinds.cuh"
#include "ptx.cuh"
#include "scan_common.h"
#include "tile_chain.cuh"

namespace lscan {

template <int ITEMS_, int CWARPS_, int STAGES_, int OSTAGES_ = 1, int MINB_ = 1,
          int NCARRY_ = 1, int RUN_ = 1, int SLOTW_ = 0>
struct TileCfg {
    static constexpr int ITEMS = ITEMS_;
    static constexpr int CWARPS = CWARPS_;
    static constexpr int STAGES = STAGES_;
    static constexpr int OSTAGES = OSTAGES_;  // output staging buffers (0: direct)
    static constexpr int MINB = MINB_;        // CTAs per SM the registers must fit
    static constexpr int NCARRY = NCARRY_;    // carry warps (ring slots round-robin)
    // consecutive tiles per ticket: only the first tile of a run looks back
    // across CTAs; the others take the inclusive prefix of the CTA's own
    // previous tile
    static constexpr int RUN = RUN_;
    // 64-bit status words per tile slot (0: the rule of status_slot_words)
    static constexpr int SLOTW = SLOTW_;
    static constexpr int CTHREADS = CWARPS * 32;
    // + producer, reducer and NCARRY carry warps
    static constexpr int THREADS = CTHREADS + 64 + 32 * NCARRY;
    static constexpr int TILE = ITEMS * CTHREADS;
};

constexpr int align_up_c(int v, int a) { return (v + a - 1) / a * a; }

template <class Acc>
struct alignas(16) WarpTotal {
    Acc v;
    uint32_t f;
};

// Kinds whose tile aggregate several reducer warps fold (consecutive parts
// of a full tile in shared memory; single arrays) in configurations of one
// CTA per SM -- with two CTAs per SM the second CTA's reducer already sits
// on another sub-partition, and the hand-off costs more than it saves
// (measured) -- how many, and the CTA's thread count.  Three parts put one
// reducer warp on each SM sub-partition but the carry warp's; two where a
// third warp would pass the 1024-thread limit of a CTA.
template <class K, class Cfg, int MODE, bool TMA>
constexpr bool split_reduce() {
    return has_split_reduce<K>::value && MODE == MODE_SINGLE && TMA && Cfg::MINB == 1;
}
template <class K, class Cfg, int MODE, bool TMA>
constexpr int reduce_parts() {
    if constexpr (!split_reduce<K, Cfg, MODE, TMA>()) {
        return 1;
    } else {
        return Cfg::THREADS + 64 <= 1024 ? 3 : 2;
    }
}
template <class K, class Cfg, int MODE, bool TMA>
constexpr int kernel_threads() {
    constexpr int n = Cfg::THREADS + 32 * (reduce_parts<K, Cfg, MODE, TMA>() - 1);
    static_assert(n <= 1024, "a CTA holds at most 1024 threads");
    return n;
}

// Full tiles of a single array move between HBM and shared memory as tensor
// copies with the 128-byte swizzle: in every 1024-byte block of a 1024-byte
// aligned tile, the 16-byte chunk at byte offset b sits at b ^ (((b >> 7) &
// 7) << 4) (swz128).  With thread rows (one consumer thread's elements) of
// 32, 64 or 128 bytes, the eight chunks a quarter-warp reads or writes at
// once then fall in eight distinct 16-byte bank groups while every thread
// reads and writes its chunks in element order: no register permutation
// after the load or before the store.  The other variants (batched modes,
// stream compaction, 16-byte rows, direct stores) keep plain bulk copies
// and the XOR-rotated accesses.
template <class K, class Cfg, int MODE, bool TMA>
struct Swz {
    static constexpr int RBI = Cfg::ITEMS * int(sizeof(typename K::In));
    static constexpr int RBO = Cfg::ITEMS * int(sizeof(typename K::Out));
    static constexpr bool kAny = MODE == MODE_SINGLE && TMA && !is_select<K>::value;
    static constexpr bool IN = kAny && (RBI == 32 || RBI == 64 || RBI == 128);
    static constexpr bool OUT =
        kAny && Cfg::OSTAGES >= 1 && (RBO == 32 || RBO == 64 || RBO == 128);
    // 1024-byte blocks per input tile and per consumer warp's output rows
    static constexpr int kInBlocks = Cfg::TILE * int(sizeof(typename K::In)) / 1024;
    static constexpr int kOutWarpBlocks = 32 * RBO / 1024;
};

// Where the byte at offset `off` of a 1024-byte aligned tile lives under the
// 128-byte swizzle.
__device__ __forceinline__ uint32_t swz128(uint32_t off) {
    return off ^ (((off >> 7) & 7u) << 4);
}

// Shared-memory layout of one CTA.
template <class K, class Cfg, int MODE, bool TMA>
struct Layout {
    using In = typename K::In;
    using Out = typename K::Out;
    static constexpr int kIn = TMA ? Cfg::STAGES * Cfg::TILE * int(sizeof(In)) : 0;
    // output staging: bulk-copy variants, and stream compaction in every
    // variant (it compacts each tile there before a coalesced copy)
    static constexpr int kOut = (TMA || is_select<K>::value)
                                    ? Cfg::OSTAGES * Cfg::TILE * int(sizeof(Out))
                                    : 0;
    static constexpr int kBits =
        MODE != MODE_SINGLE ? Cfg::STAGES * Cfg::TILE / 8 : 0;
    // stream compaction with staged values: each slot's values
    static constexpr int kVal =
        is_staged_select<K>::value ? Cfg::STAGES * Cfg::TILE * int(sizeof(Out)) : 0;
    // (the ring starts the dynamic shared memory; swizzled tiles need
    // 1024-byte boundaries, which every slot size keeps)
    static constexpr int off_in = 0;
    static constexpr int off_val = align_up_c(off_in + kIn, 128);
    static constexpr int off_out =
        align_up_c(off_val + kVal, Swz<K, Cfg, MODE, TMA>::OUT ? 1024 : 128);
    static constexpr int off_bits = align_up_c(off_out + kOut, 128);
    // carry hand-off ring (carry warps -> consumers), deeper than the tile ring
    // so that no input slot waits for a look-back
    static constexpr int CR = 2 * Cfg::STAGES;
    // mbarriers full[ST], empty[ST] (tile slots); ticketed[CR], reduced[CR],
    // carried[CR] (carry ring)
    static constexpr int off_bar = align_up_c(off_bits + kBits, 128);
    static constexpr int off_tile = off_bar + 8 * (2 * Cfg::STAGES + 3 * CR);  // int64[ST]
    static constexpr int off_tr = off_tile + 8 * Cfg::STAGES;       // int64[CR]
    static constexpr int off_agg = off_tr + 8 * CR;                 // Car[CR]
    static constexpr int off_carry = off_agg + 8 * CR;              // CarA[CR]
    // u32 head[CR], stop[CR], head0[CR], inner[ST]
    static constexpr int off_flags = off_carry + 8 * CR;
    // per-slot tile descriptor: x and y of the tile's first element, count
    static constexpr int off_sx = align_up_c(off_flags + 4 * (3 * CR + Cfg::STAGES), 16);  // ptr[ST]
    static constexpr int off_sy = off_sx + 8 * Cfg::STAGES;         // ptr[ST]
    static constexpr int off_snt = off_sy + 8 * Cfg::STAGES;        // i32[ST]
    static constexpr int off_wtot = align_up_c(off_snt + 4 * Cfg::STAGES, 16);
    // warp totals, double-buffered by tile parity (one barrier per tile)
    static constexpr int off_abort = off_wtot + 2 * 16 * Cfg::CWARPS;
    // split reduce: the other reducer warps' part totals (two sets, by ring
    // use parity) and mbarriers half_done[2], half_free[2]
    static constexpr int off_half = align_up_c(off_abort + 16, 16);
    static constexpr int off_hbar =
        off_half + 2 * 16 * (reduce_parts<K, Cfg, MODE, TMA>() > 1
                                 ? reduce_parts<K, Cfg, MODE, TMA>() - 1
                                 : 1);
    static constexpr int bytes = align_up_c(off_hbar + 4 * 8, 128);
    // every field is naturally aligned (a misaligned 8-byte shared access
    // faults the launch)
    static_assert(off_in % 16 == 0 && off_val % 16 == 0 && off_out % 16 == 0 &&
                      off_bits % 16 == 0,
                  "ring");
    static_assert(!Swz<K, Cfg, MODE, TMA>::IN ||
                      (Cfg::TILE * int(sizeof(In))) % 1024 == 0,
                  "swizzled input slots on 1024-byte boundaries");
    static_assert(!Swz<K, Cfg, MODE, TMA>::OUT ||
                      (off_out % 1024 == 0 && (32 * Cfg::ITEMS * int(sizeof(Out))) % 1024 == 0),
                  "swizzled output regions on 1024-byte boundaries");
    static_assert(off_bar % 8 == 0 && off_tile % 8 == 0 && off_tr % 8 == 0 &&
                      off_agg % 8 == 0, "8-byte");
    static_assert(off_carry % 8 == 0 && off_sx % 8 == 0 && off_snt % 4 == 0, "8-byte");
    static_assert(off_wtot % 16 == 0 && off_abort % 4 == 0, "totals");
    static_assert(off_half % 16 == 0 && off_hbar % 8 == 0 && sizeof(typename K::Acc) <= 16,
                  "split reduce");
};

// ------------------------------------------ element <-> 16-byte chunk packs
template <class T>
__device__ __forceinline__ T word_to(uint32_t w) {
    T r;
    memcpy(&r, &w, sizeof(T));
    return r;
}
template <class T>
__device__ __forceinline__ uint32_t to_word(T v) {
    uint32_t w;
    memcpy(&w, &v, sizeof(T));
    return w;
}

template <class E, int ITEMS, int C>
__device__ __forceinline__ void unpack_chunks(const uint4 (&t)[C], E (&e)[ITEMS]) {
    static_assert(ITEMS * sizeof(E) == 16 * C, "chunk size mismatch");
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const uint32_t w[4] = {t[c].x, t[c].y, t[c].z, t[c].w};
        if constexpr (sizeof(E) == 8) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const uint64_t d = static_cast<uint64_t>(w[2 * q]) |
                                   (static_cast<uint64_t>(w[2 * q + 1]) << 32);
                memcpy(&e[2 * c + q], &d, 8);
            }
        } else if constexpr (sizeof(E) == 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) e[4 * c + q] = word_to<E>(w[q]);
        } else if constexpr (sizeof(E) == 2) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                e[8 * c + 2 * q] = static_cast<E>(w[q] & 0xffffu);
                e[8 * c + 2 * q + 1] = static_cast<E>(w[q] >> 16);
            }
        } else {
            static_assert(sizeof(E) == 1, "1-, 2-, 4- or 8-byte elements");
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    e[16 * c + 4 * q + b] = static_cast<E>((w[q] >> (8 * b)) & 0xffu);
        }
    }
}

template <class E, int ITEMS, int C>
__device__ __forceinline__ void pack_chunks(const E (&e)[ITEMS], uint4 (&t)[C]) {
    static_assert(ITEMS * sizeof(E) == 16 * C, "chunk size mismatch");
#pragma unroll
    for (int c = 0; c < C; ++c) {
        uint32_t w[4];
        if constexpr (sizeof(E) == 8) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                uint64_t d;
                memcpy(&d, &e[2 * c + q], 8);
                w[2 * q] = static_cast<uint32_t>(d);
                w[2 * q + 1] = static_cast<uint32_t>(d >> 32);
            }
        } else if constexpr (sizeof(E) == 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q] = to_word(e[4 * c + q]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                w[q] = static_cast<uint32_t>(e[8 * c + 2 * q]) |
                       (static_cast<uint32_t>(e[8 * c + 2 * q + 1]) << 16);
        }
        t[c] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// t[j] <- t[j ^ xr] for all j (an involution), done with selects.
template <int C>
__device__ __forceinline__ void xor_permute(uint4 (&t)[C], uint32_t xr) {
#pragma unroll
    for (int b = 1; b < C; b <<= 1) {
        const bool sw = (xr & b) != 0;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if (!(j & b)) {
                uint4 a = t[j], c = t[j | b];
                t[j] = sw ? c : a;
                t[j | b] = sw ? a : c;
            }
        }
    }
}

// Rotation that makes each quarter-warp's 16-byte accesses hit 8 distinct
// 16-byte bank groups when every lane owns C consecutive chunks.
template <int C>
__device__ __forceinline__ uint32_t chunk_rot(int lane) {
    if constexpr (C == 1) {
        return 0u;
    } else {
        return static_cast<uint32_t>((lane / (8 / C)) % C);
    }
}

// Thread-blocked load of ITEMS elements (row `row` of a shared-memory
// tile).  SW: the tile is swizzled (swz128), so chunk j of the row is read
// where the swizzle put it and lands in order; otherwise the row is dense and
// the chunks, read in the rotated order, are put back in order with selects.
template <class E, int ITEMS, bool SW = false>
__device__ __forceinline__ void lds_blocked(const uint8_t *tile_smem, int row,
                                            int lane, E (&e)[ITEMS]) {
    constexpr int BYTES = ITEMS * int(sizeof(E));
    constexpr int C = BYTES / 16;
    static_assert(C >= 1 && C <= 8 && (C & (C - 1)) == 0, "1..8 chunks");
    uint4 t[C];
    if constexpr (SW) {
        // the row's chunks stay inside one 128-byte line: one XOR mask
        const uint32_t base = static_cast<uint32_t>(row) * BYTES;
        const uint32_t xm = ((base >> 7) & 7u) << 4;
#pragma unroll
        for (int j = 0; j < C; ++j)
            t[j] = *reinterpret_cast<const uint4 *>(tile_smem + ((base + 16u * j) ^ xm));
    } else {
        const uint8_t *p = tile_smem + row * BYTES;
        const uint32_t xr = chunk_rot<C>(lane);
#pragma unroll
        for (int j = 0; j < C; ++j)
            t[j] = *reinterpret_cast<const uint4 *>(p + 16 * (j ^ xr));
        xor_permute<C>(t, xr);
    }
    unpack_chunks<E, ITEMS, C>(t, e);
}

// Thread-blocked store of ITEMS elements into row `idx` of a shared-memory
// region (SW: the region is swizzled, as in lds_blocked).
template <class E, int ITEMS, bool SW = false>
__device__ __forceinline__ void sts_blocked(uint8_t *region, int idx, int lane,
                                            const E (&e)[ITEMS]) {
    constexpr int BYTES = ITEMS * int(sizeof(E));
    constexpr int C = BYTES / 16;
    static_assert(C >= 1 && C <= 8 && (C & (C - 1)) == 0, "1..8 chunks");
    uint4 t[C];
    pack_chunks<E, ITEMS, C>(e, t);
    if constexpr (SW) {
        const uint32_t base = static_cast<uint32_t>(idx) * BYTES;
        const uint32_t xm = ((base >> 7) & 7u) << 4;
#pragma unroll
        for (int j = 0; j < C; ++j)
            *reinterpret_cast<uint4 *>(region + ((base + 16u * j) ^ xm)) = t[j];
    } else {
        uint8_t *p = region + idx * BYTES;
        const uint32_t xr = chunk_rot<C>(lane);
        xor_permute<C>(t, xr);
#pragma unroll
        for (int j = 0; j < C; ++j)
            *reinterpret_cast<uint4 *>(p + 16 * (j ^ xr)) = t[j];
    }
}

// The carry-in of a single-array scan: the caller's output-type element, a
// carry-type value (the total a previous chunk of the same array handed on),
// or the operator's identity.
template <class K>
__device__ __forceinline__ typename K::Car carry_in_of(const ScanParams &p) {
    if (p.carry_in == nullptr) return K::cident();
    if (p.carry_in_car) return *static_cast<const typename K::Car *>(p.carry_in);
    return K::car_of_out(*static_cast<const typename K::Out *>(p.carry_in));
}

// First index i in [0, cnt) with a[i] >= key (cnt if none); whole warp.
__device__ __forceinline__ int64_t warp_lower_bound(const int64_t *a,
                                                    int64_t cnt, int64_t key,
                                                    int lane) {
    int64_t lo = 0, hi = cnt;
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t probe = lo + static_cast<int64_t>(lane + 1) * step - 1;
        const bool ge = probe >= hi ? true : (a[probe] >= key);
        const uint32_t m = __ballot_sync(0xffffffffu, ge);
        if (m == 0) return hi;
        const int b = __ffs(m) - 1;
        const int64_t nlo = lo + static_cast<int64_t>(b) * step;
        const int64_t nhi = lo + static_cast<int64_t>(b + 1) * step;
        lo = nlo;
        hi = nhi < hi ? nhi : hi;
    }
    if (lo >= hi) return hi;
    const int64_t i = lo + lane;
    const bool ge = i >= hi ? true : (a[i] >= key);
    const uint32_t m = __ballot_sync(0xffffffffu, ge);
    if (m == 0) return hi;
    const int64_t r = lo + (__ffs(m) - 1);
    return r < hi ? r : hi;
}

// Reduction of a tile in any order: the operators are commutative (float max
// keeps the first occurrence through the element index).
template <class K>
struct TileReduce {
    using Acc = typename K::Acc;
    Acc v;
    int32_t i;
    __device__ void init() {
        v = K::ident();
        i = INT32_MAX;
    }
    __device__ void add(Acc x, int32_t idx) {
        if constexpr (K::kTieOrdered) {
            if (K::gt(x, v) || (!K::gt(v, x) && idx < i)) {
                v = x;
                i = idx;
            }
        } else {
            v = K::op(v, x);
        }
    }
    // x comes after every element folded so far (a left fold)
    __device__ void add_in_order(Acc x, int32_t idx) {
        if constexpr (K::kTieOrdered) {
            if (K::gt(x, v)) {
                v = x;
                i = idx;
            }
        } else {
            v = op_step<K>(v, x);  // x is one element
        }
    }
    __device__ void warp_all() {
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const Acc ov = shfl_idx_any(v, (threadIdx.x ^ off) & 31);
            const int32_t oi = __shfl_xor_sync(0xffffffffu, i, off);
            add(ov, oi);
        }
    }
};

// Maximum of a full tile of fp32 or bf16 values under the scan's rule
// (first occurrence on ties, so +0 and -0 compare equal), found on the raw
// bits by one warp.  As signed integers the bits of non-negative floats
// order like their values, and those of negative floats in reverse with -0
// the smallest: so the signed maximum m1 of the raw bits is the largest
// non-negative value when there is one (m1 >= 0), and otherwise the signed
// minimum m2 is the negative value closest to zero (-0 if present; then no
// +0 exists and every zero of the tile is -0).  Equal values other than
// zeros have equal bits, so the result is exact except when the maximum is
// +0 and a -0 may precede it: only then (m1 == 0) the tile is searched for
// its first zero.  Two integer min/max per element (bf16: per two elements,
// 16-bit SIMD) instead of a compare-select chain with index tracking.
// SW: the tile is swizzled (swz128); only the search for the first zero
// depends on where each element sits.
template <class In, int TILE, bool SW = false>
__device__ __forceinline__ float raw_float_max_tile(const uint8_t *tsm, int lane) {
    constexpr int WORDS = TILE * int(sizeof(In)) / 4;
    const uint4 *q4 = reinterpret_cast<const uint4 *>(tsm);
    int32_t m1, m2;
    if constexpr (sizeof(In) == 4) {
        m1 = INT32_MIN;
        m2 = INT32_MAX;
        for (int c = lane; c < WORDS / 4; c += 32) {
            const uint4 q = q4[c];
            const int32_t w[4] = {int32_t(q.x), int32_t(q.y), int32_t(q.z), int32_t(q.w)};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                m1 = max(m1, w[j]);
                m2 = min(m2, w[j]);
            }
        }
    } else {
        static_assert(sizeof(In) == 2, "fp32 or bf16");
        uint32_t p1 = 0x80008000u, p2 = 0x7fff7fffu;  // per 16-bit half
        for (int c = lane; c < WORDS / 4; c += 32) {
            const uint4 q = q4[c];
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                p1 = __vmaxs2(p1, w[j]);
                p2 = __vmins2(p2, w[j]);
            }
        }
        m1 = max(int32_t(int16_t(p1 & 0xffffu)), int32_t(int16_t(p1 >> 16)));
        m2 = min(int32_t(int16_t(p2 & 0xffffu)), int32_t(int16_t(p2 >> 16)));
    }
    m1 = __reduce_max_sync(0xffffffffu, m1);
    m2 = __reduce_min_sync(0xffffffffu, m2);
    uint32_t bits;
    if (m1 > 0) {
        bits = static_cast<uint32_t>(m1);
    } else if (m1 < 0) {
        bits = static_cast<uint32_t>(m2);
    } else {
        // the maximum is a zero: the first zero of the tile decides its sign
        // the elements' bit patterns (an unsigned word of the element's size)
        using Bits = std::conditional_t<sizeof(In) == 4, uint32_t, uint16_t>;
        constexpr uint32_t MAG = sizeof(In) == 4 ? 0x7fffffffu : 0x7fffu;
        const Bits *e = reinterpret_cast<const Bits *>(tsm);
        bits = 0u;
        for (int base = 0; base < TILE; base += 32) {
            int i = base + lane;
            if constexpr (SW)
                i = static_cast<int>(swz128(static_cast<uint32_t>(i) * sizeof(In)) / sizeof(In));
            const uint32_t b = static_cast<uint32_t>(e[i]);
            const uint32_t z = __ballot_sync(0xffffffffu, (b & MAG) == 0u);
            if (z) {
                bits = __shfl_sync(0xffffffffu, b, __ffs(z) - 1);
                break;
            }
        }
    }
    if constexpr (sizeof(In) == 4) {
        return __uint_as_float(bits);
    } else {
        return __uint_as_float((bits & 0xffffu) << 16);
    }
}

// Two signed 16-bit maxima in one instruction (per half of the word).
__device__ __forceinline__ uint32_t vmax_s16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// bf16 max scanned on packed pairs of raw bits.  Once the running maximum
// is a positive float, the order of positive floats is the order of their
// bits read as signed 16-bit integers, and every negative value or zero
// reads as a smaller integer than any positive one: the running maximum of
// the raw bits is then bit-exact (equal positive values have equal bits).
// A pair (lo, hi) with running maximum R in both halves gives, with two
// 16-bit SIMD maxima and two byte permutes, its inclusive outputs
// (max(R, lo), max(R, lo, hi)) and the next R.
template <bool INCL>
__device__ __forceinline__ uint32_t packed_max_step(uint32_t w, uint32_t &R) {
    const uint32_t ps = vmax_s16x2(vmax_s16x2(w, __byte_perm(w, 0u, 0x1010u)), R);
    const uint32_t o = INCL ? ps : __byte_perm(R, ps, 0x5410u);  // (R, max(R, lo))
    R = __byte_perm(ps, 0u, 0x3232u);
    return o;
}

// ------------------------------------------------------------------ kernel
template <class K, class Cfg, int MODE, bool TMA>
__global__ void __launch_bounds__(kernel_threads<K, Cfg, MODE, TMA>(), Cfg::MINB)
    lscan_kernel(const __grid_constant__ ScanParams p) {
    using In = typename K::In;
    using Out = typename K::Out;
    using Acc = typename K::Acc;
    using Car = typename K::Car;
    using CarA = typename K::CarA;
    using L = Layout<K, Cfg, MODE, TMA>;
    constexpr int ITEMS = Cfg::ITEMS;
    constexpr int CW = Cfg::CWARPS;
    constexpr int CT = Cfg::CTHREADS;
    constexpr int TILE = Cfg::TILE;
    constexpr int ST = Cfg::STAGES;
    constexpr int OS = Cfg::OSTAGES;
    constexpr bool SEG = MODE != MODE_SINGLE;  // segment heads exist
    constexpr int NC = Cfg::NCARRY;
    constexpr int CR = L::CR;
    constexpr int SLOT = status_slot_words<K, Cfg>();  // status words per tile
    constexpr int W_PROD = CW, W_RED = CW + 1, W_CARRY = CW + 2;  // .. + NC - 1
    // split reduce: NRP - 1 more reducer warps after the carry warps
    constexpr bool SPLIT = split_reduce<K, Cfg, MODE, TMA>();
    constexpr int NRP = reduce_parts<K, Cfg, MODE, TMA>();
    constexpr int W_RED2 = W_CARRY + NC;
    // full tiles of x in and of y out as swizzled tensor copies (Swz)
    constexpr bool SWI = Swz<K, Cfg, MODE, TMA>::IN;
    constexpr bool SWO = Swz<K, Cfg, MODE, TMA>::OUT;
    constexpr int kInBlocks = Swz<K, Cfg, MODE, TMA>::kInBlocks;
    constexpr int kOutWarpBlocks = Swz<K, Cfg, MODE, TMA>::kOutWarpBlocks;
    static_assert(ITEMS <= 32 && (32 % ITEMS) == 0, "head bits in one word");
    static_assert(OS >= 0 && OS <= 2, "0 (direct stores), 1 or 2 staging buffers");
    // Each carry warp must see every phase of the ring entries it waits on
    // (an mbarrier parity wait aliases if a phase is skipped), so carry warp
    // c always takes the same entries: CR = 2 ST must be a multiple of NC.
    // NC <= ST also keeps the terminator hand-off below safe.
    static_assert(NC >= 1 && ST % NC == 0, "carry warps must own whole entries");

    extern __shared__ __align__(1024) uint8_t smem[];
    // Tile slots (input data, per slot s = k % ST of ring use k) and the
    // carry ring (per entry c = k % CR): the carry warp only touches the
    // ring, so it never holds an input slot while it looks back.
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::off_bar);
    uint64_t *empty = full + ST;       // slot consumed: consumer warps + reducer
    uint64_t *ticketed = empty + ST;   // [CR] producer: tile index, head0
    uint64_t *reduced = ticketed + CR;  // [CR] reducer: tile aggregate published
    uint64_t *carried = reduced + CR;  // [CR] carry warp: the tile's carry
    volatile int64_t *tile_of = reinterpret_cast<int64_t *>(smem + L::off_tile);  // [ST]
    volatile int64_t *tile_r = reinterpret_cast<int64_t *>(smem + L::off_tr);     // [CR]
    Car *agg_r = reinterpret_cast<Car *>(smem + L::off_agg);        // [CR] reducer -> carry
    CarA *carry_s = reinterpret_cast<CarA *>(smem + L::off_carry);  // [CR] carry -> consumers
    volatile uint32_t *head_r = reinterpret_cast<uint32_t *>(smem + L::off_flags);  // [CR]
    volatile uint32_t *stop_s = head_r + CR;   // [CR]
    volatile uint32_t *head0_r = stop_s + CR;  // [CR] head at the tile's first element
    // tile has a segment head after its first element (segmented code needed)
    volatile uint32_t *inner_s = head0_r + CR;  // [ST]
    WarpTotal<Acc> *wtot = reinterpret_cast<WarpTotal<Acc> *>(smem + L::off_wtot);
    volatile uint32_t *abort_s = reinterpret_cast<uint32_t *>(smem + L::off_abort);
    uint32_t *bits = reinterpret_cast<uint32_t *>(smem + L::off_bits);
    Acc *half_s = reinterpret_cast<Acc *>(smem + L::off_half);   // [2][NRP - 1]
    uint64_t *half_done = reinterpret_cast<uint64_t *>(smem + L::off_hbar);  // [2]
    uint64_t *half_free = half_done + 2;                                 // [2]
    const In *volatile *slot_x = reinterpret_cast<const In *volatile *>(smem + L::off_sx);
    Out *volatile *slot_y = reinterpret_cast<Out *volatile *>(smem + L::off_sy);
    volatile int32_t *slot_nt = reinterpret_cast<int32_t *>(smem + L::off_snt);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CW + NRP);  // consumer warps + reducer warps
            tile_of[s] = INT64_MAX;
            inner_s[s] = 0;
        }
        for (int c = 0; c < CR; ++c) {
            mbar_init(&ticketed[c], 1);
            mbar_init(&reduced[c], 1);
            mbar_init(&carried[c], 1);
            tile_r[c] = INT64_MAX;
            head_r[c] = 0;
            head0_r[c] = 0;
            stop_s[c] = 0;
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&half_done[b], NRP > 1 ? NRP - 1 : 1);
            mbar_init(&half_free[b], 1);
        }
        *abort_s = 0;
        fence_mbar_init();
    }
    __syncthreads();
    // Launched with programmatic stream serialization, this CTA may start
    // while the previous kernel of the stream still runs: everything above
    // touched only this CTA's shared memory.  Wait for that kernel (its
    // writes, and the scratch it re-armed at its end, are then visible),
    // then let the next kernel's CTAs be scheduled early in turn.
    grid_dependency_wait();
    grid_launch_dependents();

    const uint32_t epoch = *reinterpret_cast<volatile uint32_t *>(p.ctl + CTL_EPOCH);
    const uint32_t ebase = (epoch & kEpochMask) << 2;
    const WaitCtx wc{p.ctl, p.wait_limit_ns, epoch};
    const In *__restrict__ x = static_cast<const In *>(p.x);
    Out *__restrict__ y = static_cast<Out *>(p.y);

    // The swizzle places chunks by shared-memory address bits 4 .. 9, so
    // the tile ring and the output staging start on 1024-byte boundaries;
    // should the dynamic shared memory not, nothing runs and the launch
    // reports it (its CTAs still take part in the launch-end count).
    const bool misaligned = (SWI || SWO) && (smem_addr(smem) & 1023u) != 0u;
    if (misaligned) {
        if (tid == 0) note_gave_up(wc, DEV_ERR_SMEM_ALIGN);
    } else if (warp == W_PROD) {
        // ============================ producer warp ============================
        uint32_t armed_mask = 0;  // slots whose last phase was a bulk copy
        uint32_t par_mask = 0;    // parity of each slot's last bulk copy
        // A CTA's tickets only increase, so the array (list mode) or the
        // next segment head (segmented mode) of its next tile lies at or
        // after the one its previous tile needed: both searches resume here.
        int64_t cur = 0;
        int64_t t = 0;     // tile of this ring use
        int run_left = 0;  // tiles of the current run not yet issued
        for (int64_t k = 0;; ++k) {
            const int s = static_cast<int>(k % ST);
            if (k >= ST) {
                // lane 0 waits; the decision is made warp-uniform
                bool ok = true;
                if (lane == 0)
                    ok = wait_phase(&empty[s], static_cast<uint32_t>(((k / ST) - 1) & 1), wc);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                __syncwarp();
                if (!ok) {
                    if (lane == 0) *abort_s = 1;
                    break;
                }
            }
            if (run_left == 0 || t + 1 >= p.n_tiles) {
                // a ticket hands out a run of RUN consecutive tiles
                int64_t u = 0;
                if (lane == 0) u = static_cast<int64_t>(atomicAdd(p.ctl + CTL_TICKET, 1u));
                t = __shfl_sync(0xffffffffu, u, 0) * Cfg::RUN;
                run_left = Cfg::RUN - 1;
            } else {
                ++t;
                --run_left;
            }
            if (lane == 0) tile_of[s] = t;
            if (t >= p.n_tiles) {
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&full[s]);     // consumer warps and reducer stop
                    armed_mask &= ~(1u << s);  // this slot's last phase is plain
                    // every carry warp stops at its next ring use: uses k ..
                    // k + NC - 1.  Entry (k + j) % CR was last used by
                    // k + j - 2 ST <= k - ST - 1 (NC <= ST), whose carry the
                    // consumers took before releasing slot s for use k.
                    for (int64_t j = 0; j < NC; ++j) {
                        const int cj = static_cast<int>((k + j) % CR);
                        tile_r[cj] = INT64_MAX;
                        mbar_arrive(&ticketed[cj]);
                    }
                }
                break;
            }
            // ---- tile descriptor: where the tile's elements live ----
            const In *tx;
            Out *ty;
            int nt;
            bool list_head = false;
            int64_t ts = 0, te = 0;
            if constexpr (MODE == MODE_LIST) {
                // array holding tile t: the last a with first_tile[a] <= t.
                // One round of independent loads probes arrays cur .. cur+31
                // (their descriptors and the next arrays' first tiles); a
                // binary search covers longer jumps.
                const int64_t j = cur + lane;
                const int64_t fnext = (j + 1 <= p.n_seg) ? p.offsets[j + 1] : INT64_MAX;
                SegDesc dj{nullptr, nullptr, 0};
                if (j < p.n_seg) dj = p.segs[j];
                const uint32_t m = __ballot_sync(0xffffffffu, fnext > t);
                SegDesc d;
                if (m) {
                    const int b = __ffs(m) - 1;
                    cur += b;
                    d.x = reinterpret_cast<const void *>(__shfl_sync(
                        0xffffffffu, reinterpret_cast<unsigned long long>(dj.x), b));
                    d.y = reinterpret_cast<void *>(__shfl_sync(
                        0xffffffffu, reinterpret_cast<unsigned long long>(dj.y), b));
                    d.n = __shfl_sync(0xffffffffu, static_cast<long long>(dj.n), b);
                } else {
                    // first_tile[cur+1 .. cur+32] <= t, so cur + 32 < n_seg
                    const int64_t lo = cur + 33;
                    cur = lo + warp_lower_bound(p.offsets + lo, p.n_seg + 1 - lo, t + 1, lane) - 1;
                    d = p.segs[cur];
                }
                const int64_t lt = t - p.offsets[cur];
                const int64_t left = d.n - lt * TILE;
                nt = left < TILE ? static_cast<int>(left) : TILE;
                tx = static_cast<const In *>(d.x) + lt * TILE;
                ty = static_cast<Out *>(d.y) + lt * TILE;
                list_head = lt == 0;
            } else {
                ts = t * TILE;
                te = (ts + TILE < p.n) ? ts + TILE : p.n;
                nt = static_cast<int>(te - ts);
                tx = x + ts;
                ty = y + ts;
            }
            // A full tile is one bulk copy; a partial tile (the end of an
            // array) a bulk copy of its 16-byte-aligned prefix plus the last
            // few bytes copied by the lanes, so that it is read from shared
            // memory like a full tile.
            const uint32_t tbytes = static_cast<uint32_t>(nt) * uint32_t(sizeof(In));
            const uint32_t bulk_bytes = TMA ? (tbytes & ~15u) : 0u;
            // stream compaction with staged values: the tile's values follow
            // its flags into the slot (a bulk copy of their 16-byte prefix
            // when the flags take one, the rest by the lanes)
            constexpr bool SV = is_staged_select<K>::value;
            const Out *tv = SV ? static_cast<const Out *>(p.values) + ts : nullptr;
            const uint32_t vbulk =
                (SV && bulk_bytes > 0u) ? (static_cast<uint32_t>(nt) * uint32_t(sizeof(Out))) & ~15u
                                        : 0u;
            if (lane == 0) {
                slot_x[s] = tx;
                slot_y[s] = ty;
                slot_nt[s] = nt;
                if (bulk_bytes > 0u) {
                    // start the copy now; the slot's phase also needs the
                    // arrival below, made once the head bitmap is written
                    mbar_expect_tx(&full[s], bulk_bytes + vbulk);
                    if (SWI && nt == TILE) {
                        // the tile is 1024-byte blocks t kInBlocks .. of x's map
                        tensor_g2s_3d(smem + L::off_in + s * TILE * sizeof(In), &p.tm_x, 0, 0,
                                      static_cast<int>(t * kInBlocks), &full[s]);
                    } else {
                        bulk_g2s(smem + L::off_in + s * TILE * sizeof(In), tx, bulk_bytes,
                                 &full[s]);
                    }
                    if (vbulk > 0u)
                        bulk_g2s(smem + L::off_val + s * TILE * sizeof(Out), tv, vbulk, &full[s]);
                    armed_mask |= 1u << s;
                    par_mask = (par_mask & ~(1u << s)) |
                               (static_cast<uint32_t>((k / ST) & 1) << s);
                } else {
                    armed_mask &= ~(1u << s);
                }
            }
            if constexpr (TMA) {
                if (bulk_bytes < tbytes) {
                    In *sin = reinterpret_cast<In *>(smem + L::off_in + s * TILE * sizeof(In));
                    for (int i = static_cast<int>(bulk_bytes / sizeof(In)) + lane; i < nt; i += 32)
                        sin[i] = tx[i];
                    // these generic writes precede the slot's next bulk copy
                    fence_proxy_async_smem();
                }
                if constexpr (SV) {
                    if (vbulk < static_cast<uint32_t>(nt) * uint32_t(sizeof(Out))) {
                        Out *sv = reinterpret_cast<Out *>(smem + L::off_val + s * TILE * sizeof(Out));
                        for (int i = static_cast<int>(vbulk / sizeof(Out)) + lane; i < nt; i += 32)
                            sv[i] = tv[i];
                        fence_proxy_async_smem();
                    }
                }
            }
            if constexpr (MODE == MODE_LIST) {
                uint32_t *bm = bits + s * (TILE / 32);
                for (int i = lane; i < TILE / 32; i += 32) bm[i] = 0u;
                __syncwarp();
                if (lane == 0) {
                    if (list_head) bm[0] = 1u;  // each array starts a chain
                    inner_s[s] = 0u;            // its only head is element 0
                }
                __threadfence_block();
            } else if constexpr (SEG) {
                // heads in [ts, te), from the first offset not below the
                // previous tile's end; a binary search skips runs of more
                // than 32 offsets that lie before ts
                uint32_t *bm = bits + s * (TILE / 32);
                for (int i = lane; i < TILE / 32; i += 32) bm[i] = 0u;
                __syncwarp();
                int64_t i0 = cur;
                int64_t o = (i0 + lane <= p.n_seg) ? p.offsets[i0 + lane] : INT64_MAX;
                if (__ballot_sync(0xffffffffu, o >= ts) == 0u) {
                    // offsets[i0 .. i0+31] < ts, so i0 + 31 <= n_seg
                    const int64_t lo = i0 + 32;
                    i0 = lo + warp_lower_bound(p.offsets + lo, p.n_seg + 1 - lo, ts, lane);
                    o = (i0 + lane <= p.n_seg) ? p.offsets[i0 + lane] : INT64_MAX;
                }
                bool inner = false;
                while (true) {
                    if (o >= ts && o < te) {
                        const int64_t r = o - ts;
                        atomicOr(&bm[r >> 5], 1u << (r & 31));
                    }
                    inner = inner || __any_sync(0xffffffffu, o > ts && o < te);
                    const uint32_t before_end = __ballot_sync(0xffffffffu, o < te);
                    if (before_end != 0xffffffffu) {
                        cur = i0 + __popc(before_end);  // offsets are sorted
                        break;
                    }
                    i0 += 32;
                    o = (i0 + lane <= p.n_seg) ? p.offsets[i0 + lane] : INT64_MAX;
                }
                if (lane == 0) inner_s[s] = inner ? 1u : 0u;
                __threadfence_block();
            }
            __syncwarp();
            if (lane == 0) {
                // the carry warp may start this tile's look-back now, while
                // its data is still in flight
                const int c = static_cast<int>(k % CR);
                tile_r[c] = t;
                bool h0 = false;
                if constexpr (MODE == MODE_LIST) {
                    h0 = list_head;
                } else if constexpr (SEG) {
                    h0 = (bits[s * (TILE / 32)] & 1u) != 0u;
                }
                head0_r[c] = h0 ? 1u : 0u;
                mbar_arrive(&ticketed[c]);
                mbar_arrive(&full[s]);
            }
        }
        // Never leave the CTA with a bulk copy still writing its shared memory:
        // wait for every slot whose LAST phase was a bulk copy.  (A slot re-armed
        // by a plain arrive afterwards has had its copy consumed already, and its
        // barrier has moved two phases on, so its old parity must not be tested.)
        if (lane == 0) {
#pragma unroll
            for (int s = 0; s < ST; ++s)
                if (armed_mask & (1u << s))
                    (void)wait_phase(&full[s], (par_mask >> s) & 1u, wc);
        }
    } else if (warp == W_RED || (SPLIT && warp >= W_RED2 && warp < W_RED2 + NRP - 1)) {
        // ======================= reducer warp =========================
        // Publishes each tile's aggregate as soon as its data lands, so the
        // carry of later tiles never waits on this CTA's consumer queue.
        // Split reduce: reducer warp q > 0 folds part q of a full tile and
        // hands its total to the first (half_done, one arrival per part),
        // which combines the parts in order and publishes; the first frees
        // the hand-off buffers (half_free) for the use two tiles later.  All
        // waits are bounded like every other.
        const int part = (SPLIT && warp != W_RED) ? warp - W_RED2 + 1 : 0;
        const bool second = part > 0;
        for (int64_t k = 0;; ++k) {
            const int s = static_cast<int>(k % ST);
            const bool ok = wait_phase(&full[s], static_cast<uint32_t>((k / ST) & 1), wc);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) *abort_s = 1;
                break;
            }
            const int64_t t = __shfl_sync(0xffffffffu, static_cast<long long>(tile_of[s]), 0);
            if (t >= p.n_tiles) break;
            const In *tx = slot_x[s];
            const int nt = slot_nt[s];
            int start = 0;  // reduce elements [start, nt)
            bool has_head = false;
            const bool inner = SEG && inner_s[s] != 0u;
            if (inner) {
                // last segment head in the tile: the aggregate restarts there
                int last = -1;
                for (int w = lane; w < TILE / 32; w += 32) {
                    const uint32_t b = bits[s * (TILE / 32) + w];
                    if (b) last = w * 32 + 31 - __clz(b);
                }
                last = __reduce_max_sync(0xffffffffu, last);
                has_head = last >= 0;
                start = has_head ? last : 0;
            } else if (SEG) {
                has_head = (bits[s * (TILE / 32)] & 1u) != 0u;  // element 0 at most
            }
            TileReduce<K> r;
            r.init();
            // with and without a head inside the tile
            auto reduce_tile = [&](auto seg_tag) {
                constexpr bool SG = decltype(seg_tag)::value;
                if constexpr (has_raw_max<K>::value && !SG && TMA) {
                    if (nt == TILE) {
                        // whole tile, one value: every lane holds it
                        r.v = raw_float_max_tile<In, TILE, SWI>(
                            smem + L::off_in + s * TILE * sizeof(In), lane);
                        r.i = 0;
                        return;
                    }
                }
                if (TMA && nt == TILE) {
                    // one accumulator per element position in a 16-byte chunk:
                    // EPC independent left folds (instruction-level
                    // parallelism), merged with the order-free rule at the end
                    constexpr int EPC = 16 / int(sizeof(In));
                    const uint8_t *tsm = smem + L::off_in + s * TILE * sizeof(In);
                    TileReduce<K> ra[EPC];
#pragma unroll
                    for (int u = 0; u < EPC; ++u) ra[u].init();
                    constexpr int NCH = TILE / EPC;  // 16-byte chunks
                    // parts start on 128-byte lines: eight consecutive
                    // chunks of one line fill the 32 banks once (swizzled or
                    // not); eight that straddle two lines may collide
                    const int c0 = part * (NCH / 8) / NRP * 8;
                    const int c1 = (part + 1) * (NCH / 8) / NRP * 8;
                    for (int c = c0 + lane; c < c1; c += 32) {
                        const uint32_t qo = SWI ? swz128(16u * static_cast<uint32_t>(c))
                                                : 16u * static_cast<uint32_t>(c);
                        const uint4 q = *reinterpret_cast<const uint4 *>(tsm + qo);
                        const uint4 qa[1] = {q};
                        In e[EPC];
                        unpack_chunks<In, EPC, 1>(qa, e);
#pragma unroll
                        for (int u = 0; u < EPC; ++u) {
                            // accumulator u only sees position u of each
                            // chunk: it tracks the chunk index c
                            if (!SG || c * EPC + u >= start)
                                ra[u].add_in_order(K::load(e[u]), c);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < EPC; ++u)
                        r.add(ra[u].v, ra[u].i == INT32_MAX ? INT32_MAX : ra[u].i * EPC + u);
                } else {
                    // partial tile: from the slot (bulk variants) or global
                    const In *src = TMA ? reinterpret_cast<const In *>(
                                              smem + L::off_in + s * TILE * sizeof(In))
                                        : tx;
                    // (split reduce: a partial tile is the first warp's alone)
                    if (!second)
                        for (int i = lane; i < nt; i += 32)
                            if (!SG || i >= start) r.add(K::load(src[i]), i);
                }
            };
            if (inner) {
                reduce_tile(std::true_type{});
            } else {
                reduce_tile(std::false_type{});
            }
            r.warp_all();
            if constexpr (SPLIT) {
                const int b = static_cast<int>(k & 1);
                if (second) {
                    // buffer b was last used two tiles ago: wait until the
                    // first warp has taken that total
                    bool okf = true;
                    if (k >= 2 && lane == 0)
                        okf = wait_phase(&half_free[b], static_cast<uint32_t>(((k - 2) >> 1) & 1), wc);
                    okf = __shfl_sync(0xffffffffu, okf, 0);
                    if (lane == 0) {
                        if (!okf) *abort_s = 1;
                        half_s[b * (NRP - 1) + part - 1] = r.v;
                        mbar_arrive(&half_done[b]);
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[s]);
                    continue;
                }
                bool okh = true;
                if (lane == 0) okh = wait_phase(&half_done[b], static_cast<uint32_t>((k >> 1) & 1), wc);
                okh = __shfl_sync(0xffffffffu, okh, 0);
                if (lane == 0) {
                    if (okh) {
#pragma unroll
                        for (int q = 0; q < NRP - 1; ++q)  // parts in order
                            r.v = K::op(r.v, half_s[b * (NRP - 1) + q]);
                    } else {
                        *abort_s = 1;
                    }
                    mbar_arrive(&half_free[b]);
                }
            }
            if (lane == 0) {
                const Car agg = K::to_car(r.v);
                // tile 0 of a single-array scan with a carry-in publishes
                // carry-in (+) aggregate as its inclusive prefix
                const Car pub = (!SEG && t == 0 && p.carry_in != nullptr)
                                    ? K::cop(carry_in_of<K>(p), agg)
                                    : agg;
                if (t != p.skip_tile)
                    StatusIO<K, SLOT>::publish(p.status, t,
                                         ebase | ((t == 0 || has_head) ? ST_INCLUSIVE
                                                                        : ST_AGGREGATE),
                                         pub);
                const int c = static_cast<int>(k % CR);
                agg_r[c] = agg;
                head_r[c] = has_head ? 1u : 0u;
                mbar_arrive(&reduced[c]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    } else if (warp >= W_CARRY) {
        // ========================= carry warps ==========================
        // Resolve each tile's exclusive prefix (Section 4.3) as soon as the
        // reducer has published the tile's aggregate, running ahead of the
        // consumer warps, and publish the tile's inclusive prefix.  The carry
        // warp reads only the carry ring, so the tile's input slot is
        // released by the consumers and the reducer alone.  Carry warp c
        // takes ring uses k = c, c + NC, ...: the tiles of one CTA are not
        // neighbours (tickets interleave across CTAs), so their look-backs
        // are independent and may overlap.
        static_assert(Cfg::RUN == 1 || NC == 1, "a run's tiles share one carry warp");
        Car run_incl = K::cident();  // inclusive prefix of the last tile carried
        for (int64_t k = warp - W_CARRY;; k += NC) {
            const int c = static_cast<int>(k % CR);
            const uint32_t par = static_cast<uint32_t>((k / CR) & 1);
            const bool okt = wait_phase(&ticketed[c], par, wc);
            if (!__all_sync(0xffffffffu, okt)) {
                if (lane == 0) *abort_s = 1;
                break;
            }
            const int64_t t = __shfl_sync(0xffffffffu, static_cast<long long>(tile_r[c]), 0);
            if (t >= p.n_tiles) break;
            const bool head0 = SEG && head0_r[c] != 0u;
            // Measured on GB300: looking back once the tile's own aggregate
            // is out is as fast for int32 and faster for fp32 add than
            // starting at the ticket (the early look-back only polls longer
            // for predecessors whose data is still in flight).
            const bool okr = wait_phase(&reduced[c], par, wc);
            if (!__all_sync(0xffffffffu, okr) && lane == 0) *abort_s = 1;
            Car excl = K::cident();
            if (t > 0 && !head0) {
                if (Cfg::RUN > 1 && t % Cfg::RUN != 0)
                    excl = run_incl;  // the previous tile of the run is ours
                else
                    excl = p.carry_mode == CARRY_CHAINED
                               ? chained_wait<K, SLOT>(p.status, wc, t, ebase, lane)
                               : lookback<K, SLOT>(p.status, wc, t, ebase, lane);
            } else if (!SEG && t == 0) {
                excl = carry_in_of<K>(p);
            }
            const bool has_head = SEG && head_r[c] != 0u;
            // inclusive prefix of this tile (a tile holding a head restarts
            // at its last head: the reducer's aggregate)
            const Car incl = has_head ? agg_r[c] : K::cop(excl, agg_r[c]);
            if constexpr (Cfg::RUN > 1) run_incl = incl;
            if (lane == 0) {
                // tile 0 and tiles holding a head got theirs from the reducer
                if (t > 0 && !has_head && t != p.skip_tile)
                    StatusIO<K, SLOT>::publish(p.status, t, ebase | ST_INCLUSIVE, incl);
                // the last tile's inclusive prefix is the array's total (the
                // carry-in of the next chunk when an array is scanned in chunks)
                if (!SEG && t == p.n_tiles - 1 && p.total_out != nullptr)
                    *static_cast<Car *>(p.total_out) = incl;
                carry_s[c] = K::to_apply(excl);
                stop_s[c] = *abort_s;  // one snapshot for every consumer warp
                mbar_arrive(&carried[c]);
            }
        }
    } else {
        // ============================ consumer warps ===========================
        const int e0 = tid * ITEMS;  // first element of this thread in a tile
        // Consumer warps leave the loop only together (they share named
        // barriers): each tile starts with a vote.  A warp votes to stop on
        // the terminator, on a wait that ran out (its slot or tile index may
        // then be stale) or when the previous tile's carry did not arrive or
        // came with the abort flag.
        bool stop_next = false;

        // bf16 max, one array: the tile on packed pairs of raw bits
        // (packed_max_step) -- the thread total from 16-bit SIMD maxima, the
        // outputs from a 16-bit SIMD running maximum.  A thread whose total
        // or base is not a positive float (a running maximum that is a zero
        // or negative, where +0 / -0 ties keep the first zero's bits) folds
        // its elements one by one with the kind's tie-ordered operator.
        constexpr bool kPackedMax =
            has_raw_max<K>::value && sizeof(In) == 2 && !SEG && !is_select<K>::value;
        auto packed_max_tile = [&](int s, int64_t k, int64_t t, int nt, bool full_tile,
                                   const In *tx, Out *ty) -> bool {
            (void)t;
            if constexpr (!kPackedMax) {
                return false;
            } else {
            constexpr int NW = ITEMS / 2;  // packed words per thread
            uint32_t w[NW];
            if (TMA && full_tile) {
                lds_blocked<uint32_t, NW, SWI>(smem + L::off_in + s * TILE * sizeof(In), tid,
                                               lane, w);
            } else {
                const uint16_t *src =
                    TMA ? reinterpret_cast<const uint16_t *>(smem + L::off_in +
                                                             s * TILE * sizeof(In))
                        : reinterpret_cast<const uint16_t *>(tx);
#pragma unroll
                for (int i = 0; i < NW; ++i) {
                    const int j = e0 + 2 * i;  // elements past the end: -inf
                    const uint32_t lo = j < nt ? static_cast<uint32_t>(src[j]) : 0xff80u;
                    const uint32_t hi = j + 1 < nt ? static_cast<uint32_t>(src[j + 1]) : 0xff80u;
                    w[i] = lo | (hi << 16);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);  // slot may be refilled
            // element j of this thread (j a compile-time index) as a float
            auto elem = [&](int j) -> Acc {
                const uint32_t b = (j & 1) ? (w[j >> 1] >> 16) : (w[j >> 1] & 0xffffu);
                return __uint_as_float(b << 16);
            };

            // ---- thread total ----
            uint32_t m = w[0];
#pragma unroll
            for (int i = 1; i < NW; ++i) m = vmax_s16x2(m, w[i]);
            const int32_t m1 =
                max(int32_t(int16_t(m & 0xffffu)), int32_t(int16_t(m >> 16)));
            Acc tot;
            if (m1 > 0) {
                tot = __uint_as_float(static_cast<uint32_t>(m1) << 16);
            } else {
                tot = K::ident();
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) tot = K::op(tot, elem(j));
            }

            // ---- warp scan, block scan of warp totals (Algorithm 3) ----
            Acc wv = tot;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const Acc ov = shfl_up_any(wv, d);
                if (lane >= d) wv = K::op(ov, wv);
            }
            Acc lv = shfl_up_any(wv, 1);
            if (lane == 0) lv = K::ident();
            WarpTotal<Acc> *wt = wtot + (k & 1) * CW;
            if (lane == 31) {
                wt[warp].v = wv;
                wt[warp].f = 0u;
            }
            named_bar_sync(1, CT);
            Acc bv = lane < CW ? wt[lane].v : K::ident();
#pragma unroll
            for (int d = 1; d < CW; d <<= 1) {
                const Acc ov = shfl_up_any(bv, d);
                if (lane >= d) bv = K::op(ov, bv);
            }
            Acc wev = shfl_idx_any(bv, warp > 0 ? warp - 1 : 0);
            if (warp == 0) wev = K::ident();
            const Acc tbv = K::op(wev, lv);

            // ---- carry from the carry warp (Section 4.3) ----
            const int cslot = static_cast<int>(k % CR);
            const bool okc = __all_sync(
                0xffffffffu,
                wait_phase(&carried[cslot], static_cast<uint32_t>((k / CR) & 1), wc));
            if (!okc && lane == 0) *abort_s = 1;
            const CarA cin = carry_s[cslot];
            const bool stop = !okc || stop_s[cslot] != 0u;
            const CarA B = K::base(cin, tbv);

            // ---- apply carry and write y once (Section 4.4) ----
            uint32_t o[NW];
            if (B > 0.0f) {
                const uint32_t bb = __float_as_uint(B) >> 16;
                uint32_t R = bb | (bb << 16);
                if (p.inclusive) {
#pragma unroll
                    for (int i = 0; i < NW; ++i) o[i] = packed_max_step<true>(w[i], R);
                } else {
#pragma unroll
                    for (int i = 0; i < NW; ++i) o[i] = packed_max_step<false>(w[i], R);
                }
            } else {
                Acc r = B;
#pragma unroll
                for (int i = 0; i < NW; ++i) {
                    uint32_t ob[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const Acc x = elem(2 * i + h);
                        if (p.inclusive) {
                            r = K::op(r, x);
                            ob[h] = f32_to_bf16_bits_exact(r);
                        } else {
                            ob[h] = f32_to_bf16_bits_exact(r);
                            r = K::op(r, x);
                        }
                    }
                    o[i] = ob[0] | (ob[1] << 16);
                }
            }
            if (TMA && full_tile && OS == 0) {
                constexpr int C = NW * 4 / 16;
                uint4 ov[C];
                pack_chunks<uint32_t, NW, C>(o, ov);
                uint4 *dst = reinterpret_cast<uint4 *>(ty + e0);
#pragma unroll
                for (int j = 0; j < C; ++j) dst[j] = ov[j];
            } else if (TMA && full_tile) {
                constexpr int WBYTES = 32 * ITEMS * int(sizeof(Out));
                uint8_t *region = smem + L::off_out +
                                  (OS == 2 ? (k & 1) : 0) * (TILE * sizeof(Out)) +
                                  warp * WBYTES;
                if (lane == 0) {
                    if constexpr (OS == 2) {
                        bulk_wait_read<1>();
                    } else {
                        bulk_wait_read<0>();
                    }
                }
                __syncwarp();
                sts_blocked<uint32_t, NW, SWO>(region, lane, lane, o);
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (SWO) {
                        tensor_s2g_3d(&p.tm_y, region, 0, 0,
                                      static_cast<int>((t * CW + warp) * kOutWarpBlocks));
                    } else {
                        bulk_s2g(ty + warp * 32 * ITEMS, region, WBYTES);
                    }
                    bulk_commit();
                }
            } else if (TMA && OS >= 1) {
                // partial tile: through this warp's staging region
                constexpr int WE = 32 * ITEMS;
                uint8_t *rb = smem + L::off_out +
                              (OS == 2 ? (k & 1) : 0) * (TILE * sizeof(Out)) +
                              warp * WE * sizeof(Out);
                if (lane == 0) bulk_wait_read<0>();
                __syncwarp();
#pragma unroll
                for (int i = 0; i < NW; ++i) reinterpret_cast<uint32_t *>(rb)[lane * NW + i] = o[i];
                __syncwarp();
                const Out *region = reinterpret_cast<const Out *>(rb);
                const int wbase = warp * WE;
                const int valid = nt - wbase < WE ? nt - wbase : WE;
                for (int j = lane; j < valid; j += 32) ty[wbase + j] = region[j];
                __syncwarp();
            } else {
#pragma unroll
                for (int i = 0; i < NW; ++i) {
                    if (e0 + 2 * i < nt) ty[e0 + 2 * i] = static_cast<Out>(o[i] & 0xffffu);
                    if (e0 + 2 * i + 1 < nt) ty[e0 + 2 * i + 1] = static_cast<Out>(o[i] >> 16);
                }
            }
            return stop;
            }
        };

        for (int64_t k = 0;; ++k) {
            const int s = static_cast<int>(k % ST);
            const uint32_t par = static_cast<uint32_t>((k / ST) & 1);
            const bool ok = __all_sync(0xffffffffu, wait_phase(&full[s], par, wc));
            if (!ok && lane == 0) *abort_s = 1;
            const int64_t t =
                ok ? __shfl_sync(0xffffffffu, static_cast<long long>(tile_of[s]), 0) : INT64_MAX;
            if (named_bar_or(2, CT, !ok || t >= p.n_tiles || stop_next)) break;
            const In *tx = slot_x[s];
            Out *ty = slot_y[s];
            const int nt = slot_nt[s];
            const bool full_tile = nt == TILE;

            if constexpr (kPackedMax) {
                stop_next = packed_max_tile(s, k, t, nt, full_tile, tx, ty);
                continue;
            }

            // ---- load (Section 4.1 step 1) ----
            Acc v[ITEMS];
            if (TMA && full_tile) {
                In xv[ITEMS];
                lds_blocked<In, ITEMS, SWI>(smem + L::off_in + s * TILE * sizeof(In),
                                            tid, lane, xv);
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) v[i] = K::load(xv[i]);
            } else {
                // partial tile: from the slot (bulk variants) or global
                const In *src = TMA ? reinterpret_cast<const In *>(
                                          smem + L::off_in + s * TILE * sizeof(In))
                                    : tx;
#pragma unroll
                for (int i = 0; i < ITEMS; ++i)
                    v[i] = (e0 + i < nt) ? K::load(src[e0 + i]) : K::ident();
            }
            // A tile whose only segment head is its first element takes the
            // unsegmented code: its carry is the identity (the carry warp
            // skips the look-back for it), which restarts the chain there.
            const bool inner = SEG && inner_s[s] != 0u;
            uint32_t hb = 0;  // head bits of my ITEMS elements
            if (inner) {
                const uint32_t w = bits[s * (TILE / 32) + (e0 >> 5)];
                hb = (w >> (e0 & 31)) & (ITEMS == 32 ? 0xffffffffu : ((1u << ITEMS) - 1u));
            }
            // (staged compaction values are read from the slot after the
            // block scan: the slot is released then)
            constexpr bool SV = is_staged_select<K>::value;
            __syncwarp();
            if (!SV && lane == 0) mbar_arrive(&empty[s]);  // slot may be refilled
            // stream compaction: start loading this thread's values now, so
            // they arrive while the tile is scanned and its carry awaited
            constexpr int SELN = (is_select<K>::value && !SV) ? ITEMS : 1;
            Out selv[SELN];
            if constexpr (is_select<K>::value && !SV) {
                const Out *xv = static_cast<const Out *>(p.values) +
                                t * static_cast<int64_t>(TILE) + e0;
                if (full_tile && (reinterpret_cast<uintptr_t>(p.values) & 15u) == 0u) {
                    constexpr int VC = ITEMS * int(sizeof(Out)) / 16;
                    uint4 q[VC];
#pragma unroll
                    for (int j = 0; j < VC; ++j) q[j] = reinterpret_cast<const uint4 *>(xv)[j];
                    unpack_chunks<Out, ITEMS, VC>(q, selv);
                } else {
#pragma unroll
                    for (int i = 0; i < ITEMS; ++i)
                        if (e0 + i < nt) selv[i] = xv[i];
                }
            }
            // the rest of the tile, compiled with and without segment heads
            auto finish_tile = [&](auto seg_tag) -> bool {
            constexpr bool SG = decltype(seg_tag)::value;
            // ---- thread-serial scan ----
#pragma unroll
            for (int i = 1; i < ITEMS; ++i) {
                if (SG && ((hb >> i) & 1u)) continue;
                v[i] = op_step<K>(v[i - 1], v[i]);
            }
            // ---- warp scan of thread totals (Hillis-Steele, 5 rounds) ----
            Acc wv = v[ITEMS - 1];
            uint32_t wf = SG ? (hb != 0u) : 0u;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const Acc ov = shfl_up_any(wv, d);
                const uint32_t of = SG ? __shfl_up_sync(0xffffffffu, wf, d) : 0u;
                if (lane >= d) {
                    if (!(SG && wf)) wv = K::op(ov, wv);
                    wf |= of;
                }
            }
            // exclusive lane prefix
            Acc lv = shfl_up_any(wv, 1);
            uint32_t lf = SG ? __shfl_up_sync(0xffffffffu, wf, 1) : 0u;
            if (lane == 0) {
                lv = K::ident();
                lf = 0u;
            }
            // ---- block scan of warp totals (Algorithm 3) ----
            // One barrier per tile: a warp can be at most one tile ahead of the
            // slowest (it cannot pass the next barrier before it), so two
            // buffers keep a fast warp from overwriting totals still being read.
            WarpTotal<Acc> *wt = wtot + (k & 1) * CW;
            if (lane == 31) {
                wt[warp].v = wv;
                wt[warp].f = wf;
            }
            named_bar_sync(1, CT);
            Acc bv = K::ident();
            uint32_t bf = 0u;
            if (lane < CW) {
                bv = wt[lane].v;
                bf = SG ? wt[lane].f : 0u;
            }
#pragma unroll
            for (int d = 1; d < CW; d <<= 1) {
                const Acc ov = shfl_up_any(bv, d);
                const uint32_t of = SG ? __shfl_up_sync(0xffffffffu, bf, d) : 0u;
                if (lane >= d) {
                    if (!(SG && bf)) bv = K::op(ov, bv);
                    bf |= of;
                }
            }
            Acc wev = shfl_idx_any(bv, warp > 0 ? warp - 1 : 0);
            uint32_t wef = SG ? __shfl_sync(0xffffffffu, bf, warp > 0 ? warp - 1 : 0) : 0u;
            if (warp == 0) {
                wev = K::ident();
                wef = 0u;
            }
            // thread base = warp offset (+) lane offset
            Acc tbv;
            if (SG && lf) {
                tbv = lv;
            } else {
                tbv = K::op(wev, lv);
            }
            const uint32_t tbf = SG ? (wef | lf) : 0u;

            if constexpr (SV) {
                // staged compaction: the in-tile index of each kept value is
                // known (thread base + v[i] - 1), so compact the tile into the
                // staging buffer now and free the slot before the carry wait
                // (the previous tile's copy out of the buffer ended before
                // this tile's vote, which every consumer thread passed)
                Out *stg = reinterpret_cast<Out *>(smem + L::off_out);
                Out vals[ITEMS];
                lds_blocked<Out, ITEMS>(smem + L::off_val + s * TILE * sizeof(Out), tid, lane,
                                        vals);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);  // slot may be refilled
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    const Acc kept = i == 0 ? v[0] : v[i] - v[i - 1];
                    if (e0 + i < nt && kept != 0u) stg[tbv + v[i] - 1u] = vals[i];
                }
            }

            // ---- carry from the carry warp (Section 4.3) ----
            const int cslot = static_cast<int>(k % CR);
            const bool okc = __all_sync(
                0xffffffffu,
                wait_phase(&carried[cslot], static_cast<uint32_t>((k / CR) & 1), wc));
            if (!okc && lane == 0) *abort_s = 1;
            const CarA cin = carry_s[cslot];
            const bool stop = !okc || stop_s[cslot] != 0u;

            if constexpr (is_select<K>::value) {
                // stream compaction: v[i] counts the kept elements of this
                // thread up to i; a kept element goes to carry + thread base
                // + v[i] - 1, each written once
                // compact the tile's kept values in shared memory (index in
                // the tile = thread base + v[i] - 1), then copy them to
                // y[carry ..) with coalesced stores
                const CarA Bs = K::base(cin, tbv);  // kept before this thread
                static_assert(L::kOut >= TILE * int(sizeof(Out)),
                              "compaction needs a whole tile of staging");
                Out *stg = reinterpret_cast<Out *>(smem + L::off_out);
                if constexpr (!SV) {
#pragma unroll
                    for (int i = 0; i < ITEMS; ++i) {
                        const Acc kept = i == 0 ? v[0] : v[i] - v[i - 1];
                        if (e0 + i < nt && kept != 0u) stg[tbv + v[i] - 1u] = selv[i];
                    }
                }
                const Acc tile_kept = shfl_idx_any(bv, CW - 1);  // block total
                named_bar_sync(3, CT);
                // The carry is where this tile's output starts.  A carry that
                // did not arrive (this warp's wait ran out: cin is stale) must
                // not address memory: write nothing then.  One that arrived is
                // at most the true count before the tile (a look-back that
                // gave up sums only what it saw), so the copy stays inside
                // y[0, n); the bound is checked all the same.
                const bool place = !stop && cin <= static_cast<CarA>(p.n) &&
                                   static_cast<CarA>(tile_kept) <= static_cast<CarA>(p.n) - cin;
                Out *yo = static_cast<Out *>(p.y) + (place ? cin : 0);
                if (place)
                    for (int j = tid; j < static_cast<int>(tile_kept); j += CT) yo[j] = stg[j];
                // (the next tile writes stg only after its block-scan barrier,
                // which every consumer thread reaches after this copy)
                // the owner of the array's last element writes the count
                // (elements past the end load as flag 0, so v[ITEMS - 1]
                // counts up to the last element)
                if (place && t == p.n_tiles - 1 && nt - 1 >= e0 && nt - 1 < e0 + ITEMS)
                    *p.count_out = static_cast<unsigned long long>(Bs + v[ITEMS - 1]);
                return stop;
            } else {
            // ---- apply carry and write y once (Section 4.4) ----
            const CarA B = K::base(cin, tbv);            // carry (+) thread base
            const CarA BL = K::base_local(tbv);          // head earlier in tile
            const CarA BI = K::base_local(K::ident());   // head earlier in thread
            constexpr bool kPackBf16Out =
                has_fin_f<K>::value && sizeof(Out) == 2 && ITEMS % 2 == 0;
            Out o[ITEMS];
            float of[kPackBf16Out ? ITEMS : 1];
            // element i's output from base b and in-thread prefix pv
            auto emit = [&](int i, const CarA &b, const Acc &pv) {
                if constexpr (kPackBf16Out) {
                    of[i] = K::fin_f(b, pv);
                } else {
                    o[i] = K::fin(b, pv);
                }
            };
            if constexpr (!SG) {
                // no heads: one base for the thread, and the inclusive /
                // exclusive choice made once rather than per element
                if (p.inclusive) {
#pragma unroll
                    for (int i = 0; i < ITEMS; ++i) emit(i, B, v[i]);
                } else {
                    emit(0, B, K::ident());
#pragma unroll
                    for (int i = 1; i < ITEMS; ++i) emit(i, B, v[i - 1]);
                }
            } else {
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                Acc pv;
                bool pf;  // a head at or before the contributing prefix, in thread
                if (p.inclusive) {
                    pv = v[i];
                    pf = SG && ((hb & ((2u << i) - 1u)) != 0u);
                } else if (SG && ((hb >> i) & 1u)) {
                    pv = K::ident();  // a segment head's exclusive value
                    pf = true;
                } else if (i == 0) {
                    pv = K::ident();
                    pf = false;
                } else {
                    pv = v[i - 1];
                    pf = SG && ((hb & ((1u << i) - 1u)) != 0u);
                }
                const CarA b = pf ? BI : ((SG && tbf) ? BL : B);
                emit(i, b, pv);
            }
            }
            if constexpr (kPackBf16Out) {
                // bf16 output: each pair rounded and packed by one conversion
#pragma unroll
                for (int i = 0; i < ITEMS; i += 2) {
                    const uint32_t w = f32x2_to_bf16x2_rn(of[i], of[i + 1]);
                    o[i] = static_cast<Out>(w & 0xffffu);
                    o[i + 1] = static_cast<Out>(w >> 16);
                }
            }
            if (TMA && full_tile && OS == 0) {
                // 16-byte stores straight from registers (no staging buffer)
                constexpr int OB = ITEMS * int(sizeof(Out));
                uint4 ov[OB / 16];
                pack_chunks<Out, ITEMS, OB / 16>(o, ov);
                uint4 *dst = reinterpret_cast<uint4 *>(ty + e0);
#pragma unroll
                for (int j = 0; j < OB / 16; ++j) dst[j] = ov[j];
            } else if (TMA && full_tile) {
                constexpr int WBYTES = 32 * ITEMS * int(sizeof(Out));
                uint8_t *region = smem + L::off_out +
                                  (OS == 2 ? (k & 1) : 0) * (TILE * sizeof(Out)) +
                                  warp * WBYTES;
                if (lane == 0) {
                    if constexpr (OS == 2) {
                        bulk_wait_read<1>();
                    } else {
                        bulk_wait_read<0>();
                    }
                }
                __syncwarp();
                sts_blocked<Out, ITEMS, SWO>(region, lane, lane, o);
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (SWO) {
                        // this warp's rows: 1024-byte blocks (t CW + warp) kOutWarpBlocks ..
                        tensor_s2g_3d(&p.tm_y, region, 0, 0,
                                      static_cast<int>((t * CW + warp) * kOutWarpBlocks));
                    } else {
                        bulk_s2g(ty + warp * 32 * ITEMS, region, WBYTES);
                    }
                    bulk_commit();
                }
            } else if (TMA && OS >= 1) {
                // partial tile: through this warp's staging region, then
                // coalesced stores of its valid elements
                constexpr int WE = 32 * ITEMS;  // elements per warp region
                Out *region = reinterpret_cast<Out *>(
                    smem + L::off_out + (OS == 2 ? (k & 1) : 0) * (TILE * sizeof(Out)) +
                    warp * WE * sizeof(Out));
                if (lane == 0) bulk_wait_read<0>();  // earlier bulk stores read it
                __syncwarp();
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) region[lane * ITEMS + i] = o[i];
                __syncwarp();
                const int wbase = warp * WE;
                const int valid = nt - wbase < WE ? nt - wbase : WE;
                for (int j = lane; j < valid; j += 32) ty[wbase + j] = region[j];
                __syncwarp();  // read before the next tile writes the region
            } else {
#pragma unroll
                for (int i = 0; i < ITEMS; ++i)
                    if (e0 + i < nt) ty[e0 + i] = o[i];
            }
            return stop;
            }
            };
            if constexpr (SEG) {
                stop_next = inner ? finish_tile(std::true_type{}) : finish_tile(std::false_type{});
            } else {
                stop_next = finish_tile(std::false_type{});
            }
        }
        if (lane == 0) bulk_wait_all<0>();
    }

    __syncthreads();
    // last CTA of this launch: re-arm the scratch for the next launch, and
    // hand the launch's error word to the host when asked
    if (tid == 0 && chain_launch_end(p.ctl, epoch) && p.err_host != nullptr) {
        volatile uint32_t *c = p.ctl;
        *reinterpret_cast<volatile uint32_t *>(p.err_host) = c[CTL_ERROR];
        c[CTL_ERROR] = 0u;
        __threadfence_system();
    }
}

}  // namespace lscan
