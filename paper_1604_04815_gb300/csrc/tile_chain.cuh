// tile_chain.cuh -- CTA-to-CTA messaging of a single-pass kernel: the
// inter-block carry chain of LightScan Section 4.3 (Algorithm 4) as a
// reusable primitive, used by the scan kernel (and its stream-compaction
// kinds) and by the reduction of sharded scans.
//
// A launch numbers its blocks of work ("tiles") 0, 1, 2, ... in the order
// they are handed out.  Each tile owns a status slot of SLOT 64-bit words in
// global memory (L2).  A word holds 32 bits of payload and a 32-bit tag:
// (launch epoch mod 2^30) << 2 | state, state = aggregate (the tile's own
// total) or inclusive (everything up to and including the tile).  A payload
// wider than 32 bits spans several words, each with the full tag, so a read
// that sees different tags (a torn read) counts as not yet published.
// Because every word carries the launch's epoch, consecutive launches (and
// CUDA-graph replays) need no clearing of the slots: the last CTA of a
// launch advances the epoch (chain_launch_end).
//
//   StatusIO<K, SLOT>::publish / read   one tile's slot (relaxed, gpu scope)
//   lookback<K, SLOT>                  decoupled look-back by one warp: the
//                                      exclusive prefix of tile t
//   chained_wait<K, SLOT>              the paper's neighbour hand-off: wait
//                                      for tile t-1's inclusive prefix
//   wait_phase                         bounded mbarrier wait (tile rings)
//   chain_launch_end                   the last CTA re-arms ticket and epoch
//
// K is a carry operator: Car (the payload type), cident() its identity,
// cop(earlier, later) the associative combine, and kTieOrdered / gt() for
// maxima whose equal values can differ in bits (+0 / -0), which keep the
// earliest tile on ties.  Every wait is bounded by a %globaltimer limit; a
// wait that runs out sets the launch's error word (DEV_ERR_CARRY_WAIT or
// DEV_ERR_BARRIER_WAIT) and every later wait of the same launch gives up at
// once, so a launch never hangs and the host reads the error afterwards.
#pragma once
#include <cstdint>
#include <cstring>

#include "ptx.cuh"
#include "scan_common.h"

namespace lscan {

// --------------------------------------------------- 32-bit word shuffles
template <class T>
__device__ __forceinline__ T shfl_up_any(T v, int d) {
    static_assert(sizeof(T) % 4 == 0, "word-sized types only");
    constexpr int W = sizeof(T) / 4;
    uint32_t w[W];
    memcpy(w, &v, sizeof(T));
#pragma unroll
    for (int i = 0; i < W; ++i) w[i] = __shfl_up_sync(0xffffffffu, w[i], d);
    T r;
    memcpy(&r, w, sizeof(T));
    return r;
}
template <class T>
__device__ __forceinline__ T shfl_down_any(T v, int d) {
    constexpr int W = sizeof(T) / 4;
    uint32_t w[W];
    memcpy(w, &v, sizeof(T));
#pragma unroll
    for (int i = 0; i < W; ++i) w[i] = __shfl_down_sync(0xffffffffu, w[i], d);
    T r;
    memcpy(&r, w, sizeof(T));
    return r;
}
template <class T>
__device__ __forceinline__ T shfl_idx_any(T v, int src) {
    constexpr int W = sizeof(T) / 4;
    uint32_t w[W];
    memcpy(w, &v, sizeof(T));
#pragma unroll
    for (int i = 0; i < W; ++i) w[i] = __shfl_sync(0xffffffffu, w[i], src);
    T r;
    memcpy(&r, w, sizeof(T));
    return r;
}

// ------------------------------------------------------------ status words
// Words per tile slot.  Every carry warp polls, and the reducers and carry
// warps publish to, the same few status lines near the frontier; the L2
// slices holding them then slow the streaming traffic that maps there, so
// fewer tiles per 128-byte line pay.  Measured on GB300 at 2^28: a 32-bit
// carry (int32 add, 16 KiB tiles) with 1/2/4/8 words per tile
// 5256/5667/5668/5545 GB/s; a two-word FP64 carry with 32 KiB tiles (fp32
// add, config 3) 2 words 5336, 4 words 5487, 8 words 5457 (means of 3),
// but with 16 KiB tiles 4 words lost (bf16 add, config 2: 4892 -> 4684).
template <class K, class Cfg>
__host__ __device__ constexpr int status_slot_words() {
    constexpr int W = int(sizeof(typename K::Car) / 4);
    constexpr int TILE_BYTES = Cfg::TILE * int(sizeof(typename K::In));
    if constexpr (Cfg::SLOTW > 0) {
        static_assert(Cfg::SLOTW >= W, "a slot holds the carry's words");
        return Cfg::SLOTW;
    }
    return W == 1 ? 2 : (TILE_BYTES >= 32768 ? 2 * W : W);
}

template <class K, int SLOT>
struct StatusIO {
    using Car = typename K::Car;
    static constexpr int W = int(sizeof(Car) / 4);
    static_assert(SLOT >= W, "a slot holds the carry's words");

    __device__ static void publish(uint64_t *status, int64_t t, uint32_t tag,
                                   Car c) {
        uint32_t w[W];
        memcpy(w, &c, sizeof(Car));
#pragma unroll
        for (int i = 0; i < W; ++i)
            st_relaxed_gpu(status + t * SLOT + i,
                           (static_cast<uint64_t>(w[i]) << 32) | tag);
    }
    // State of tile t for this launch (ST_INVALID if absent or torn).
    __device__ static uint32_t read(const uint64_t *status, int64_t t,
                                    uint32_t ebase, Car &c) {
        uint32_t w[W];
        const uint64_t r0 = ld_relaxed_gpu(status + t * SLOT);
        const uint32_t tag0 = static_cast<uint32_t>(r0);
        w[0] = static_cast<uint32_t>(r0 >> 32);
        bool same = true;
#pragma unroll
        for (int i = 1; i < W; ++i) {
            const uint64_t r = ld_relaxed_gpu(status + t * SLOT + i);
            same = same && (static_cast<uint32_t>(r) == tag0);
            w[i] = static_cast<uint32_t>(r >> 32);
        }
        if (!same || (tag0 & ~3u) != ebase) return ST_INVALID;
        const uint32_t st = tag0 & 3u;
        if (st != ST_AGGREGATE && st != ST_INCLUSIVE) return ST_INVALID;
        memcpy(&c, w, sizeof(Car));
        return st;
    }
};

// Records that a wait of this launch gave up; later waits of the same launch
// then give up at once, so a launch never takes much more than one limit.
__device__ __forceinline__ void note_gave_up(const WaitCtx &w, uint32_t bit) {
    atomicOr(w.ctl + CTL_ERROR, bit);
    atomicExch(w.ctl + CTL_ERR_EPOCH, w.epoch + 1u);
}
__device__ __forceinline__ bool launch_gave_up(const WaitCtx &w) {
    return *reinterpret_cast<volatile uint32_t *>(w.ctl + CTL_ERR_EPOCH) ==
           w.epoch + 1u;
}
// A wait reads the launch-wide give-up word only once it has lasted this
// long: normal waits end well before, so waiting warps do not all poll one
// global word, and a launch that gave up elsewhere still ends quickly.
constexpr uint64_t kGiveUpCheckNs = 20000;
__device__ __forceinline__ bool wait_over(const WaitCtx &w, uint64_t waited_ns) {
    return waited_ns > kGiveUpCheckNs && (waited_ns > w.limit_ns || launch_gave_up(w));
}

// Bounded wait on an mbarrier phase; false (and a device error bit) if the
// limit ran out.
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity,
                                           const WaitCtx &w) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (wait_over(w, global_timer_ns() - t0)) {
            note_gave_up(w, DEV_ERR_BARRIER_WAIT);
            return false;
        }
    }
    return true;
}

// Decoupled look-back, run by one full warp: exclusive prefix of tile t.
//
// A round loads the status words of kLookbackWindows 32-tile windows (lane l
// of window j reads tile base - 32 j - l).  From the ballots alone it finds
// how far it may go: every window up to the first one that holds an
// inclusive prefix (cut after that lane) or a not-yet-published tile.  Each
// lane folds its own tiles of those windows, then one butterfly combines the
// lanes (depth kLookbackWindows + 5).  The operators are commutative; float
// max keeps the first occurrence by comparing tile indices on ties.
// Measured on GB300 with aggregates published at data arrival: one window
// per round is fastest (int32, 2^28: 5462 GB/s with 1 window, 5290 with 2,
// 4900 with 4, 4024 with 8); the status words near the frontier are read by
// every carry warp, and more words per round cost more than the rounds they
// save.  A two-level variant (cached 32-tile group statuses) measured slower
// still (3455 GB/s): the groups near the frontier are always fresh.
constexpr int kLookbackWindows = 1;

template <class K>
struct CarryFold {
    using Car = typename K::Car;
    Car v;
    int64_t i;  // earliest tile holding v (tie order of float max)
    __device__ void init() {
        v = K::cident();
        i = INT64_MAX;
    }
    __device__ void add(Car x, int64_t idx) {
        if constexpr (K::kTieOrdered) {
            if (K::gt(x, v) || (!K::gt(v, x) && idx < i)) {
                v = x;
                i = idx;
            }
        } else {
            v = K::cop(v, x);
        }
    }
};

template <class K, int SLOT>
__device__ typename K::Car lookback(const uint64_t *status, const WaitCtx &wc,
                                    int64_t t, uint32_t ebase, int lane) {
    using Car = typename K::Car;
    constexpr int P = kLookbackWindows;
    CarryFold<K> excl;
    excl.init();
    int64_t base = t - 1;  // tile seen by lane 0 of window 0
    uint64_t t0 = 0;
    bool started = false, gave_up = false;
    while (true) {
        uint32_t st[P];
        Car val[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int64_t idx = base - 32 * j - lane;
            st[j] = ST_INCLUSIVE;  // before tile 0: identity, inclusive
            val[j] = K::cident();
            if (idx >= 0) st[j] = StatusIO<K, SLOT>::read(status, idx, ebase, val[j]);
            if (gave_up && st[j] == ST_INVALID) {
                st[j] = ST_INCLUSIVE;
                val[j] = K::cident();
            }
        }
        // how far this round may go (warp-uniform, from ballots only)
        int use = 0;             // windows fully or partly consumed
        uint32_t last_mask = 0;  // lanes consumed in window use - 1
        bool found = false;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const uint32_t inc = __ballot_sync(0xffffffffu, st[j] == ST_INCLUSIVE);
            const uint32_t bad = __ballot_sync(0xffffffffu, st[j] == ST_INVALID);
            if (found || use != j) continue;
            const uint32_t need = inc ? (((inc & (0u - inc)) << 1) - 1u) : 0xffffffffu;
            if (bad & need) continue;  // window j not ready: stop before it
            use = j + 1;
            last_mask = need;
            found = inc != 0u;
        }
        if (use == 1 && last_mask == 1u) {
            // only the nearest tile is needed and it holds an inclusive
            // prefix (the common case): no butterfly
            const Car v0 = shfl_idx_any(val[0], 0);
            if constexpr (K::kTieOrdered) {
                excl.add(v0, base);
            } else {
                excl.v = K::cop(v0, excl.v);
            }
            break;
        }
        if (use > 0) {
            CarryFold<K> part;
            part.init();
#pragma unroll
            for (int j = P - 1; j >= 0; --j) {  // earliest tiles first
                if (j >= use) continue;
                const bool in = (j < use - 1) || ((last_mask >> lane) & 1u);
                if (in) part.add(val[j], base - 32 * j - lane);
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                const Car ov = shfl_idx_any(part.v, lane ^ off);
                const int64_t oi = __shfl_xor_sync(0xffffffffu, part.i, off);
                part.add(ov, oi);
            }
            // part covers tiles earlier than everything folded into excl so far
            if constexpr (K::kTieOrdered) {
                excl.add(part.v, part.i);
            } else {
                excl.v = K::cop(part.v, excl.v);
            }
            if (found) break;
            base -= 32 * use;
            continue;  // progress: next round at once
        }
        if (!started) {
            t0 = global_timer_ns();
            started = true;
        } else {
            bool over = wait_over(wc, global_timer_ns() - t0);
            over = __shfl_sync(0xffffffffu, over, 0);
            if (over && !gave_up) {
                gave_up = true;
                if (lane == 0) note_gave_up(wc, DEV_ERR_CARRY_WAIT);
            }
        }
    }
    return excl.v;
}

// Chained hand-off (Algorithm 4): wait for tile t-1's inclusive prefix.
template <class K, int SLOT>
__device__ typename K::Car chained_wait(const uint64_t *status, const WaitCtx &wc,
                                        int64_t t, uint32_t ebase, int lane) {
    using Car = typename K::Car;
    Car v = K::cident();
    if (lane == 0) {
        uint32_t st = StatusIO<K, SLOT>::read(status, t - 1, ebase, v);
        if (st != ST_INCLUSIVE) {
            const uint64_t t0 = global_timer_ns();
            while (true) {
                st = StatusIO<K, SLOT>::read(status, t - 1, ebase, v);
                if (st == ST_INCLUSIVE) break;
                if (wait_over(wc, global_timer_ns() - t0)) {
                    note_gave_up(wc, DEV_ERR_CARRY_WAIT);
                    v = K::cident();
                    break;
                }
            }
        }
    }
    return shfl_idx_any(v, 0);
}

// Ends a launch of a chained kernel: the CTA that finishes last (a done
// counter; nobody waits) resets the tile ticket and the done counter and
// advances the epoch that tags status words, so the next launch on the same
// control block starts clean.  Called by one thread per CTA after all of the
// CTA's work; returns true in the last CTA.
__device__ __forceinline__ bool chain_launch_end(uint32_t *ctl, uint32_t epoch) {
    __threadfence();
    const uint32_t prev = atomicAdd(ctl + CTL_DONE, 1u);
    if (prev != gridDim.x - 1) return false;
    volatile uint32_t *c = ctl;
    c[CTL_TICKET] = 0u;
    c[CTL_DONE] = 0u;
    c[CTL_EPOCH] = epoch + 1u;
    __threadfence();
    return true;
}

}  // namespace lscan
