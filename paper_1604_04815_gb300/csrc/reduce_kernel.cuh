// reduce_kernel.cuh -- the total x_0 (+) ... (+) x_{n-1} of an array in the
// kind's carry type: the reduce pass of a scan sharded over devices.
//
// A scan split into contiguous shards needs, for shard g, the total of the
// shards before it (the inter-block carry of Section 4.3 lifted one level
// up: there one tile's prefix, here one device's).  In the reduce-then-scan
// form each shard is read once to get its total (this kernel), the totals
// are exchanged, and each shard is scanned once with the fold of the earlier
// totals as its carry-in: 3N bytes moved instead of the 4N of
// scan-then-add.
//
// Blocks: CTA c reduces a contiguous range of the array (whole 16-byte
// chunks when x is 16-byte aligned; the ragged tail goes to the last CTA),
// so CTA order is element order.  Within a CTA each thread folds the chunks
// c0 + tid, c0 + tid + 256, ... (each chunk in the scan's in-tile
// arithmetic, the kinds with an exact two-sum step included, and the chunk
// totals in the carry type, so the total is as accurate as the carry chain
// of a single-array scan), and the threads' partials are combined with
// element indices deciding ties of float max (+0 / -0: the first occurrence
// wins).  The CTAs' partials then travel through the inter-block carry
// chain (tile_chain.cuh): every CTA publishes its partial as its tile's
// aggregate (CTA 0 as inclusive), and the CTA that owns the last range looks
// back for the fold of all earlier ones -- the same bounded, epoch-tagged
// protocol as the scan, so a wait that runs out is reported on the stream
// instead of hanging, and no clearing is needed between launches.
#pragma once
#include <cstdint>

#include "kinds.cuh"
#include "scan_common.h"
#include "scan_kernel.cuh"
#include "tile_chain.cuh"

namespace lscan {

constexpr int kReduceThreads = 256;
constexpr int kReduceUnroll = 4;  // 16-byte loads in flight per thread

struct ReduceParams {
    const void *x;
    int64_t n;
    int64_t units_per_cta;  // 16-byte chunks (aligned x) or elements per CTA
    int32_t aligned;        // x starts on a 16-byte boundary
    int32_t reserved;
    uint32_t *ctl;          // control block (epoch, error, ticket, done)
    uint64_t *status;       // a status slot per CTA
    uint64_t wait_limit_ns;
    int64_t skip_tile;      // fault injection: this CTA never publishes (-1 off)
    void *total_out;        // Car
};

// Status words per CTA: the carry's words, at least 2 (16-byte slots).
template <class K>
constexpr int reduce_slot_words() {
    return int(sizeof(typename K::Car)) / 4 > 2 ? int(sizeof(typename K::Car)) / 4 : 2;
}

// Running total in the carry type; for tie-ordered max the index of the
// element it came from, so that equal values keep the earliest one whatever
// the order of combination within the CTA.
template <class K>
struct RFold {
    using Car = typename K::Car;
    Car v;
    int64_t i;
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

// Fold of EPC consecutive elements starting at index base: value in the
// carry type and (tie-ordered kinds) the index of its first occurrence.
template <class K, int EPC>
__device__ __forceinline__ void fold_chunk(const typename K::In (&e)[EPC], int64_t base,
                                           RFold<K> &f) {
    using Acc = typename K::Acc;
    Acc a = K::load(e[0]);
    int first = 0;
#pragma unroll
    for (int u = 1; u < EPC; ++u) {
        const Acc b = K::load(e[u]);
        if constexpr (K::kTieOrdered) {
            if (K::gt(b, a)) {
                a = b;
                first = u;
            }
        } else {
            a = op_step<K>(a, b);
        }
    }
    f.add(K::to_car(a), base + first);
}

template <class K>
__global__ void __launch_bounds__(kReduceThreads) lscan_reduce_kernel(const ReduceParams p) {
    using In = typename K::In;
    using Car = typename K::Car;
    constexpr int EPC = 16 / int(sizeof(In));
    constexpr int SLOT = reduce_slot_words<K>();
    const In *x = static_cast<const In *>(p.x);
    const int64_t n = p.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t epoch = *reinterpret_cast<volatile uint32_t *>(p.ctl + CTL_EPOCH);
    const uint32_t ebase = (epoch & kEpochMask) << 2;
    const WaitCtx wc{p.ctl, p.wait_limit_ns, epoch};
    const int64_t c = blockIdx.x;
    const bool last_cta = c == gridDim.x - 1;

    RFold<K> f;
    f.init();
    if (p.aligned) {
        // this CTA's 16-byte chunks, kReduceUnroll loads in flight per thread
        const int64_t nchunks = n / EPC;
        const int64_t u0 = c * p.units_per_cta;
        const int64_t u1 = last_cta ? nchunks : min(nchunks, u0 + p.units_per_cta);
        const uint4 *xv = reinterpret_cast<const uint4 *>(x);
        for (int64_t k0 = u0 + tid; k0 < u1; k0 += kReduceThreads * kReduceUnroll) {
            uint4 q[kReduceUnroll];
#pragma unroll
            for (int u = 0; u < kReduceUnroll; ++u) {
                const int64_t k = k0 + u * kReduceThreads;
                if (k < u1) q[u] = __ldcs(xv + k);
            }
#pragma unroll
            for (int u = 0; u < kReduceUnroll; ++u) {
                const int64_t k = k0 + u * kReduceThreads;
                if (k < u1) {
                    const uint4 qa[1] = {q[u]};
                    In e[EPC];
                    unpack_chunks<In, EPC, 1>(qa, e);
                    fold_chunk<K, EPC>(e, k * EPC, f);
                }
            }
        }
        // the ragged tail belongs to the last range
        if (last_cta)
            for (int64_t i = nchunks * EPC + tid; i < n; i += kReduceThreads) {
                const In e[1] = {x[i]};
                fold_chunk<K, 1>(e, i, f);
            }
    } else {
        const int64_t i0 = c * p.units_per_cta;
        const int64_t i1 = last_cta ? n : min(n, i0 + p.units_per_cta);
        for (int64_t i = i0 + tid; i < i1; i += kReduceThreads) {
            const In e[1] = {x[i]};
            fold_chunk<K, 1>(e, i, f);
        }
    }

    // CTA partial: shuffle tree in each warp, then warp 0 over the warp totals
    __shared__ Car wv[kReduceThreads / 32];
    __shared__ int64_t wi[kReduceThreads / 32];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const Car ov = shfl_down_any(f.v, off);
        const int64_t oi = __shfl_down_sync(0xffffffffu, f.i, off);
        if (lane + off < 32) f.add(ov, oi);
    }
    if (lane == 0) {
        wv[warp] = f.v;
        wi[warp] = f.i;
    }
    __syncthreads();
    if (warp == 0) {
        RFold<K> b;
        b.init();
        if (lane == 0)
            for (int w = 0; w < kReduceThreads / 32; ++w) b.add(wv[w], wi[w]);
        const Car part = shfl_idx_any(b.v, 0);
        // publish this range's partial (range 0: the inclusive prefix)
        if (lane == 0 && c != p.skip_tile)
            StatusIO<K, SLOT>::publish(p.status, c,
                                       ebase | (c == 0 ? ST_INCLUSIVE : ST_AGGREGATE), part);
        if (last_cta) {
            // the fold of every earlier range, then this one (earlier first)
            Car total = part;
            if (c > 0) total = K::cop(lookback<K, SLOT>(p.status, wc, c, ebase, lane), part);
            if (lane == 0) *static_cast<Car *>(p.total_out) = total;
        }
    }
    __syncthreads();
    if (tid == 0) (void)chain_launch_end(p.ctl, epoch);
}

}  // namespace lscan
