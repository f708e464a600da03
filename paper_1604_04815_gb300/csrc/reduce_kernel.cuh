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
// Precision follows the kind: each 16-byte chunk is folded in the in-tile
// type Acc (the compensated kinds with their exact two-sum step), and the
// chunk totals are accumulated in the carry type Car (FP64 or double-float
// for the float adds that carry that way), so a shard total is as accurate
// as the carry chain of a single-array scan.  Max kinds whose equal values
// may differ in bits (float max: +0 / -0) keep the first occurrence by
// tracking element indices, so the grouping of the reduction does not
// matter.  The CTA partials are folded in CTA order by the CTA that
// finishes last (a done counter; no CTA waits), which writes the total and
// re-arms the counter.
#pragma once
#include <cstdint>

#include "kinds.cuh"
#include "scan_kernel.cuh"

namespace lscan {

constexpr int kReduceThreads = 256;
constexpr int kReduceUnroll = 4;  // 16-byte loads in flight per thread

struct ReduceParams {
    const void *x;
    int64_t n;
    int32_t aligned;     // x starts on a 16-byte boundary
    int32_t reserved;
    void *partials;      // Car[gridDim.x]
    int64_t *part_idx;   // [gridDim.x]: element index of a max partial
    uint32_t *done;      // CTAs finished: zero on entry and on exit
    void *total_out;     // Car
};

// Load of a word-sized value through L2 only (another CTA wrote it).
template <class T>
__device__ __forceinline__ T ld_cg(const T *p) {
    static_assert(sizeof(T) % 4 == 0, "word-sized types only");
    constexpr int W = sizeof(T) / 4;
    uint32_t w[W];
    const unsigned int *q = reinterpret_cast<const unsigned int *>(p);
#pragma unroll
    for (int i = 0; i < W; ++i) w[i] = __ldcg(q + i);
    T r;
    memcpy(&r, w, sizeof(T));
    return r;
}

// Running total in the carry type; for tie-ordered max the index of the
// element it came from, so that equal values keep the earliest one whatever
// the order of combination.
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
    const In *x = static_cast<const In *>(p.x);
    const int64_t n = p.n;
    const int64_t nchunks = p.aligned ? n / EPC : 0;
    const int64_t gtid = static_cast<int64_t>(blockIdx.x) * kReduceThreads + threadIdx.x;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kReduceThreads;

    RFold<K> f;
    f.init();
    // whole 16-byte chunks, kReduceUnroll loads in flight per thread; each
    // thread visits its chunks in increasing order
    const uint4 *xv = reinterpret_cast<const uint4 *>(x);
    for (int64_t c0 = gtid; c0 < nchunks; c0 += stride * kReduceUnroll) {
        uint4 q[kReduceUnroll];
#pragma unroll
        for (int u = 0; u < kReduceUnroll; ++u) {
            const int64_t c = c0 + u * stride;
            if (c < nchunks) q[u] = __ldcs(xv + c);
        }
#pragma unroll
        for (int u = 0; u < kReduceUnroll; ++u) {
            const int64_t c = c0 + u * stride;
            if (c < nchunks) {
                const uint4 qa[1] = {q[u]};
                In e[EPC];
                unpack_chunks<In, EPC, 1>(qa, e);
                fold_chunk<K, EPC>(e, c * EPC, f);
            }
        }
    }
    // the rest (everything when x is not 16-byte aligned), one element each
    for (int64_t i = nchunks * EPC + gtid; i < n; i += stride) {
        const In e[1] = {x[i]};
        fold_chunk<K, 1>(e, i, f);
    }

    // CTA total: shuffle tree in each warp, then warp 0 over the warp totals
    __shared__ Car wv[kReduceThreads / 32];
    __shared__ int64_t wi[kReduceThreads / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    if (threadIdx.x == 0) {
        RFold<K> b;
        b.init();
        for (int w = 0; w < kReduceThreads / 32; ++w) b.add(wv[w], wi[w]);
        static_cast<Car *>(p.partials)[blockIdx.x] = b.v;
        p.part_idx[blockIdx.x] = b.i;
        __threadfence();
        const uint32_t prev = atomicAdd(p.done, 1u);
        last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        // every other CTA's partial is visible (each fenced before counting);
        // read them from L2 (ld.cg), past this SM's L1
        __threadfence();
        RFold<K> t;
        t.init();
        for (unsigned c = 0; c < gridDim.x; ++c)
            t.add(ld_cg<Car>(static_cast<const Car *>(p.partials) + c),
                  ld_cg<int64_t>(p.part_idx + c));
        *static_cast<Car *>(p.total_out) = t.v;
        *p.done = 0u;
    }
}

}  // namespace lscan
