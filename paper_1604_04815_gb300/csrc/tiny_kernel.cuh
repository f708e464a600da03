// tiny_kernel.cuh -- single-CTA scan for arrays of at most one tile.
//
// An array of n <= kTinyMax elements has no inter-tile carry (Section 4.3
// never runs), so it needs none of the persistent kernel's machinery:
// ticket, tile ring, status words, scratch.  One CTA stages x through shared
// memory with coalesced loads, each thread scans its kTinyItems consecutive
// elements (Section 2.3 row scan), a warp shuffle scan (Algorithm 2) and a
// block scan of warp totals (Algorithm 3) give each thread its offset, the
// optional carry-in is applied (Section 4.4), and y goes back through shared
// memory for coalesced stores.  The kind traits are the same as the
// persistent kernel's, so the results follow the same rules.
#pragma once
#include <cstdint>

#include "kinds.cuh"
#include "scan_kernel.cuh"

namespace lscan {

template <class K>
__global__ void __launch_bounds__(kTinyThreads) lscan_tiny_kernel(const TinyParams p) {
    using In = typename K::In;
    using Out = typename K::Out;
    using Acc = typename K::Acc;
    using CarA = typename K::CarA;
    constexpr int W = kTinyThreads / 32;
    constexpr int EB = sizeof(In) > sizeof(Out) ? sizeof(In) : sizeof(Out);
    __shared__ __align__(16) uint8_t buf[kTinyMax * EB];
    __shared__ Acc wsum[W];

    // launched with programmatic stream serialization: wait for the
    // previous kernel of the stream before reading or writing global memory
    grid_dependency_wait();
    grid_launch_dependents();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = p.n;
    const In *x = static_cast<const In *>(p.x);
    Out *y = static_cast<Out *>(p.y);
    In *sx = reinterpret_cast<In *>(buf);
    Out *sy = reinterpret_cast<Out *>(buf);

    for (int i = tid; i < n; i += kTinyThreads) sx[i] = x[i];
    __syncthreads();
    const int e0 = tid * kTinyItems;
    Acc v[kTinyItems];
#pragma unroll
    for (int i = 0; i < kTinyItems; ++i)
        v[i] = (e0 + i < n) ? K::load(sx[e0 + i]) : K::ident();
    __syncthreads();  // sx is reused for the outputs below

    // thread-serial scan, then the thread totals across the warp
#pragma unroll
    for (int i = 1; i < kTinyItems; ++i) v[i] = op_step<K>(v[i - 1], v[i]);
    Acc wv = v[kTinyItems - 1];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const Acc ov = shfl_up_any(wv, d);
        if (lane >= d) wv = K::op(ov, wv);
    }
    Acc lv = shfl_up_any(wv, 1);
    if (lane == 0) lv = K::ident();
    if (lane == 31) wsum[warp] = wv;
    __syncthreads();
    // warp offsets: every warp scans the W totals itself
    Acc bv = lane < W ? wsum[lane] : K::ident();
#pragma unroll
    for (int d = 1; d < W; d <<= 1) {
        const Acc ov = shfl_up_any(bv, d);
        if (lane >= d) bv = K::op(ov, bv);
    }
    Acc wev = shfl_idx_any(bv, warp > 0 ? warp - 1 : 0);
    if (warp == 0) wev = K::ident();
    const Acc tbv = K::op(wev, lv);

    typename K::Car cin = K::cident();
    if (p.carry_in != nullptr)
        cin = p.carry_in_car ? *static_cast<const typename K::Car *>(p.carry_in)
                             : K::car_of_out(*static_cast<const Out *>(p.carry_in));
    const CarA B = K::base(K::to_apply(cin), tbv);
    // the last thread's inclusive value covers the whole array (identities
    // pad it past n): the total handed to the next chunk of a chunked scan
    if (p.total_out != nullptr && tid == kTinyThreads - 1)
        *static_cast<typename K::Car *>(p.total_out) =
            K::cop(cin, K::to_car(K::op(tbv, v[kTinyItems - 1])));
#pragma unroll
    for (int i = 0; i < kTinyItems; ++i) {
        if (e0 + i >= n) break;
        const Acc pv = p.inclusive ? v[i] : (i == 0 ? K::ident() : v[i - 1]);
        sy[e0 + i] = K::fin(B, pv);
    }
    __syncthreads();
    for (int i = tid; i < n; i += kTinyThreads) y[i] = sy[i];
}

}  // namespace lscan
