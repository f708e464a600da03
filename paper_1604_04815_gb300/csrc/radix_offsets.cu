// radix_offsets.cu -- radix-sort digit offsets in one pass over the keys.
//
// Not in the paper, which lists parallel sorting among the applications of
// scan (Section 1); radix sort is the sort built on it.  A radix-sort pass
// on digit p moves each key to the start of its bucket plus its rank among
// the keys with the same digit before it; the bucket starts are the
// exclusive scan of the digit-p histogram.  This kernel produces them for
// every digit position at once, reading the keys once:
//  * Histograms.  A persistent grid streams the keys with 16-byte loads
//    (grid-stride, four vectors in flight per thread) and counts every digit
//    of every key into its warp's copy of the P x B counters in shared
//    memory (shared-memory atomics; one copy per warp, or per pair of warps
//    for 64-bit keys with 8-bit digits, so warps do not contend).
//  * Merge.  Each CTA sums its copies and adds the non-zero counters to a
//    per-stream global array with 64-bit atomics.
//  * Scan.  The CTA that finishes last (a done counter; no CTA ever waits)
//    scans each position's B counters, one warp per position: each lane
//    takes ceil(B / 32) consecutive buckets and scans them serially (the row
//    scan of Section 2.3), and a 5-round shuffle scan of the lane totals
//    (Section 2.1, Algorithm 2) gives each lane its offset.  It writes the
//    offsets and zeroes the global counters and the done counter, so the
//    next launch on the stream starts clean.
// HBM traffic: the keys once (4 or 8 B per key) plus 8 B per counter.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "../../include/lscan.h"
#include "lscan_internal.h"

namespace lscan {
namespace {

constexpr int kRadixThreads = 512;
constexpr int kRadixWarps = kRadixThreads / 32;
// P x B <= 8 x 256: 64-bit keys with 8-bit digits is the largest case
constexpr int kRadixMaxCounters = 2048;
constexpr int kRadixSmemBudget = 64 * 1024;  // histogram copies per CTA
constexpr int kRadixUnroll = 4;              // 16-byte loads in flight per thread

struct RadixParams {
    const void *keys;
    int64_t n;
    unsigned long long *counts;  // [P * B]: zero on entry, zeroed on exit
    unsigned int *done;          // CTAs finished: zero on entry and exit
    int64_t *offsets;            // [P * B] output
    int32_t digit_bits;
    int32_t positions;           // P
    int32_t copies;              // histogram copies in shared memory
    int32_t aligned;             // keys start on a 16-byte boundary
};

template <class Key>
__device__ __forceinline__ void count_key(uint32_t *h, Key k, int P, int b, int B,
                                          Key mask) {
    for (int q = 0; q < P; ++q)
        atomicAdd(h + q * B + static_cast<int>((k >> (q * b)) & mask), 1u);
}

template <class Key>
__global__ void __launch_bounds__(kRadixThreads) radix_offsets_kernel(const RadixParams p) {
    extern __shared__ uint32_t hist[];  // copies x P x B
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = p.digit_bits, P = p.positions, B = 1 << b;
    const int NB = P * B;
    const Key mask = static_cast<Key>(B - 1);
    for (int i = tid; i < p.copies * NB; i += kRadixThreads) hist[i] = 0u;
    __syncthreads();

    // ---- histograms of every digit position ----
    uint32_t *h = hist + (warp % p.copies) * NB;
    const Key *keys = static_cast<const Key *>(p.keys);
    const int64_t gtid = static_cast<int64_t>(blockIdx.x) * kRadixThreads + tid;
    const int64_t gstride = static_cast<int64_t>(gridDim.x) * kRadixThreads;
    int64_t rest = 0;  // first key left for the scalar loop
    if (p.aligned) {
        constexpr int EPV = 16 / int(sizeof(Key));
        const int64_t nv = p.n / EPV;
        const uint4 *kv = reinterpret_cast<const uint4 *>(keys);
        for (int64_t i = gtid; i < nv; i += kRadixUnroll * gstride) {
            uint4 q[kRadixUnroll];
#pragma unroll
            for (int u = 0; u < kRadixUnroll; ++u)
                if (i + u * gstride < nv) q[u] = __ldcs(kv + i + u * gstride);
#pragma unroll
            for (int u = 0; u < kRadixUnroll; ++u) {
                if (i + u * gstride >= nv) break;
                Key e[EPV];
                memcpy(e, &q[u], 16);
#pragma unroll
                for (int x = 0; x < EPV; ++x) count_key<Key>(h, e[x], P, b, B, mask);
            }
        }
        rest = nv * EPV;
    }
    for (int64_t j = rest + gtid; j < p.n; j += gstride) count_key<Key>(h, keys[j], P, b, B, mask);
    __syncthreads();

    // ---- merge this CTA's copies into the global counters ----
    for (int i = tid; i < NB; i += kRadixThreads) {
        uint32_t s = 0;
        for (int c = 0; c < p.copies; ++c) s += hist[c * NB + i];
        if (s != 0u) atomicAdd(p.counts + i, static_cast<unsigned long long>(s));
    }
    __threadfence();  // this thread's counter updates before the done count
    __syncthreads();
    __shared__ uint32_t is_last;
    if (tid == 0) is_last = atomicAdd(p.done, 1u) == gridDim.x - 1 ? 1u : 0u;
    __syncthreads();
    if (is_last == 0u) return;
    __threadfence();

    // ---- last CTA: exclusive scan of each position's buckets ----
    const int per_lane = (B + 31) / 32;  // 1 .. 8 consecutive buckets per lane
    for (int q = warp; q < P; q += kRadixWarps) {
        unsigned long long c[8];
        unsigned long long tot = 0ull;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int v = lane * per_lane + j;
            c[j] = (j < per_lane && v < B) ? __ldcg(p.counts + q * B + v) : 0ull;
            tot += c[j];
        }
        unsigned long long inc = tot;  // inclusive scan of the lane totals
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += o;
        }
        unsigned long long run = inc - tot;  // buckets of the lanes before
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int v = lane * per_lane + j;
            if (j < per_lane && v < B) {
                p.offsets[q * B + v] = static_cast<int64_t>(run);
                p.counts[q * B + v] = 0ull;
            }
            run += c[j];
        }
    }
    __syncthreads();
    if (tid == 0) *p.done = 0u;
}

struct RadixScratch {
    unsigned long long *counts = nullptr;  // kRadixMaxCounters
    unsigned int *done = nullptr;
};

std::mutex g_radix_mu;
std::map<std::pair<int, void *>, RadixScratch> g_radix_scratch;
std::map<std::pair<int, const void *>, bool> g_radix_attr;  // smem limit set
std::map<std::pair<std::pair<int, const void *>, int>, int> g_radix_bps;  // CTAs/SM

bool ranges_overlap(const void *a, size_t an, const void *b, size_t bn) {
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
    return a0 < b0 + bn && b0 < a0 + an;
}

}  // namespace

void shutdown_radix() {
    std::lock_guard<std::mutex> lk(g_radix_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_radix_scratch) {
        cudaSetDevice(kv.first.first);
        cudaDeviceSynchronize();
        if (kv.second.counts) cudaFree(kv.second.counts);
    }
    g_radix_scratch.clear();
    g_radix_attr.clear();
    g_radix_bps.clear();
    cudaSetDevice(cur);
}

}  // namespace lscan

using namespace lscan;

extern "C" lscan_status lscan_radix_offsets(const void *keys, int32_t key_bytes, int64_t n,
                                            int32_t digit_bits, int64_t *d_offsets,
                                            void *stream) {
    if ((key_bytes != 4 && key_bytes != 8) || digit_bits < 1 || digit_bits > 8 || n < 0 ||
        n > int64_t{0xffffffff})
        return LSCAN_ERR_INVALID;
    if (d_offsets == nullptr || reinterpret_cast<uintptr_t>(d_offsets) % 8 != 0)
        return LSCAN_ERR_INVALID;
    const int P = (8 * key_bytes + digit_bits - 1) / digit_bits;
    const int B = 1 << digit_bits;
    const int NB = P * B;
    const size_t out_bytes = static_cast<size_t>(NB) * sizeof(int64_t);
    if (n > 0) {
        if (keys == nullptr || reinterpret_cast<uintptr_t>(keys) % key_bytes != 0)
            return LSCAN_ERR_INVALID;
        if (ranges_overlap(keys, static_cast<size_t>(n) * key_bytes, d_offsets, out_bytes))
            return LSCAN_ERR_INVALID;
    }
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (n == 0)  // every bucket of every position starts at 0
        return cudaMemsetAsync(d_offsets, 0, out_bytes, cs) == cudaSuccess ? LSCAN_OK
                                                                            : LSCAN_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LSCAN_ERR_CUDA;

    // histogram copies: one per warp while they fit the budget
    int copies = kRadixWarps;
    while (copies > 1 && copies * NB * 4 > kRadixSmemBudget) copies /= 2;
    const int smem = copies * NB * 4;
    const void *fn = key_bytes == 4 ? reinterpret_cast<const void *>(&radix_offsets_kernel<uint32_t>)
                                    : reinterpret_cast<const void *>(&radix_offsets_kernel<uint64_t>);
    RadixScratch sc;
    int bps = 1;
    {
        std::lock_guard<std::mutex> lk(g_radix_mu);
        RadixScratch &s = g_radix_scratch[{dev, stream}];
        if (s.counts == nullptr) {
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(cs, &cap) != cudaSuccess) return LSCAN_ERR_CUDA;
            if (cap != cudaStreamCaptureStatusNone) return LSCAN_ERR_BUSY;
            // counters, then the done word on its own 128-byte line
            const size_t bytes = kRadixMaxCounters * sizeof(unsigned long long) + 128;
            if (cudaMalloc(&s.counts, bytes) != cudaSuccess) {
                s.counts = nullptr;
                return LSCAN_ERR_NOMEM;
            }
            if (cudaMemsetAsync(s.counts, 0, bytes, cs) != cudaSuccess) return LSCAN_ERR_CUDA;
            s.done = reinterpret_cast<unsigned int *>(s.counts + kRadixMaxCounters);
        }
        sc = s;
        // the function's shared-memory limit: the budget, once per device
        bool &attr = g_radix_attr[{dev, fn}];
        if (!attr) {
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kRadixSmemBudget) != cudaSuccess)
                return LSCAN_ERR_CUDA;
            attr = true;
        }
        int &nb = g_radix_bps[{{dev, fn}, smem}];
        if (nb == 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kRadixThreads, smem) !=
                    cudaSuccess ||
                nb < 1)
                nb = 1;
        }
        bps = nb;
    }
    int sms = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    // no more CTAs than there are groups of in-flight 16-byte loads
    const int64_t per_cta = static_cast<int64_t>(kRadixThreads) * kRadixUnroll * (16 / key_bytes);
    int64_t grid = static_cast<int64_t>(bps) * sms;
    const int64_t useful = (n + per_cta - 1) / per_cta;
    if (grid > useful) grid = useful;
    if (grid < 1) grid = 1;

    RadixParams rp;
    rp.keys = keys;
    rp.n = n;
    rp.counts = sc.counts;
    rp.done = sc.done;
    rp.offsets = d_offsets;
    rp.digit_bits = digit_bits;
    rp.positions = P;
    rp.copies = copies;
    rp.aligned = reinterpret_cast<uintptr_t>(keys) % 16 == 0 ? 1 : 0;
    void *args[] = {&rp};
    if (cudaLaunchKernel(fn, dim3(static_cast<unsigned>(grid)), dim3(kRadixThreads), args, smem,
                         cs) != cudaSuccess)
        return LSCAN_ERR_CUDA;
    note_launch();
    return LSCAN_OK;
}
