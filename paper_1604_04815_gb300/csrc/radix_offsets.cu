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
//  * Scan.  The CTA that finishes last scans each position's counters into
//    the offsets and re-arms the scratch (finish_offsets).
// With 8-bit digits and at least 2^20 keys the histograms come from joint
// histograms of digit pairs instead (radix_pairs_kernel): half the shared-
// memory atomics per key, each key read by P / 2 CTAs (once from HBM).
// HBM traffic: the keys once (4 or 8 B per key) plus 8 B per counter.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "../../include/lscan.h"
#include "lscan_internal.h"
#include "ptx.cuh"

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
    int32_t groups;              // pair kernel: CTAs that read the same keys
};

// After a CTA has added its counts to p.counts: the CTA that finishes last
// (a done counter; no CTA ever waits) scans each position's B counters, one
// warp per position: each lane takes ceil(B / 32) consecutive buckets and
// scans them serially (the row scan of Section 2.3), and a 5-round shuffle
// scan of the lane totals (Section 2.1, Algorithm 2) gives each lane its
// offset.  It writes the offsets and zeroes the global counters and the done
// counter, so the next launch on the stream starts clean.
template <int THREADS>
__device__ void finish_offsets(const RadixParams &p) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int P = p.positions, B = 1 << p.digit_bits;
    __threadfence();  // this thread's counter updates before the done count
    __syncthreads();
    __shared__ uint32_t is_last;
    if (tid == 0) is_last = atomicAdd(p.done, 1u) == gridDim.x - 1 ? 1u : 0u;
    __syncthreads();
    if (is_last == 0u) return;
    __threadfence();

    const int per_lane = (B + 31) / 32;  // 1 .. 8 consecutive buckets per lane
    for (int q = warp; q < P; q += THREADS / 32) {
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

template <class Key>
__device__ __forceinline__ void count_key(uint32_t *h, Key k, int P, int b, int B,
                                          Key mask) {
    for (int q = 0; q < P; ++q)
        atomicAdd(h + q * B + static_cast<int>((k >> (q * b)) & mask), 1u);
}

template <class Key>
__global__ void __launch_bounds__(kRadixThreads, 3) radix_offsets_kernel(const RadixParams p) {
    extern __shared__ uint32_t hist[];  // copies x P x B
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // launched with programmatic stream serialization: wait for the previous
    // kernel of the stream (it may have re-armed this scratch) first
    grid_dependency_wait();
    grid_launch_dependents();
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
    finish_offsets<kRadixThreads>(p);
}

// ---- joint histograms of digit pairs (8-bit digits, n >= kPairMinKeys) ----
//
// Four shared-memory atomics per 32-bit key (one per digit position) bound
// the kernel above by the shared-memory atomic rate, not by HBM.  Counting
// two adjacent 8-bit digits at once halves them: the 65536-bin histogram of
// the 16-bit field (d_{2m+1}, d_{2m}) gives both digits' histograms as its
// row and column sums.  Its counters are 16 bits wide, two per word (128
// KiB per CTA, one CTA per SM), so one CTA holds one pair: the grid is made
// of groups of G = P / 2 CTAs that read the same keys (the second read of a
// line comes from L2) and member m of a group counts pair m.  Each 16-bit
// half is a 15-bit count below a guard bit: the increment that takes a count
// from 0x7fff to 0x8000 (the atomic returns the old word) clears the guard
// again and adds 32768 to both digits' global counters, so a half never
// carries into its neighbour and the count stays exact for any key
// distribution (a bin needs 32768 more increments to reach the guard's
// neighbour, far more than land while one thread clears it).
constexpr int kPairThreads = 1024;
constexpr int kPairWords = 32768;                       // 65536 16-bit counters
constexpr int kPairSmem = kPairWords * 4 + 2 * 256 * 4;  // table + row/column sums
constexpr int64_t kPairMinKeys = int64_t{1} << 20;

template <class Key>
__device__ __forceinline__ void count_pair(uint32_t *tab, Key k, int sh, int m,
                                           unsigned long long *counts) {
    const uint32_t bin = static_cast<uint32_t>(k >> sh) & 0xffffu;
    const uint32_t s = (bin & 1u) * 16u;
    const uint32_t old = atomicAdd(tab + (bin >> 1), 1u << s);
    if (((old >> s) & 0xffffu) == 0x7fffu) {
        // this increment set the guard bit: clear it, count 32768 globally
        atomicAdd(tab + (bin >> 1), 0u - (0x8000u << s));
        atomicAdd(counts + (2 * m) * 256 + (bin & 255u), 32768ull);
        atomicAdd(counts + (2 * m + 1) * 256 + (bin >> 8), 32768ull);
    }
}

template <class Key>
__global__ void __launch_bounds__(kPairThreads, 1) radix_pairs_kernel(const RadixParams p) {
    extern __shared__ uint32_t tab[];  // kPairWords, then row and column sums
    // launched with programmatic stream serialization: wait for the previous
    // kernel of the stream (it may have re-armed this scratch) first
    grid_dependency_wait();
    grid_launch_dependents();
    uint32_t *srow = tab + kPairWords;     // [256] by the high digit of the pair
    uint32_t *scol = srow + 256;           // [256] by the low digit
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < kPairWords + 512; i += kPairThreads) tab[i] = 0u;
    __syncthreads();

    const int G = p.groups;
    const int m = static_cast<int>(blockIdx.x) % G;    // the pair this CTA counts
    const int64_t c = blockIdx.x / G, C = gridDim.x / G;  // key stream of the group
    const int sh = 16 * m;
    const Key *keys = static_cast<const Key *>(p.keys);
    const int64_t gtid = c * kPairThreads + tid;
    const int64_t gstride = C * kPairThreads;
    int64_t rest = 0;
    if (p.aligned) {
        constexpr int EPV = 16 / int(sizeof(Key));
        const int64_t nv = p.n / EPV;
        const uint4 *kv = reinterpret_cast<const uint4 *>(keys);
        for (int64_t i = gtid; i < nv; i += kRadixUnroll * gstride) {
            uint4 q[kRadixUnroll];
#pragma unroll
            for (int u = 0; u < kRadixUnroll; ++u)
                if (i + u * gstride < nv) q[u] = kv[i + u * gstride];
#pragma unroll
            for (int u = 0; u < kRadixUnroll; ++u) {
                if (i + u * gstride >= nv) break;
                Key e[EPV];
                memcpy(e, &q[u], 16);
#pragma unroll
                for (int x = 0; x < EPV; ++x) count_pair<Key>(tab, e[x], sh, m, p.counts);
            }
        }
        rest = nv * EPV;
    }
    for (int64_t j = rest + gtid; j < p.n; j += gstride) count_pair<Key>(tab, keys[j], sh, m, p.counts);
    __syncthreads();

    // row sums (high digit) and column sums (low digit) of the 256 x 256
    // table: word hi * 128 + lo / 2 holds lo even (low half) and lo odd.
    // Thread t reads column word t % 128 of rows t / 128, t / 128 + 8, ...
    {
        const int cw = tid & 127;
        uint32_t c0 = 0u, c1 = 0u;
        for (int hi = tid >> 7; hi < 256; hi += kPairThreads / 128) {
            const uint32_t w = tab[hi * 128 + cw];
            c0 += w & 0xffffu;
            c1 += w >> 16;
            uint32_t r = (w & 0xffffu) + (w >> 16);
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) r += __shfl_down_sync(0xffffffffu, r, d);
            if (lane == 0) atomicAdd(srow + hi, r);
        }
        atomicAdd(scol + 2 * cw, c0);
        atomicAdd(scol + 2 * cw + 1, c1);
    }
    __syncthreads();
    for (int i = tid; i < 512; i += kPairThreads) {
        const uint32_t v = i < 256 ? scol[i] : srow[i - 256];
        const int pos = i < 256 ? 2 * m : 2 * m + 1;
        if (v != 0u)
            atomicAdd(p.counts + pos * 256 + (i & 255), static_cast<unsigned long long>(v));
    }
    finish_offsets<kPairThreads>(p);
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

    int sms = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    // 8-bit digits on a large array: joint histograms of digit pairs
    const bool pairs = digit_bits == 8 && n >= kPairMinKeys && sms >= P / 2;
    // histogram copies: one per warp while they fit the budget
    int copies = kRadixWarps;
    while (copies > 1 && copies * NB * 4 > kRadixSmemBudget) copies /= 2;
    const int smem = copies * NB * 4;
    const void *fn =
        pairs ? (key_bytes == 4 ? reinterpret_cast<const void *>(&radix_pairs_kernel<uint32_t>)
                                : reinterpret_cast<const void *>(&radix_pairs_kernel<uint64_t>))
              : (key_bytes == 4 ? reinterpret_cast<const void *>(&radix_offsets_kernel<uint32_t>)
                                : reinterpret_cast<const void *>(&radix_offsets_kernel<uint64_t>));
    const int fn_smem = pairs ? kPairSmem : smem;
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
        // the function's shared-memory limit, once per device
        bool &attr = g_radix_attr[{dev, fn}];
        if (!attr) {
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     pairs ? kPairSmem : kRadixSmemBudget) != cudaSuccess)
                return LSCAN_ERR_CUDA;
            attr = true;
        }
        int &nb = g_radix_bps[{{dev, fn}, fn_smem}];
        if (nb == 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &nb, fn, pairs ? kPairThreads : kRadixThreads, fn_smem) != cudaSuccess ||
                nb < 1)
                nb = 1;
        }
        bps = nb;
    }
    // no more CTAs (pair kernel: groups) than there are groups of in-flight
    // 16-byte loads
    const int threads = pairs ? kPairThreads : kRadixThreads;
    const int group = pairs ? P / 2 : 1;
    const int64_t per_cta = static_cast<int64_t>(threads) * kRadixUnroll * (16 / key_bytes);
    int64_t streams = static_cast<int64_t>(bps) * sms / group;
    const int64_t useful = (n + per_cta - 1) / per_cta;
    if (streams > useful) streams = useful;
    if (streams < 1) streams = 1;
    const int64_t grid = streams * group;

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
    rp.groups = group;
    void *args[] = {&rp};
    if (launch_serialized(fn, dim3(static_cast<unsigned>(grid)), dim3(threads), fn_smem, cs,
                          args) != cudaSuccess)
        return LSCAN_ERR_CUDA;
    note_launch();
    return LSCAN_OK;
}
