// resident_kernel.cu -- the resident lane of the scan server: a persistent
// kernel on a few SMs that serves small scan requests from a ring in host
// memory mapped for the device, with no CUDA call per request.
//
// Not in the paper (the serving pattern of this library).  Each request is
// scanned by ONE CTA of 512 threads: its elements in chunks of 16384 (8192
// for 8-byte types), each chunk loaded at once (one round trip to memory),
// staged through shared memory (one pad element per 32 elements keeps the
// thread-blocked reads free of bank conflicts) and scanned like the
// single-CTA kernel (a thread-serial scan of 32 or 16 items per thread as
// in Section 2.3, the shuffle scan of Algorithm 2 over thread totals, a
// block scan of warp totals as in Algorithm 3), with the running total of
// the earlier chunks as the carry-in of the next (Section 4.4 applied
// within one CTA).  No CTA waits on another CTA.  The host publishes a
// request by writing its ring entry and then bumping a counter (release); a
// CTA claims the next published entry with an atomic compare-and-swap on a
// counter in device memory, scans it, makes its output visible system-wide
// and writes the entry's done word (release) for the host to poll.  A CTA
// that finds nothing to claim for idle_ns leaves (bounded wait); the host
// launches the kernel again when it publishes work and the kernel has ended.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "kinds.cuh"
#include "lscan_internal.h"
#include "resident.h"
#include "scan_kernel.cuh"

namespace lscan {
namespace {

constexpr int kResThreads = 512;
constexpr int kResWarps = kResThreads / 32;  // 16
// staging (dynamic shared memory): a chunk with one pad element per 32, so
// that thread-blocked reads (lane L reads elements 32L .. 32L + 31) fall in
// distinct banks
constexpr int kResChunkBytes = 66 * 1024;
__device__ __forceinline__ int res_pad(int i) { return i + (i >> 5); }
// elements per chunk: 16384 of up to 4 bytes (32 per thread), 8192 of 8
template <class K>
constexpr int res_chunk() {
    return int(sizeof(typename K::In)) <= 4 && int(sizeof(typename K::Out)) <= 4 ? 16384 : 8192;
}
constexpr int kResSmem = kResChunkBytes + kResWarps * 16 + 16;

__device__ __forceinline__ uint64_t ld_acquire_sys(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_sys32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(uint64_t *p, uint64_t v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// 16 bytes of host-written memory in one access (ordered after an acquire)
__device__ __forceinline__ void ld_relaxed_sys_v2(const void *p, uint64_t &a, uint64_t &b) {
    asm volatile("ld.relaxed.sys.global.v2.u64 {%0, %1}, [%2];"
                 : "=l"(a), "=l"(b)
                 : "l"(p)
                 : "memory");
}

// One request scanned by the whole CTA: chunks of res_chunk<K>() elements
// (one chunk for every request of the small lane with 4-byte types), each
// loaded at once -- every thread issues all of its strided loads before the
// chunk is scanned, so a chunk costs one round trip to memory -- and the
// running carry (the kind's carry type) passed from chunk to chunk.
template <class K>
__device__ __noinline__ void res_scan(const void *xv, void *yv, int64_t n, int inclusive,
                         uint8_t *buf, uint8_t *wbuf, uint8_t *cbuf) {
    using In = typename K::In;
    using Out = typename K::Out;
    using Acc = typename K::Acc;
    using Car = typename K::Car;
    using CarA = typename K::CarA;
    constexpr int CHUNK = res_chunk<K>();
    constexpr int ITEMS = CHUNK / kResThreads;  // 32 or 16
    static_assert((CHUNK + CHUNK / 32) * int(sizeof(In)) <= kResChunkBytes &&
                      (CHUNK + CHUNK / 32) * int(sizeof(Out)) <= kResChunkBytes,
                  "chunk staging");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const In *x = static_cast<const In *>(xv);
    Out *y = static_cast<Out *>(yv);
    In *sx = reinterpret_cast<In *>(buf);
    Out *sy = reinterpret_cast<Out *>(buf);
    Acc *wsum = reinterpret_cast<Acc *>(wbuf);
    Car *carry = reinterpret_cast<Car *>(cbuf);
    if (tid == 0) *carry = K::cident();
    for (int64_t c0 = 0; c0 < n; c0 += CHUNK) {
        const int m = static_cast<int>(n - c0 < CHUNK ? n - c0 : CHUNK);
        In ld[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const int i = tid + k * kResThreads;
            if (i < m) ld[k] = x[c0 + i];
        }
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const int i = tid + k * kResThreads;
            if (i < m) sx[res_pad(i)] = ld[k];
        }
        __syncthreads();
        const int e0 = tid * ITEMS;
        Acc v[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
            v[i] = (e0 + i < m) ? K::load(sx[res_pad(e0 + i)]) : K::ident();
        const Car cin = *carry;
        __syncthreads();  // sx and the carry are reused below
#pragma unroll
        for (int i = 1; i < ITEMS; ++i) v[i] = op_step<K>(v[i - 1], v[i]);
        Acc wv = v[ITEMS - 1];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Acc ov = shfl_up_any(wv, d);
            if (lane >= d) wv = K::op(ov, wv);
        }
        Acc lv = shfl_up_any(wv, 1);
        if (lane == 0) lv = K::ident();
        if (lane == 31) wsum[warp] = wv;
        __syncthreads();
        Acc bv = lane < kResWarps ? wsum[lane] : K::ident();
#pragma unroll
        for (int d = 1; d < kResWarps; d <<= 1) {
            const Acc ov = shfl_up_any(bv, d);
            if (lane >= d) bv = K::op(ov, bv);
        }
        Acc wev = shfl_idx_any(bv, warp > 0 ? warp - 1 : 0);
        if (warp == 0) wev = K::ident();
        const Acc tbv = K::op(wev, lv);
        const CarA B = K::base(K::to_apply(cin), tbv);
        // the last thread's inclusive value covers the chunk (identities pad
        // it): the carry of the next chunk
        if (tid == kResThreads - 1) *carry = K::cop(cin, K::to_car(K::op(tbv, v[ITEMS - 1])));
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            if (e0 + i >= m) break;
            const Acc pv = inclusive ? v[i] : (i == 0 ? K::ident() : v[i - 1]);
            sy[res_pad(e0 + i)] = K::fin(B, pv);
        }
        __syncthreads();
        for (int i = tid; i < m; i += kResThreads) y[c0 + i] = sy[res_pad(i)];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kResThreads, 2) lscan_resident_kernel(const ResParams p) {
    extern __shared__ __align__(16) uint8_t res_smem[];  // kResSmem bytes
    uint8_t *buf = res_smem;                        // chunk staging
    uint8_t *wbuf = res_smem + kResChunkBytes;      // warp totals
    uint8_t *cbuf = wbuf + kResWarps * 16;          // running carry
    __shared__ long long s_idx;
    __shared__ ResReq s_req;
    const int tid = threadIdx.x;
    while (true) {
        if (tid == 0) {
            long long idx = -1;
            const uint64_t t0 = global_timer_ns();
            for (uint32_t it = 0;; ++it) {
                // one round trip to host memory per poll; the stop word only
                // every 64 polls
                const uint64_t pub = ld_acquire_sys(p.published);
                const unsigned long long c =
                    *reinterpret_cast<volatile unsigned long long *>(p.claim);
                if (pub > c) {
                    if (atomicCAS(p.claim, c, c + 1ull) == c) {
                        idx = static_cast<long long>(c);
                        // the entry was written before the counter was
                        // bumped (release / acquire): two 16-byte loads
                        const ResReq *e = p.ring + (idx % p.ring_size);
                        uint64_t w[4];
                        ld_relaxed_sys_v2(e, w[0], w[1]);
                        ld_relaxed_sys_v2(reinterpret_cast<const uint8_t *>(e) + 16, w[2],
                                          w[3]);
                        memcpy(&s_req, w, sizeof(ResReq));
                        break;
                    }
                    continue;  // another CTA took it: try the next one
                }
                if ((it & 63u) == 63u && ld_relaxed_sys32(p.stop) != 0u) break;
                if (global_timer_ns() - t0 > p.idle_ns) break;  // idle: leave
                __nanosleep(100);
            }
            s_idx = idx;
        }
        __syncthreads();
        const long long idx = s_idx;
        if (idx < 0) break;
        const void *x = s_req.x;
        void *y = s_req.y;
        const int64_t n = s_req.n;
        const int kind = s_req.kind;
        const int inclusive = s_req.inclusive;
        switch (kind) {
            case KIND_I32_ADD: res_scan<KI32Add>(x, y, n, inclusive, buf, wbuf, cbuf); break;
            case KIND_I32_MAX: res_scan<KI32Max>(x, y, n, inclusive, buf, wbuf, cbuf); break;
            case KIND_F32_MAX: res_scan<KFMax<float>>(x, y, n, inclusive, buf, wbuf, cbuf); break;
            case KIND_BF16_MAX:
                res_scan<KFMax<uint16_t>>(x, y, n, inclusive, buf, wbuf, cbuf);
                break;
            case KIND_F32_ADD_DF:
                res_scan<KFAddDF<float, float>>(x, y, n, inclusive, buf, wbuf, cbuf);
                break;
            case KIND_BF16_ADD_DF_F32:
                res_scan<KFAddDF<uint16_t, float>>(x, y, n, inclusive, buf, wbuf, cbuf);
                break;
            case KIND_I64_ADD: res_scan<KI64Add>(x, y, n, inclusive, buf, wbuf, cbuf); break;
            case KIND_I64_MAX: res_scan<KI64Max>(x, y, n, inclusive, buf, wbuf, cbuf); break;
            case KIND_F64_MAX: res_scan<KF64Max>(x, y, n, inclusive, buf, wbuf, cbuf); break;
            case KIND_F64_ADD: res_scan<KF64Add>(x, y, n, inclusive, buf, wbuf, cbuf); break;
            default: break;  // the host only publishes the kinds above
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence_system();  // the output before the done word
            st_release_sys(p.done + (idx % p.ring_size), static_cast<uint64_t>(idx) + 1ull);
        }
        __syncthreads();  // s_idx is reused
    }
}

}  // namespace

bool resident_kind_supported(int kind) {
    switch (kind) {
        case KIND_I32_ADD: case KIND_I32_MAX: case KIND_F32_MAX: case KIND_BF16_MAX:
        case KIND_F32_ADD_DF: case KIND_BF16_ADD_DF_F32: case KIND_I64_ADD:
        case KIND_I64_MAX: case KIND_F64_MAX: case KIND_F64_ADD:
            return true;
        default:
            return false;
    }
}

lscan_status launch_resident(const ResParams &p, int ctas, cudaStream_t s) {
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(reinterpret_cast<const void *>(&lscan_resident_kernel),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kResSmem);
    });
    if (attr_err != cudaSuccess) return LSCAN_ERR_CUDA;
    ResParams q = p;
    void *args[] = {&q};
    if (cudaLaunchKernel(reinterpret_cast<const void *>(&lscan_resident_kernel), dim3(ctas),
                         dim3(kResThreads), args, kResSmem, s) != cudaSuccess)
        return LSCAN_ERR_CUDA;
    note_launch();
    return LSCAN_OK;
}

}  // namespace lscan
