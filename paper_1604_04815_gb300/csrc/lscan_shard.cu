// lscan_shard.cu -- the pieces of a scan sharded over devices.
//
// Not in the paper, whose arrays live on one GPU; the method's inter-block
// chaining (Section 4.3) lifted one level up.  An array split into
// contiguous shards, one per device, is scanned in the reduce-then-scan
// form (3N bytes per element pass instead of the 4N of scan-then-add):
//   1. each device reduces its shard to a total in the kind's carry type
//      (lscan_reduce: one pass that reads the shard once);
//   2. the P totals (4 or 8 bytes each) are all-gathered by the caller's
//      collective (NCCL, gloo, ...);
//   3. each device folds the totals of the shards before it
//      (lscan_carry_combine, on the host: P is small) and scans its shard
//      with that fold as the carry-in (lscan_scan, carry_in_type = 1).
// The carry type keeps each precision path's accuracy across the shard
// boundary (an FP64 or double-float total for the float adds that carry so).
//
// lscan_carry_combine restates each kind's carry operator in plain host C++
// (wrapping integer adds, max keeping the earlier operand on ties, the
// double-float two-sum of kinds.cuh written with host float arithmetic), so
// the offset logic runs and is tested without a GPU.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "../../include/lscan.h"
#include "kernel_table.h"
#include "kinds.cuh"
#include "lscan_internal.h"
#include "reduce_kernel.cuh"

namespace lscan {
namespace {

std::mutex g_red_mu;
std::map<std::pair<int, const void *>, int> g_red_bps;  // CTAs per SM

// ---- host restatement of the carry operators ----------------------------
// s + e == a + b exactly (two-sum, TAOCP vol. 2, 4.2.2) in host fp32
void h_two_sum(float a, float b, float *s, float *e) {
    const float ss = a + b;
    const float bb = ss - a;
    *e = (a - (ss - bb)) + (b - bb);
    *s = ss;
}
// the double-float addition of kinds.cuh (df_add)
void h_df_add(const float a[2], const float b[2], float out[2]) {
    float s, se;
    h_two_sum(a[0], b[0], &s, &se);
    const float e = se + (a[1] + b[1]);
    h_two_sum(s, e, &out[0], &out[1]);
}
// order-preserving key of a double's bits (KF64Max)
int64_t h_f64_key(int64_t b) {
    return b ^ static_cast<int64_t>(static_cast<uint64_t>(b >> 63) >> 1);
}
bool h_f64_key_gt(int64_t a, int64_t b) { return a > b && !(b == -1 && a == 0); }

enum CarryOp { C_U32_ADD, C_I32_MAX, C_F32_MAX, C_F32_ADD, C_F64_ADD, C_DF_ADD,
               C_U64_ADD, C_I64_MAX, C_F64_KEY_MAX, C_NONE };

CarryOp carry_op_of(int kind) {
    switch (kind) {
        case KIND_I32_ADD: return C_U32_ADD;
        case KIND_I32_MAX: return C_I32_MAX;
        case KIND_F32_MAX:
        case KIND_BF16_MAX: return C_F32_MAX;
        case KIND_F32_ADD_PLAIN:
        case KIND_BF16_ADD_PLAIN_F32:
        case KIND_BF16_ADD_PLAIN_BF16: return C_F32_ADD;
        case KIND_F32_ADD_F64:
        case KIND_BF16_ADD_F64_F32:
        case KIND_BF16_ADD_F64_BF16:
        case KIND_F64_ADD: return C_F64_ADD;
        case KIND_F32_ADD_DF:
        case KIND_BF16_ADD_DF_F32:
        case KIND_BF16_ADD_DF_BF16:
        case KIND_F32_ADD_COMP:
        case KIND_BF16_ADD_COMP_F32:
        case KIND_BF16_ADD_COMP_BF16: return C_DF_ADD;
        case KIND_I64_ADD: return C_U64_ADD;
        case KIND_I64_MAX: return C_I64_MAX;
        case KIND_F64_MAX: return C_F64_KEY_MAX;
        default: return C_NONE;
    }
}

// acc <- acc (+) v (acc earlier), both of the kind's carry type
void carry_fold(CarryOp op, uint8_t *acc, const uint8_t *v) {
    switch (op) {
        case C_U32_ADD: {
            uint32_t a, b;
            memcpy(&a, acc, 4);
            memcpy(&b, v, 4);
            a += b;
            memcpy(acc, &a, 4);
            break;
        }
        case C_I32_MAX: {
            int32_t a, b;
            memcpy(&a, acc, 4);
            memcpy(&b, v, 4);
            if (b > a) memcpy(acc, &b, 4);
            break;
        }
        case C_F32_MAX: {  // b > a ? b : a: a tie (+0 / -0) keeps the earlier
            float a, b;
            memcpy(&a, acc, 4);
            memcpy(&b, v, 4);
            if (b > a) memcpy(acc, &b, 4);
            break;
        }
        case C_F32_ADD: {
            float a, b;
            memcpy(&a, acc, 4);
            memcpy(&b, v, 4);
            a = a + b;
            memcpy(acc, &a, 4);
            break;
        }
        case C_F64_ADD: {
            double a, b;
            memcpy(&a, acc, 8);
            memcpy(&b, v, 8);
            a = a + b;
            memcpy(acc, &a, 8);
            break;
        }
        case C_DF_ADD: {
            float a[2], b[2], r[2];
            memcpy(a, acc, 8);
            memcpy(b, v, 8);
            h_df_add(a, b, r);
            memcpy(acc, r, 8);
            break;
        }
        case C_U64_ADD: {
            uint64_t a, b;
            memcpy(&a, acc, 8);
            memcpy(&b, v, 8);
            a += b;
            memcpy(acc, &a, 8);
            break;
        }
        case C_I64_MAX: {
            int64_t a, b;
            memcpy(&a, acc, 8);
            memcpy(&b, v, 8);
            if (b > a) memcpy(acc, &b, 8);
            break;
        }
        case C_F64_KEY_MAX: {
            int64_t a, b;
            memcpy(&a, acc, 8);
            memcpy(&b, v, 8);
            if (h_f64_key_gt(b, a)) memcpy(acc, &b, 8);
            break;
        }
        default:
            break;
    }
}

// identity of the carry operator, in the carry type
void carry_identity(CarryOp op, uint8_t *out) {
    memset(out, 0, 8);
    switch (op) {
        case C_I32_MAX: {
            const int32_t v = INT32_MIN;
            memcpy(out, &v, 4);
            break;
        }
        case C_F32_MAX: {
            const float v = -INFINITY;
            memcpy(out, &v, 4);
            break;
        }
        case C_I64_MAX: {
            const int64_t v = INT64_MIN;
            memcpy(out, &v, 8);
            break;
        }
        case C_F64_KEY_MAX: {
            const int64_t v = h_f64_key(static_cast<int64_t>(0xfff0000000000000ull));
            memcpy(out, &v, 8);
            break;
        }
        default:
            break;  // zero: the identity of every add
    }
}

}  // namespace

}  // namespace lscan

using namespace lscan;

extern "C" {

int32_t lscan_carry_bytes(lscan_op op, lscan_dtype dtype, const lscan_options *opts) {
    int kind = -1;
    if (resolve_kind(op, dtype, opts, &kind, nullptr) != LSCAN_OK) return 0;
    return g_carry_bytes[kind];
}

lscan_status lscan_reduce(lscan_op op, lscan_dtype dtype, const void *x, int64_t n,
                          const lscan_options *opts, void *d_total, void *stream) {
    int kind = -1;
    lscan_status st = resolve_kind(op, dtype, opts, &kind, nullptr);
    if (st != LSCAN_OK) return st;
    const int isz = dtype_size(dtype);
    const int cb = g_carry_bytes[kind];
    if (n < 0 || d_total == nullptr || reinterpret_cast<uintptr_t>(d_total) % cb != 0)
        return LSCAN_ERR_INVALID;
    if (n > 0 && (x == nullptr || reinterpret_cast<uintptr_t>(x) % isz != 0))
        return LSCAN_ERR_INVALID;
    if (n > 0) {
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(x), t0 =
                                                                 reinterpret_cast<uintptr_t>(d_total);
        if (t0 < a0 + static_cast<uintptr_t>(n) * isz && a0 < t0 + cb) return LSCAN_ERR_INVALID;
    }
    const void *fn = g_reduce_kernels[kind];
    if (fn == nullptr) return LSCAN_ERR_UNSUPPORTED;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LSCAN_ERR_CUDA;
    int bps = 1;
    {
        std::lock_guard<std::mutex> lk(g_red_mu);
        int &nb = g_red_bps[{dev, fn}];
        if (nb == 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kReduceThreads, 0) !=
                    cudaSuccess ||
                nb < 1)
                nb = 1;
        }
        bps = nb;
    }
    int sms = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    // ranges: 16-byte chunks when x is aligned (elements otherwise), at least
    // one round of in-flight loads per thread each
    const bool aligned = reinterpret_cast<uintptr_t>(x) % 16 == 0;
    const int64_t units = aligned ? n / (16 / isz) : n;
    const int64_t min_units = static_cast<int64_t>(kReduceThreads) * kReduceUnroll;
    int64_t grid = static_cast<int64_t>(bps) * sms;
    const int64_t useful = (units + min_units - 1) / min_units;
    if (grid > useful) grid = useful;
    if (grid < 1) grid = 1;
    const int64_t per = (units + grid - 1) / grid;
    // the scan's per-stream scratch: control block and a status slot per CTA
    DevBuffers db{nullptr, nullptr};
    st = acquire_stream_scratch(stream, static_cast<size_t>(grid) * 4, &db);
    if (st != LSCAN_OK) return st;
    ReduceParams rp;
    rp.x = x;
    rp.n = n;
    rp.units_per_cta = per > 0 ? per : 1;
    rp.aligned = aligned ? 1 : 0;
    rp.reserved = 0;
    rp.ctl = db.ctl;
    rp.status = db.status;
    rp.wait_limit_ns = current_wait_limit_ns();
    rp.skip_tile = take_skip_tile();
    rp.total_out = d_total;
    void *args[] = {&rp};
    if (cudaLaunchKernel(fn, dim3(static_cast<unsigned>(grid)), dim3(kReduceThreads), args, 0,
                         cs) != cudaSuccess)
        return LSCAN_ERR_CUDA;
    note_launch();
    return LSCAN_OK;
}

lscan_status lscan_carry_combine(lscan_op op, lscan_dtype dtype, const lscan_options *opts,
                                 const void *h_totals, int32_t count, void *h_out) {
    int kind = -1;
    const lscan_status st = resolve_kind(op, dtype, opts, &kind, nullptr);
    if (st != LSCAN_OK) return st;
    if (count < 0 || h_out == nullptr || (count > 0 && h_totals == nullptr))
        return LSCAN_ERR_INVALID;
    const CarryOp cop = carry_op_of(kind);
    if (cop == C_NONE) return LSCAN_ERR_UNSUPPORTED;
    const int cb = g_carry_bytes[kind];
    uint8_t acc[8];
    carry_identity(cop, acc);
    const uint8_t *t = static_cast<const uint8_t *>(h_totals);
    for (int32_t i = 0; i < count; ++i) carry_fold(cop, acc, t + static_cast<size_t>(i) * cb);
    memcpy(h_out, acc, cb);
    return LSCAN_OK;
}

}  // extern "C"
