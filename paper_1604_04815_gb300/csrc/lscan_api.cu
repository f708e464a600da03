// lscan_api.cu -- the C ABI of liblscan.so: argument checks, kernel choice,
// per-stream scratch, launch, device error read-back.
//
// One scan is one kernel launch (LightScan Section 5.1: "only one kernel
// launch is needed").  The scratch a launch needs -- a status word per tile,
// the tile ticket, the epoch that tags status words, the error word -- lives
// in device memory owned by this library, one set per (device, stream), and
// is re-armed by the kernel itself (the last CTA resets the ticket and bumps
// the epoch), so no memset runs between launches and graph replays work.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "../../include/lscan.h"
#include "kernel_table.h"
#include "kinds.cuh"
#include "lscan_internal.h"

namespace lscan {

KernelEntry g_kernels[kNumKinds][MODE_COUNT][kNumVariants];
const void *g_tiny_kernels[kNumKinds] = {};
const void *g_reduce_kernels[kNumKinds] = {};
int g_carry_bytes[kNumKinds] = {};

void register_i32_add();
void register_i32_max();
void register_f32_max();
void register_bf16_max();
void register_f32_add_plain();
void register_f32_add_f64();
void register_f32_add_comp();
void register_bf16_add_plain_f32();
void register_bf16_add_f64_f32();
void register_bf16_add_comp_f32();
void register_bf16_add_plain_bf16();
void register_bf16_add_f64_bf16();
void register_bf16_add_comp_bf16();
void register_i64_add();
void register_i64_max();
void register_f64_max();
void register_f64_add();
void register_f32_add_df();
void register_bf16_add_df_f32();
void register_bf16_add_df_bf16();
void register_select();

void register_all_kernels() {
    register_i32_add();
    register_i32_max();
    register_f32_max();
    register_bf16_max();
    register_f32_add_plain();
    register_f32_add_f64();
    register_f32_add_comp();
    register_bf16_add_plain_f32();
    register_bf16_add_f64_f32();
    register_bf16_add_comp_f32();
    register_bf16_add_plain_bf16();
    register_bf16_add_f64_bf16();
    register_bf16_add_comp_bf16();
    register_i64_add();
    register_i64_max();
    register_f64_max();
    register_f64_add();
    register_f32_add_df();
    register_bf16_add_df_f32();
    register_bf16_add_df_bf16();
    register_select();
}

namespace {

std::mutex g_mu;
std::once_flag g_reg_once;
std::atomic<uint64_t> g_launches{0};
std::atomic<uint64_t> g_wait_limit_ns{1000000000ull};
std::atomic<int64_t> g_skip_tile{-1};

struct Scratch {
    int device = -1;
    uint32_t *ctl = nullptr;     // CTL_WORDS
    uint64_t *status = nullptr;  // status_words
    size_t status_words = 0;
    uint64_t launches = 0;       // launches since the last full reset
};

std::map<std::pair<int, void *>, Scratch *> g_scratch;

// cuTensorMapEncodeTiled, looked up once through the runtime (the library
// does not link the driver library itself)
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);
std::once_flag g_encode_once;
EncodeTiledFn g_encode = nullptr;

EncodeTiledFn encode_tiled() {
    std::call_once(g_encode_once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<EncodeTiledFn>(f);
    });
    return g_encode;
}

// Tensor map of `bytes` bytes at `base` (16-byte aligned) seen as 1024-byte
// blocks of eight 128-byte lines: dimensions [blocks][8][128], complete
// blocks only (a tile that reaches past the last one is never copied through
// the map).  One copy moves `blocks_per_copy` consecutive blocks, laid out in
// shared memory with the 128-byte swizzle.
bool encode_block_map(CUtensorMap *m, const void *base, uint64_t bytes, int blocks_per_copy) {
    EncodeTiledFn f = encode_tiled();
    if (f == nullptr || blocks_per_copy < 1 || blocks_per_copy > 256) return false;
    const uint64_t blocks = bytes / 1024u;
    if (blocks == 0 || blocks > static_cast<uint64_t>(INT32_MAX)) return false;
    const cuuint64_t dim[3] = {128u, 8u, blocks};
    const cuuint64_t stride[2] = {128u, 1024u};
    const cuuint32_t box[3] = {128u, 8u, static_cast<cuuint32_t>(blocks_per_copy)};
    const cuuint32_t step[3] = {1u, 1u, 1u};
    auto encode = [&] {
        return f(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3u, const_cast<void *>(base), dim, stride,
                 box, step, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    };
    CUresult r = encode();
    if (r == CUDA_ERROR_INVALID_CONTEXT) {
        // a host thread whose runtime calls so far bound no context (the
        // encoder needs one): bind the current device's primary context,
        // as the launch that follows would, and encode again
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess)
            r = encode();
    }
    return r == CUDA_SUCCESS;
}

struct FnState {
    bool attr_set = false;
    int blocks_per_sm = 0;
};
// Per-kernel and per-device launch facts, filled on first use by whichever
// host thread launches first (the API under g_mu, the no-allocation entry
// point, the server thread and graph capture all launch), so they have a
// lock of their own.
std::mutex g_prep_mu;
std::map<std::pair<int, const void *>, FnState> g_fn_state;
std::map<int, int> g_sm_count;

constexpr uint64_t kEpochPeriod = (1ull << 30) - 1;

}  // namespace

int sm_count(int dev) {
    std::lock_guard<std::mutex> lk(g_prep_mu);
    auto it = g_sm_count.find(dev);
    if (it != g_sm_count.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        n = 1;
    g_sm_count[dev] = n;
    return n;
}

// Kind id for (op, dtype, out dtype, precision); -1 if not built.
int select_kind(int op, int dtype, int out_dtype, int precision) {
    if (op == LSCAN_MAX) {
        if (out_dtype != dtype) return -1;
        if (dtype == LSCAN_I32) return KIND_I32_MAX;
        if (dtype == LSCAN_F32) return KIND_F32_MAX;
        if (dtype == LSCAN_BF16) return KIND_BF16_MAX;
        if (dtype == LSCAN_I64) return KIND_I64_MAX;
        if (dtype == LSCAN_F64) return KIND_F64_MAX;
        return -1;
    }
    if (op != LSCAN_ADD) return -1;
    if (dtype == LSCAN_I32) return out_dtype == LSCAN_I32 ? KIND_I32_ADD : -1;
    if (dtype == LSCAN_I64) return out_dtype == LSCAN_I64 ? KIND_I64_ADD : -1;
    if (dtype == LSCAN_F64) {
        // one path: double in tile and in the carry chain
        const bool ok = precision == LSCAN_PREC_DEFAULT || precision == LSCAN_PREC_F64_CARRY;
        return (out_dtype == LSCAN_F64 && ok) ? KIND_F64_ADD : -1;
    }
    const int prec = precision == LSCAN_PREC_DEFAULT ? LSCAN_PREC_DF_CARRY : precision;
    // kinds by precision path: fp32 carry, FP64 carry, compensated,
    // double-float carry
    static const int kF32[] = {KIND_F32_ADD_PLAIN, KIND_F32_ADD_F64, KIND_F32_ADD_COMP,
                               KIND_F32_ADD_DF};
    static const int kBf16F32[] = {KIND_BF16_ADD_PLAIN_F32, KIND_BF16_ADD_F64_F32,
                                   KIND_BF16_ADD_COMP_F32, KIND_BF16_ADD_DF_F32};
    static const int kBf16Bf16[] = {KIND_BF16_ADD_PLAIN_BF16, KIND_BF16_ADD_F64_BF16,
                                    KIND_BF16_ADD_COMP_BF16, KIND_BF16_ADD_DF_BF16};
    if (prec < LSCAN_PREC_F32_CARRY || prec > LSCAN_PREC_DF_CARRY) return -1;
    const int pi = prec - LSCAN_PREC_F32_CARRY;
    if (dtype == LSCAN_F32) return out_dtype == LSCAN_F32 ? kF32[pi] : -1;
    if (dtype == LSCAN_BF16) {
        if (out_dtype == LSCAN_F32) return kBf16F32[pi];
        if (out_dtype == LSCAN_BF16) return kBf16Bf16[pi];
    }
    return -1;
}

int dtype_size(int dt) {
    if (dt == LSCAN_I32 || dt == LSCAN_F32) return 4;
    if (dt == LSCAN_BF16) return 2;
    if (dt == LSCAN_I64 || dt == LSCAN_F64) return 8;
    return 0;
}

// Occupancy-derived persistent grid size for a kernel on device dev.
static lscan_status kernel_prepare(int dev, const KernelEntry &e, int *blocks_per_sm) {
    std::lock_guard<std::mutex> lk(g_prep_mu);
    FnState &st = g_fn_state[{dev, e.fn}];
    if (!st.attr_set) {
        if (cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 e.smem) != cudaSuccess)
            return LSCAN_ERR_CUDA;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, e.fn, e.threads,
                                                          e.smem) != cudaSuccess)
            return LSCAN_ERR_CUDA;
        st.blocks_per_sm = nb > 0 ? nb : 1;
        st.attr_set = true;
    }
    *blocks_per_sm = st.blocks_per_sm;
    return LSCAN_OK;
}

static bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

// Scratch for (current device, stream), with room for `words` status words.
static lscan_status get_scratch(void *stream, size_t words, Scratch **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LSCAN_ERR_CUDA;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    Scratch *&sc = g_scratch[{dev, stream}];
    if (sc == nullptr) {
        if (stream_capturing(cs)) return LSCAN_ERR_BUSY;
        sc = new Scratch();
        sc->device = dev;
        if (cudaMalloc(&sc->ctl, CTL_WORDS * sizeof(uint32_t)) != cudaSuccess) {
            delete sc;
            sc = nullptr;
            return LSCAN_ERR_NOMEM;
        }
        if (cudaMemsetAsync(sc->ctl, 0, CTL_WORDS * sizeof(uint32_t), cs) != cudaSuccess)
            return LSCAN_ERR_CUDA;
    }
    if (sc->status_words < words) {
        if (stream_capturing(cs)) return LSCAN_ERR_BUSY;
        size_t want = sc->status_words ? sc->status_words : 4096;
        while (want < words) want *= 2;
        if (sc->status) {
            // earlier launches on this stream may still read the old array
            if (cudaStreamSynchronize(cs) != cudaSuccess) return LSCAN_ERR_CUDA;
            cudaFree(sc->status);
            sc->status = nullptr;
            sc->status_words = 0;
        }
        if (cudaMalloc(&sc->status, want * sizeof(uint64_t)) != cudaSuccess)
            return LSCAN_ERR_NOMEM;
        if (cudaMemsetAsync(sc->status, 0, want * sizeof(uint64_t), cs) != cudaSuccess)
            return LSCAN_ERR_CUDA;
        sc->status_words = want;
    }
    *out = sc;
    return LSCAN_OK;
}

// Every 2^30 - 1 launches the epoch field of the tags would wrap; clear the
// status array and control block then, so an old tag can never match.
static lscan_status epoch_maintenance(Scratch *sc, cudaStream_t cs) {
    if (++sc->launches < kEpochPeriod) return LSCAN_OK;
    if (stream_capturing(cs)) return LSCAN_OK;  // retried on the next launch
    if (cudaMemsetAsync(sc->status, 0, sc->status_words * sizeof(uint64_t), cs) !=
            cudaSuccess ||
        cudaMemsetAsync(sc->ctl, 0, CTL_WORDS * sizeof(uint32_t), cs) != cudaSuccess)
        return LSCAN_ERR_CUDA;
    sc->launches = 0;
    return LSCAN_OK;
}

static bool ranges_partially_overlap(const void *x, size_t xb, const void *y, size_t yb) {
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(x), a1 = a0 + xb;
    const uintptr_t b0 = reinterpret_cast<uintptr_t>(y), b1 = b0 + yb;
    if (a1 <= b0 || b1 <= a0) return false;  // disjoint
    return !(a0 == b0 && xb == yb);          // identical = in place
}

lscan_status launch_scan(const LaunchSpec &ls, const DevBuffers &buf,
                         cudaStream_t cs) {
    if (ls.tiny) {
        // at most one tile: one CTA, no carry, no scratch
        TinyParams tp;
        tp.x = ls.x;
        tp.y = ls.y;
        tp.n = static_cast<int32_t>(ls.n);
        tp.inclusive = ls.inclusive ? 1 : 0;
        tp.carry_in = ls.carry_in;
        tp.carry_in_car = ls.carry_in_car ? 1 : 0;
        tp.reserved = 0;
        tp.total_out = ls.total_out;
        void *args[] = {&tp};
        if (launch_serialized(g_tiny_kernels[ls.kind], dim3(1), dim3(kTinyThreads), 0, cs, args) !=
            cudaSuccess)
            return LSCAN_ERR_CUDA;
        g_launches.fetch_add(1);
        return LSCAN_OK;
    }
    const KernelEntry &e = g_kernels[ls.kind][ls.mode][ls.variant];
    if (e.fn == nullptr) return LSCAN_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LSCAN_ERR_CUDA;
    int bps = 1;
    lscan_status st = kernel_prepare(dev, e, &bps);
    if (st != LSCAN_OK) return st;
    const int64_t n_tiles =
        ls.mode == MODE_LIST ? ls.list_tiles : (ls.n + e.tile - 1) / e.tile;
    int sms = sm_count(dev) - ls.reserve_sms;
    if (sms < 1) sms = 1;
    int64_t grid = static_cast<int64_t>(bps) * sms;
    if (ls.max_ctas > 0 && grid > ls.max_ctas) grid = ls.max_ctas;
    if (grid > n_tiles) grid = n_tiles;
    if (grid < 1) grid = 1;

    ScanParams p;
    p.x = ls.x;
    p.y = ls.y;
    p.n = ls.n;
    p.n_tiles = n_tiles;
    p.offsets = ls.offsets;
    p.n_seg = ls.n_seg;
    p.segs = static_cast<const SegDesc *>(ls.segs);
    p.ctl = buf.ctl;
    p.status = buf.status;
    p.wait_limit_ns = g_wait_limit_ns.load();
    p.skip_tile = g_skip_tile.exchange(-1);
    p.inclusive = ls.inclusive ? 1 : 0;
    p.carry_mode = ls.carry_mode;
    p.carry_in = ls.carry_in;
    p.carry_in_car = ls.carry_in_car ? 1 : 0;
    p.reserved = 0;
    p.total_out = ls.mode == MODE_SINGLE ? ls.total_out : nullptr;
    p.values = ls.values;
    p.count_out = ls.count_out;
    p.err_host = ls.err_host;
    std::memset(&p.tm_x, 0, sizeof(p.tm_x));
    std::memset(&p.tm_y, 0, sizeof(p.tm_y));
    if (ls.mode == MODE_SINGLE && ls.n >= e.tile) {
        // full tiles exist: their swizzled copies go through the maps (a
        // tile of x per copy; each consumer warp stores its rows of y)
        if (e.swz_in != 0 &&
            !encode_block_map(&p.tm_x, ls.x, static_cast<uint64_t>(ls.n) * e.in_size,
                              e.tile * e.in_size / 1024))
            return LSCAN_ERR_CUDA;
        if (e.swz_out != 0 &&
            !encode_block_map(&p.tm_y, ls.y, static_cast<uint64_t>(ls.n) * e.out_size,
                              32 * e.items * e.out_size / 1024))
            return LSCAN_ERR_CUDA;
    }
    void *args[] = {&p};
    cudaError_t ce = launch_serialized(e.fn, dim3(static_cast<unsigned>(grid)),
                                       dim3(e.threads), e.smem, cs, args);
    if (ce != cudaSuccess) return LSCAN_ERR_CUDA;
    g_launches.fetch_add(1);
    return LSCAN_OK;
}

lscan_status resolve_kind(int op, int dtype, const lscan_options *opts, int *kind,
                          int *out_dtype) {
    std::call_once(g_reg_once, register_all_kernels);
    if (dtype_size(dtype) == 0 || (op != LSCAN_ADD && op != LSCAN_MAX)) return LSCAN_ERR_INVALID;
    int od = dtype;
    if (op == LSCAN_ADD && dtype == LSCAN_BF16) od = LSCAN_F32;
    if (opts && opts->out_dtype > 0 && opts->out_dtype <= LSCAN_F64) od = opts->out_dtype;
    const int prec = opts ? opts->precision : LSCAN_PREC_DEFAULT;
    const int k = select_kind(op, dtype, od, prec);
    if (k < 0) return LSCAN_ERR_UNSUPPORTED;
    *kind = k;
    if (out_dtype) *out_dtype = od;
    return LSCAN_OK;
}

lscan_status plan_scan(int op, int dtype, int inclusive, const void *x, void *y,
                       int64_t n, const lscan_options *opts, int mode,
                       const int64_t *offsets, int64_t n_seg, LaunchSpec *ls) {
    std::call_once(g_reg_once, register_all_kernels);
    if (n < 0) return LSCAN_ERR_INVALID;
    const int isz = dtype_size(dtype);
    if (isz == 0 || (op != LSCAN_ADD && op != LSCAN_MAX)) return LSCAN_ERR_INVALID;
    int kind = -1, out_dtype = dtype;
    lscan_status rs = resolve_kind(op, dtype, opts, &kind, &out_dtype);
    if (rs != LSCAN_OK) return rs;
    const int osz = dtype_size(out_dtype);
    if (n > 0) {
        if (x == nullptr || y == nullptr) return LSCAN_ERR_INVALID;
        if ((reinterpret_cast<uintptr_t>(x) % isz) != 0 ||
            (reinterpret_cast<uintptr_t>(y) % osz) != 0)
            return LSCAN_ERR_INVALID;
        if (ranges_partially_overlap(x, static_cast<size_t>(n) * isz, y,
                                     static_cast<size_t>(n) * osz))
            return LSCAN_ERR_INVALID;
    }
    int cfg = opts ? opts->config : 0;
    if (cfg < 0 || cfg > kNumTmaCfg) return LSCAN_ERR_INVALID;
    int tuned_carry = LSCAN_CARRY_AUTO;
    int variant = cfg > 0 ? cfg : tuned_variant(kind, mode, n, &tuned_carry);
    const bool aligned = (reinterpret_cast<uintptr_t>(x) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(y) % 16 == 0);
    if (!aligned) variant = 0;
    const KernelEntry &e = g_kernels[kind][mode][variant];
    if (e.fn == nullptr) return LSCAN_ERR_UNSUPPORTED;
    const int64_t n_tiles = (n + e.tile - 1) / e.tile;
    if (n_tiles > (int64_t{1} << 31) - 1) return LSCAN_ERR_INVALID;
    int carry = opts ? opts->carry : LSCAN_CARRY_AUTO;
    if (carry < LSCAN_CARRY_AUTO || carry > LSCAN_CARRY_CHAINED) return LSCAN_ERR_INVALID;
    // AUTO takes what the autotuner measured for this size (look-back unless
    // the chained hand-off won)
    if (carry == LSCAN_CARRY_AUTO && cfg == 0) carry = tuned_carry;
    const void *carry_in = opts ? opts->carry_in : nullptr;
    const int cit = opts ? opts->carry_in_type : 0;
    if (cit < 0 || cit > 1) return LSCAN_ERR_INVALID;
    // a carry-in is one output element, or (type 1) a value of the kind's
    // carry type, aligned to its size
    const int cin_align = cit == 1 ? g_carry_bytes[kind] : osz;
    if (carry_in && (mode != MODE_SINGLE || reinterpret_cast<uintptr_t>(carry_in) % cin_align != 0))
        return LSCAN_ERR_INVALID;

    ls->kind = kind;
    ls->mode = mode;
    ls->variant = variant;
    ls->x = x;
    ls->y = y;
    ls->n = n;
    ls->offsets = offsets;
    ls->n_seg = n_seg;
    ls->inclusive = inclusive != 0;
    ls->carry_mode = carry == LSCAN_CARRY_CHAINED ? CARRY_CHAINED : CARRY_LOOKBACK;
    ls->max_ctas = opts ? opts->max_ctas : 0;
    ls->status_words = static_cast<size_t>(n_tiles) * e.car_words;
    ls->carry_in = carry_in;
    ls->carry_in_car = carry_in != nullptr && cit == 1;
    // arrays of at most one tile take the single-CTA kernel when the tile
    // configuration is left to the library
    ls->tiny = mode == MODE_SINGLE && cfg == 0 && n > 0 && n <= kTinyMax &&
               g_tiny_kernels[kind] != nullptr;
    if (ls->tiny) ls->status_words = 0;
    return LSCAN_OK;
}

lscan_status run_planned(const LaunchSpec &ls, void *stream) {
    if (ls.n == 0) return LSCAN_OK;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (ls.tiny) return launch_scan(ls, DevBuffers{nullptr, nullptr}, cs);
    std::lock_guard<std::mutex> lk(g_mu);
    Scratch *sc = nullptr;
    lscan_status st = get_scratch(stream, ls.status_words, &sc);
    if (st != LSCAN_OK) return st;
    st = epoch_maintenance(sc, cs);
    if (st != LSCAN_OK) return st;
    DevBuffers b{sc->ctl, sc->status};
    return launch_scan(ls, b, cs);
}

std::mutex &api_mutex() { return g_mu; }

lscan_status acquire_stream_scratch(void *stream, size_t words, DevBuffers *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    Scratch *sc = nullptr;
    lscan_status st = get_scratch(stream, words, &sc);
    if (st != LSCAN_OK) return st;
    st = epoch_maintenance(sc, static_cast<cudaStream_t>(stream));
    if (st != LSCAN_OK) return st;
    *out = DevBuffers{sc->ctl, sc->status};
    return LSCAN_OK;
}

uint64_t current_wait_limit_ns() { return g_wait_limit_ns.load(); }

int64_t take_skip_tile() { return g_skip_tile.exchange(-1); }

int planned_tile(const LaunchSpec &ls) {
    return g_kernels[ls.kind][ls.mode][ls.variant].tile;
}

int64_t planned_tiles(const LaunchSpec &ls) {
    if (ls.mode == MODE_LIST) return ls.list_tiles;
    const int64_t tile = planned_tile(ls);
    return (ls.n + tile - 1) / tile;
}

void ensure_kernels_registered() { std::call_once(g_reg_once, register_all_kernels); }

int carry_words(int kind) { return g_kernels[kind][MODE_SINGLE][1].car_words; }  // config 1

void note_launch() { g_launches.fetch_add(1); }

cudaError_t launch_serialized(const void *fn, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, void **args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = grid;
    lc.blockDim = block;
    lc.dynamicSmemBytes = smem;
    lc.stream = stream;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelExC(&lc, fn, args);
}

}  // namespace lscan

using namespace lscan;

extern "C" {

lscan_status lscan_scan(lscan_op op, lscan_dtype dtype, int inclusive, const void *x,
                        void *y, int64_t n, const lscan_options *opts, void *stream) {
    LaunchSpec ls;
    lscan_status st = plan_scan(op, dtype, inclusive, x, y, n, opts, MODE_SINGLE,
                                nullptr, 0, &ls);
    if (st != LSCAN_OK) return st;
    return run_planned(ls, stream);
}

lscan_status lscan_inclusive(lscan_op op, lscan_dtype dtype, const void *x, void *y,
                             int64_t n, void *stream) {
    return lscan_scan(op, dtype, 1, x, y, n, nullptr, stream);
}

lscan_status lscan_exclusive(lscan_op op, lscan_dtype dtype, const void *x, void *y,
                             int64_t n, void *stream) {
    return lscan_scan(op, dtype, 0, x, y, n, nullptr, stream);
}

lscan_status lscan_batched(lscan_op op, lscan_dtype dtype, int inclusive, const void *x,
                           void *y, const int64_t *d_offsets, int64_t n_seg,
                           int64_t n_total, const lscan_options *opts, void *stream) {
    if (n_seg < 0 || n_total < 0) return LSCAN_ERR_INVALID;
    if (n_total > 0 && (d_offsets == nullptr || n_seg == 0)) return LSCAN_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(d_offsets) % 8 != 0) return LSCAN_ERR_INVALID;
    LaunchSpec ls;
    lscan_status st = plan_scan(op, dtype, inclusive, x, y, n_total, opts,
                                MODE_SEGMENTED, d_offsets, n_seg, &ls);
    if (st != LSCAN_OK) return st;
    return run_planned(ls, stream);
}

lscan_status lscan_stream_status(void *stream) {
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(cs) != cudaSuccess) return LSCAN_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LSCAN_ERR_CUDA;
    uint32_t *ctl = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_scratch.find({dev, stream});
        if (it == g_scratch.end()) return LSCAN_OK;
        ctl = it->second->ctl;
    }
    uint32_t err = 0;
    if (cudaMemcpy(&err, ctl + CTL_ERROR, sizeof(err), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return LSCAN_ERR_CUDA;
    if (err == 0) return LSCAN_OK;
    if (cudaMemset(ctl + CTL_ERROR, 0, sizeof(uint32_t)) != cudaSuccess)
        return LSCAN_ERR_CUDA;
    if (err & (DEV_ERR_CARRY_WAIT | DEV_ERR_BARRIER_WAIT)) return LSCAN_ERR_TIMEOUT;
    return LSCAN_ERR_DEVICE;
}

lscan_status lscan_reserve(void *stream, int64_t max_elems) {
    if (max_elems < 0) return LSCAN_ERR_INVALID;
    std::call_once(g_reg_once, register_all_kernels);
    // the most status words any built kernel needs for max_elems elements
    size_t words = 0;
    for (int k = 0; k < kNumKinds; ++k)
        for (int m = 0; m < MODE_COUNT; ++m)
            for (int v = 0; v < kNumVariants; ++v) {
                const KernelEntry &e = g_kernels[k][m][v];
                if (!e.fn) continue;
                const size_t w = static_cast<size_t>((max_elems + e.tile - 1) / e.tile) *
                                 static_cast<size_t>(e.car_words);
                if (w > words) words = w;
            }
    std::lock_guard<std::mutex> lk(g_mu);
    Scratch *sc = nullptr;
    return get_scratch(stream, words > 0 ? words : 1, &sc);
}

void lscan_shutdown(void) {
    shutdown_host_pipes();
    shutdown_radix();
    std::lock_guard<std::mutex> lk(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_scratch) {
        Scratch *sc = kv.second;
        if (!sc) continue;
        cudaSetDevice(sc->device);
        cudaDeviceSynchronize();
        if (sc->status) cudaFree(sc->status);
        if (sc->ctl) cudaFree(sc->ctl);
        delete sc;
    }
    g_scratch.clear();
    cudaSetDevice(cur);
    shutdown_graphs_locked();
}

const char *lscan_strerror(lscan_status s) {
    switch (s) {
        case LSCAN_OK: return "ok";
        case LSCAN_ERR_INVALID: return "invalid argument";
        case LSCAN_ERR_UNSUPPORTED: return "unsupported combination";
        case LSCAN_ERR_CUDA: return "CUDA runtime error";
        case LSCAN_ERR_TIMEOUT: return "device wait ran out of time";
        case LSCAN_ERR_NOMEM: return "out of device memory or budget";
        case LSCAN_ERR_BUSY: return "scratch must grow during stream capture";
        case LSCAN_ERR_DEVICE: return "device reported malformed input";
    }
    return "unknown status";
}

const char *lscan_version(void) { return "lscan 0.1 (sm_103a)"; }

uint64_t lscan_launch_count(void) { return g_launches.load(); }

lscan_status lscan_set_wait_limit_ns(uint64_t ns) {
    if (ns == 0) return LSCAN_ERR_INVALID;
    g_wait_limit_ns.store(ns);
    return LSCAN_OK;
}

lscan_status lscan_debug_skip_publish(int64_t tile) {
    g_skip_tile.store(tile < 0 ? -1 : tile);
    return LSCAN_OK;
}

int32_t lscan_num_configs(void) { return kNumTmaCfg; }

lscan_status lscan_select_flagged(lscan_dtype dtype, const void *x, const uint8_t *flags,
                                  void *y, int64_t n, int64_t *d_count, void *stream) {
    std::call_once(g_reg_once, register_all_kernels);
    const int vsz = dtype_size(dtype);
    if (vsz == 0 || n < 0 || d_count == nullptr ||
        reinterpret_cast<uintptr_t>(d_count) % 8 != 0)
        return LSCAN_ERR_INVALID;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (n == 0)
        return cudaMemsetAsync(d_count, 0, sizeof(int64_t), cs) == cudaSuccess ? LSCAN_OK
                                                                             : LSCAN_ERR_CUDA;
    if (x == nullptr || flags == nullptr || y == nullptr) return LSCAN_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(x) % vsz != 0 || reinterpret_cast<uintptr_t>(y) % vsz != 0)
        return LSCAN_ERR_INVALID;
    const size_t vb = static_cast<size_t>(n) * vsz;
    // y is written out of step with the reads: no overlap at all
    const auto overlap = [](const void *a, size_t an, const void *b, size_t bn) {
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
        return a0 < b0 + bn && b0 < a0 + an;
    };
    if (overlap(y, vb, x, vb) || overlap(y, vb, flags, static_cast<size_t>(n)))
        return LSCAN_ERR_INVALID;
    LaunchSpec ls;
    ls.kind = vsz == 2 ? KIND_SEL16 : vsz == 4 ? KIND_SEL32 : KIND_SEL64;
    ls.mode = MODE_SINGLE;
    // flags by bulk copy when 16-byte aligned; the values too (staged in
    // the ring) when they are as well
    ls.variant = reinterpret_cast<uintptr_t>(flags) % 16 != 0 ? 0
                 : reinterpret_cast<uintptr_t>(x) % 16 == 0 && g_kernels[ls.kind][MODE_SINGLE][2].fn
                     ? 2
                     : 1;
    const KernelEntry &e = g_kernels[ls.kind][MODE_SINGLE][ls.variant];
    if (e.fn == nullptr) return LSCAN_ERR_UNSUPPORTED;
    const int64_t n_tiles = (n + e.tile - 1) / e.tile;
    if (n_tiles > (int64_t{1} << 31) - 1) return LSCAN_ERR_INVALID;
    ls.x = flags;
    ls.y = y;
    ls.n = n;
    ls.inclusive = true;
    ls.carry_mode = CARRY_LOOKBACK;
    ls.status_words = static_cast<size_t>(n_tiles) * e.car_words;
    ls.values = x;
    ls.count_out = reinterpret_cast<unsigned long long *>(d_count);
    return run_planned(ls, stream);
}

lscan_status lscan_config_info(int32_t config, lscan_dtype dtype, int32_t *items,
                               int32_t *threads, int32_t *stages, int32_t *tile) {
    std::call_once(g_reg_once, register_all_kernels);
    if (config < 0 || config > kNumTmaCfg) return LSCAN_ERR_INVALID;
    int kind = dtype == LSCAN_I32 ? KIND_I32_ADD
               : dtype == LSCAN_F32 ? KIND_F32_MAX
               : dtype == LSCAN_BF16 ? KIND_BF16_MAX
               : dtype == LSCAN_I64 ? KIND_I64_ADD
               : dtype == LSCAN_F64 ? KIND_F64_MAX : -1;
    if (kind < 0) return LSCAN_ERR_INVALID;
    const KernelEntry &e = g_kernels[kind][MODE_SINGLE][config];
    if (items) *items = e.items;
    if (threads) *threads = e.cwarps * 32;
    if (stages) *stages = e.stages;
    if (tile) *tile = e.tile;
    return LSCAN_OK;
}

}  // extern "C"
