// lscan_tune.cu -- tile-configuration table and the autotuner that fills it.
//
// Entries are (kind, mode, log2 size class) -> configuration number (1..17
// for single arrays, 1..6 for batched scans; kernel_inst.cuh lists them).
// The defaults are each kind's fastest configuration on a 2^28-element
// array measured on GB300 (for batched modes, the fastest of the first six).
// lscan_autotune times every configuration built for the mode on the
// caller's buffers with CUDA events (median of `reps` timed launches after
// two warm-up launches) and records the fastest; the table persists as JSON
// ({"lscan_tune": 1, "entries": [[kind, mode, size_class, config, carry],
// ...]}, carry an lscan_carry; 4-field entries mean carry 0 = auto) and
// is loaded at start-up from $LSCAN_TUNE_FILE when that is set.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lscan.h"
#include "kernel_table.h"
#include "kinds.cuh"
#include "lscan_internal.h"

namespace lscan {

namespace {
constexpr int kSizeClasses = 40;  // log2(n) buckets
int g_table[kNumKinds][MODE_COUNT][kSizeClasses];
std::once_flag g_tab_once;
std::mutex g_tab_mu;

lscan_status load_file(const char *path);

// Fastest configuration per kind on GB300 (GB/s in the comments), single
// arrays and (first six configurations) batched scans.  Measured at 2^28
// with full tiles moved as swizzled tensor copies, and at 2^22 .. 2^26 for
// the kinds whose best depends on the size: 4- and 8-byte kinds take
// configuration 8 (32 KiB tiles of 32 items x 8 warps, 64-byte status
// slots) from 2^22 up, the compensated fp32 add 64 KiB tiles (12) from 2^25;
// bf16 takes 48, 56, 32 or 16 KiB tiles (17, 12, 11, 13) from 2^25 up,
// 3-stage 32 KiB tiles (11) from 2^23 and smaller ones below.
int default_variant(int kind, int mode, int size_cls = 28) {
    const bool single = mode == MODE_SINGLE;
    switch (kind) {
        case KIND_I32_ADD: return single ? 8 : 6;      // 6162 (2^28), 5634 (2^26)
        case KIND_I32_MAX: return single ? 8 : 6;      // 6183, 5634
        case KIND_F32_MAX: return single ? 8 : 5;      // 6261, 5541
        case KIND_BF16_MAX:  // 5354 (2^28)
            return single ? (size_cls >= 25 ? 17 : size_cls >= 23 ? 11 : 5) : 5;
        case KIND_F32_ADD_PLAIN: return single ? 8 : 6;  // 6214
        case KIND_F32_ADD_F64: return single ? 12 : 5;   // 5780
        case KIND_F32_ADD_DF: return single ? 8 : 5;     // 5960, 5327
        case KIND_F32_ADD_COMP: return single ? (size_cls >= 25 ? 12 : 8) : 3;  // 5243, 4804
        case KIND_BF16_ADD_PLAIN_F32: return single ? 13 : 4;  // 6172
        case KIND_BF16_ADD_F64_F32: return single ? (size_cls >= 25 ? 12 : 7) : 5;  // 5789
        case KIND_BF16_ADD_DF_F32:  // 5835
            return single ? (size_cls >= 25 ? 12 : size_cls >= 23 ? 11 : 13) : 2;
        case KIND_BF16_ADD_COMP_F32: return single ? (size_cls >= 25 ? 11 : 13) : 4;  // 4007
        case KIND_BF16_ADD_PLAIN_BF16: return single ? (size_cls >= 25 ? 12 : 13) : 4;  // 4820
        case KIND_BF16_ADD_F64_BF16: return single ? (size_cls >= 25 ? 17 : 11) : 5;  // 4541
        case KIND_BF16_ADD_DF_BF16: return single ? (size_cls >= 25 ? 12 : 11) : 5;  // 4555
        case KIND_BF16_ADD_COMP_BF16: return single ? (size_cls >= 25 ? 11 : 13) : 4;  // 2831
        case KIND_I64_ADD: return single ? 8 : 5;      // 5883, 5625
        case KIND_I64_MAX: return single ? 8 : 5;      // 5651
        case KIND_F64_MAX: return single ? 8 : 4;      // 3414
        case KIND_F64_ADD: return single ? 10 : 4;     // 2038
        default: return 2;
    }
}

// a configuration number that is built for (kind, mode)
bool variant_built(int kind, int mode, int v) {
    return v >= 1 && v <= kNumTmaCfg && g_kernels[kind][mode][v].fn != nullptr;
}

void fill_defaults(int (&t)[kNumKinds][MODE_COUNT][kSizeClasses]) {
    for (int k = 0; k < kNumKinds; ++k)
        for (int m = 0; m < MODE_COUNT; ++m)
            for (int c = 0; c < kSizeClasses; ++c) t[k][m][c] = default_variant(k, m, c);
}

void init_table() {
    ensure_kernels_registered();
    fill_defaults(g_table);
    if (const char *f = std::getenv("LSCAN_TUNE_FILE")) (void)load_file(f);
}

int size_class(int64_t n) {
    int c = 0;
    while (c + 1 < kSizeClasses && (int64_t{1} << (c + 1)) <= n) ++c;
    return c;
}
}  // namespace

// A table entry is config | carry << 8 (carry: an lscan_carry, 0 = auto).
int tuned_variant(int kind, int mode, int64_t n, int *carry) {
    std::call_once(g_tab_once, init_table);
    std::lock_guard<std::mutex> lk(g_tab_mu);
    const int e = g_table[kind][mode][size_class(n)];
    if (carry) *carry = e >> 8;
    const int v = e & 0xff;
    return variant_built(kind, mode, v) ? v : default_variant(kind, mode, size_class(n));
}

void set_tuned_variant(int kind, int mode, int size_cls, int entry) {
    std::call_once(g_tab_once, init_table);
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (kind < 0 || kind >= kNumKinds || mode < 0 || mode >= MODE_COUNT) return;
    if (size_cls < 0 || size_cls >= kSizeClasses) return;
    if (!variant_built(kind, mode, entry & 0xff)) return;
    g_table[kind][mode][size_cls] = entry;
}

}  // namespace lscan

using namespace lscan;

extern "C" {

lscan_status lscan_autotune(lscan_op op, lscan_dtype dtype, int inclusive, const void *x,
                            void *y, int64_t n, const int64_t *d_offsets, int64_t n_seg,
                            const lscan_options *opts, int reps, void *stream,
                            lscan_tune_result *out) {
    if (n <= 0 || reps < 1 || reps > 1000) return LSCAN_ERR_INVALID;
    ensure_kernels_registered();
    const int mode = d_offsets ? MODE_SEGMENTED : MODE_SINGLE;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    lscan_options o{};
    if (opts) o = *opts;
    // reps + 1 events: the interval between consecutive events is one launch
    std::vector<cudaEvent_t> ev(static_cast<size_t>(reps) + 1, nullptr);
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            for (auto &d : ev)
                if (d) cudaEventDestroy(d);
            return LSCAN_ERR_CUDA;
        }
    // median launch time of plan ls (after two untimed launches), in ms
    std::vector<float> t(static_cast<size_t>(reps));
    auto time_plan = [&](const LaunchSpec &ls, float *ms) -> lscan_status {
        lscan_status st = LSCAN_OK;
        for (int w = 0; w < 2 && st == LSCAN_OK; ++w) st = run_planned(ls, stream);
        if (st == LSCAN_OK && cudaEventRecord(ev[0], cs) != cudaSuccess) st = LSCAN_ERR_CUDA;
        for (int r = 0; r < reps && st == LSCAN_OK; ++r) {
            st = run_planned(ls, stream);
            if (st == LSCAN_OK && cudaEventRecord(ev[r + 1], cs) != cudaSuccess)
                st = LSCAN_ERR_CUDA;
        }
        if (st != LSCAN_OK) return st;
        if (cudaEventSynchronize(ev[reps]) != cudaSuccess) return LSCAN_ERR_CUDA;
        for (int r = 0; r < reps; ++r) cudaEventElapsedTime(&t[r], ev[r], ev[r + 1]);
        std::sort(t.begin(), t.end());
        *ms = reps % 2 ? t[reps / 2] : 0.5f * (t[reps / 2 - 1] + t[reps / 2]);
        return LSCAN_OK;
    };
    lscan_tune_result res{};
    int best = 0, kind = -1;
    LaunchSpec best_ls;
    lscan_status result = LSCAN_OK;
    o.carry = LSCAN_CARRY_LOOKBACK;
    for (int c = 1; c <= kNumTmaCfg; ++c) {
        o.config = c;
        LaunchSpec ls;
        lscan_status st = plan_scan(op, dtype, inclusive, x, y, n, &o, mode, d_offsets,
                                    n_seg, &ls);
        if (st == LSCAN_ERR_UNSUPPORTED) continue;  // not built for this mode
        if (st != LSCAN_OK) {
            result = st;
            break;
        }
        if (ls.variant != c) break;  // unaligned buffers: nothing to tune
        kind = ls.kind;
        float ms = 0.f;
        st = time_plan(ls, &ms);
        if (st != LSCAN_OK) {
            result = st;
            break;
        }
        if (c - 1 < LSCAN_TUNE_MAX_CONFIGS) res.ms_by_config[c - 1] = ms;
        ++res.n_timed;
        if (best == 0 || ms < res.ms) {
            best = c;
            res.ms = ms;
            best_ls = ls;
        }
    }
    // the paper's chained hand-off at the fastest configuration; it costs one
    // L2 round trip per tile in series (~0.5 us), so it is timed only where
    // that can compete: arrays of at most 4096 tiles
    int best_carry = LSCAN_CARRY_LOOKBACK;
    if (result == LSCAN_OK && best > 0 && planned_tiles(best_ls) <= 4096) {
        LaunchSpec ls = best_ls;
        ls.carry_mode = CARRY_CHAINED;
        float ms = 0.f;
        result = time_plan(ls, &ms);
        res.chained_ms = ms;
        if (result == LSCAN_OK && ms < res.ms) {
            res.ms = ms;
            best_carry = LSCAN_CARRY_CHAINED;
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (result != LSCAN_OK) return result;
    if (best == 0) return LSCAN_ERR_UNSUPPORTED;
    res.config = best;
    res.carry = best_carry;
    res.default_config = default_variant(kind, mode, size_class(n));
    if (res.default_config >= 1 && res.default_config <= LSCAN_TUNE_MAX_CONFIGS)
        res.default_ms = res.ms_by_config[res.default_config - 1];
    // the look-back is what AUTO means already: record only a chained win
    const int carry_entry = best_carry == LSCAN_CARRY_CHAINED ? LSCAN_CARRY_CHAINED : 0;
    set_tuned_variant(kind, mode, size_class(n), best | (carry_entry << 8));
    if (out) *out = res;
    return LSCAN_OK;
}

lscan_status lscan_tune_save(const char *path) {
    if (!path) return LSCAN_ERR_INVALID;
    std::call_once(g_tab_once, init_table);
    std::lock_guard<std::mutex> lk(g_tab_mu);
    FILE *f = std::fopen(path, "w");
    if (!f) return LSCAN_ERR_INVALID;
    std::fprintf(f, "{\"lscan_tune\": 1, \"entries\": [");
    bool first = true;
    for (int k = 0; k < kNumKinds; ++k)
        for (int m = 0; m < MODE_COUNT; ++m)
            for (int c = 0; c < kSizeClasses; ++c)
                if (g_table[k][m][c] != default_variant(k, m, c)) {
                    std::fprintf(f, "%s[%d, %d, %d, %d, %d]", first ? "" : ", ", k, m, c,
                                 g_table[k][m][c] & 0xff, g_table[k][m][c] >> 8);
                    first = false;
                }
    std::fprintf(f, "]}\n");
    std::fclose(f);
    return LSCAN_OK;
}

lscan_status lscan_tune_load(const char *path) {
    ensure_kernels_registered();
    std::call_once(g_tab_once, init_table);
    return load_file(path);
}

lscan_status lscan_tune_reset(void) {
    std::call_once(g_tab_once, init_table);
    std::lock_guard<std::mutex> lk(g_tab_mu);
    fill_defaults(g_table);
    return LSCAN_OK;
}

}  // extern "C"

namespace lscan {
namespace {
lscan_status load_file(const char *path) {
    if (!path) return LSCAN_ERR_INVALID;
    FILE *f = std::fopen(path, "r");
    if (!f) return LSCAN_ERR_INVALID;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    const size_t at = text.find("\"entries\"");
    if (text.find("\"lscan_tune\"") == std::string::npos || at == std::string::npos)
        return LSCAN_ERR_INVALID;
    // every "[a, b, c, d]" after "entries" is one entry
    size_t pos = text.find('[', at);
    if (pos == std::string::npos) return LSCAN_ERR_INVALID;
    ++pos;
    int loaded[kNumKinds][MODE_COUNT][kSizeClasses];
    fill_defaults(loaded);
    while (true) {
        const size_t open = text.find('[', pos);
        if (open == std::string::npos) break;
        int k, m, c, v, carry = 0;
        const int got_n = std::sscanf(text.c_str() + open, "[%d , %d , %d , %d , %d ]", &k,
                                      &m, &c, &v, &carry);
        if (got_n == 4) {
            carry = 0;
        } else if (got_n != 5) {
            return LSCAN_ERR_INVALID;
        }
        if (carry < LSCAN_CARRY_AUTO || carry > LSCAN_CARRY_CHAINED) return LSCAN_ERR_INVALID;
        if (k < 0 || k >= kNumKinds || m < 0 || m >= MODE_COUNT || c < 0 ||
            c >= kSizeClasses || v < 1 || v > kNumTmaCfg)
            return LSCAN_ERR_INVALID;
        if (!variant_built(k, m, v)) return LSCAN_ERR_INVALID;
        loaded[k][m][c] = v | (carry << 8);
        pos = open + 1;
    }
    {
        // init_table may be the caller (first use): g_tab_mu is not held here
        std::lock_guard<std::mutex> lk(g_tab_mu);
        for (int k = 0; k < kNumKinds; ++k)
            for (int m = 0; m < MODE_COUNT; ++m)
                for (int c = 0; c < kSizeClasses; ++c) g_table[k][m][c] = loaded[k][m][c];
    }
    return LSCAN_OK;
}
}  // namespace
}  // namespace lscan
