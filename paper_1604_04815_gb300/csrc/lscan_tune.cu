// lscan_tune.cu -- tile-configuration table and the autotuner that fills it.
//
// Entries are (kind, mode, log2 size class) -> variant (1..kNumTmaCfg).  The
// default is each kind's fastest variant on a 2^28-element array (GB300,
// 16-segment batches agree): variant 2 (16 KiB input tiles, 8 consumer warps)
// for most kinds, variant 3 (32 KiB tiles, 16 consumer warps) for fp32 add
// with an FP64 carry (5478 vs 4454 GB/s) and for bf16 add with an FP64 carry
// and bf16 output, variant 1 for the compensated bf16 adds.
// lscan_autotune times every bulk-copy configuration on the caller's buffers
// with CUDA events and records the fastest; the table persists as JSON
// ({"lscan_tune": 1, "entries": [[kind, mode, size_class, config], ...]}) and
// is loaded at start-up from $LSCAN_TUNE_FILE when that is set.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>

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

int default_variant(int kind) {
    switch (kind) {
        case KIND_F32_ADD_F64:
        case KIND_BF16_ADD_F64_BF16:
            return 3;
        case KIND_BF16_ADD_COMP_F32:
        case KIND_BF16_ADD_COMP_BF16:
            return 1;
        default:
            return 2;
    }
}

void fill_defaults(int (&t)[kNumKinds][MODE_COUNT][kSizeClasses]) {
    for (int k = 0; k < kNumKinds; ++k)
        for (auto &b : t[k])
            for (int &v : b) v = default_variant(k);
}

void init_table() {
    fill_defaults(g_table);
    if (const char *f = std::getenv("LSCAN_TUNE_FILE")) (void)load_file(f);
}

int size_class(int64_t n) {
    int c = 0;
    while (c + 1 < kSizeClasses && (int64_t{1} << (c + 1)) <= n) ++c;
    return c;
}
}  // namespace

int tuned_variant(int kind, int mode, int64_t n) {
    std::call_once(g_tab_once, init_table);
    std::lock_guard<std::mutex> lk(g_tab_mu);
    const int v = g_table[kind][mode][size_class(n)];
    return (v >= 1 && v <= kNumTmaCfg) ? v : default_variant(kind);
}

void set_tuned_variant(int kind, int mode, int size_cls, int variant) {
    std::call_once(g_tab_once, init_table);
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (kind < 0 || kind >= kNumKinds || mode < 0 || mode >= MODE_COUNT) return;
    if (size_cls < 0 || size_cls >= kSizeClasses) return;
    if (variant < 1 || variant > kNumTmaCfg) return;
    g_table[kind][mode][size_cls] = variant;
}

}  // namespace lscan

using namespace lscan;

extern "C" {

lscan_status lscan_autotune(lscan_op op, lscan_dtype dtype, int inclusive, const void *x,
                            void *y, int64_t n, const int64_t *d_offsets, int64_t n_seg,
                            const lscan_options *opts, int reps, void *stream,
                            int32_t *best_config, float *best_ms) {
    if (n <= 0 || reps < 1 || reps > 1000) return LSCAN_ERR_INVALID;
    const int mode = d_offsets ? MODE_SEGMENTED : MODE_SINGLE;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    lscan_options o{};
    if (opts) o = *opts;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LSCAN_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LSCAN_ERR_CUDA;
    }
    int best = 0, kind = -1;
    float best_t = 0.f;
    lscan_status result = LSCAN_OK;
    for (int c = 1; c <= kNumTmaCfg; ++c) {
        o.config = c;
        LaunchSpec ls;
        lscan_status st = plan_scan(op, dtype, inclusive, x, y, n, &o, mode, d_offsets,
                                    n_seg, &ls);
        if (st != LSCAN_OK) {
            result = st;
            break;
        }
        if (ls.variant != c) break;  // unaligned buffers: nothing to tune
        kind = ls.kind;
        for (int w = 0; w < 2 && st == LSCAN_OK; ++w) st = run_planned(ls, stream);
        cudaEventRecord(e0, cs);
        for (int r = 0; r < reps && st == LSCAN_OK; ++r) st = run_planned(ls, stream);
        cudaEventRecord(e1, cs);
        if (st != LSCAN_OK || cudaEventSynchronize(e1) != cudaSuccess) {
            result = st != LSCAN_OK ? st : LSCAN_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (best == 0 || ms < best_t) {
            best = c;
            best_t = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != LSCAN_OK) return result;
    if (best == 0) return LSCAN_ERR_UNSUPPORTED;
    set_tuned_variant(kind, mode, size_class(n), best);
    if (best_config) *best_config = best;
    if (best_ms) *best_ms = best_t;
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
                if (g_table[k][m][c] != default_variant(k)) {
                    std::fprintf(f, "%s[%d, %d, %d, %d]", first ? "" : ", ", k, m, c,
                                 g_table[k][m][c]);
                    first = false;
                }
    std::fprintf(f, "]}\n");
    std::fclose(f);
    return LSCAN_OK;
}

lscan_status lscan_tune_load(const char *path) {
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
        int k, m, c, v;
        if (std::sscanf(text.c_str() + open, "[%d , %d , %d , %d ]", &k, &m, &c, &v) != 4)
            return LSCAN_ERR_INVALID;
        if (k < 0 || k >= kNumKinds || m < 0 || m >= MODE_COUNT || c < 0 ||
            c >= kSizeClasses || v < 1 || v > kNumTmaCfg)
            return LSCAN_ERR_INVALID;
        loaded[k][m][c] = v;
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
