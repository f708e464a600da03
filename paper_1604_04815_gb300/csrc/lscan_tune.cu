// lscan_tune.cu -- tile-configuration table used when lscan_options.config
// is 0.  Entries are (kind, mode, log2 size class) -> variant; the default is
// variant 2 (16 KiB input tiles, 8 consumer warps, 4-stage ring).
#include <cstdint>
#include <mutex>

#include "kernel_table.h"
#include "lscan_internal.h"

namespace lscan {

namespace {
constexpr int kSizeClasses = 40;  // log2(n) buckets
int g_table[kNumKinds][MODE_COUNT][kSizeClasses];
std::once_flag g_tab_once;
std::mutex g_tab_mu;

void init_table() {
    for (auto &a : g_table)
        for (auto &b : a)
            for (int &v : b) v = 2;
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
    return (v >= 1 && v <= kNumTmaCfg) ? v : 2;
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
