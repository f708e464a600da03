// kernel_inst.cuh -- explicit instantiation of the scan kernel for one kind.
#pragma once
#include <utility>

#include "kernel_table.h"
#include "reduce_kernel.cuh"
#include "scan_kernel.cuh"
#include "tiny_kernel.cuh"

namespace lscan {

// Tile configurations by input element size, the autotuner's search space.
// TileCfg<items/thread, consumer warps, ring stages, output staging buffers,
// CTAs per SM the registers must fit, carry warps, tiles per ticket (run),
// status words per tile slot (0: 2 for a one-word carry, more for wide
// carries with 32 KiB tiles)>.
//  - G loads straight from global memory (pointers not 16-byte aligned).
//  - List: the bulk-copy configurations 1..N of a single-array scan; the
//    first kMultiCfg are also built for batched (segmented, list) scans.
//    Every list names input tiles of 8, 16, 32, 48 or 64 KiB: ITEMS scales
//    inversely with the element size, so a configuration number means the
//    same bytes per tile for every type (bf16 entry 12 excepted, below).
// A kind whose shared memory does not fit one CTA with a configuration's
// slots takes fewer of them (fill_entry); one that does not fit with two is
// skipped when the table is filled (its entry stays empty).
template <class... Cs>
struct CfgList {};

template <int ISZ>
struct Cfgs;
template <>
struct Cfgs<4> {
    using G = TileCfg<8, 8, 4, 1, 3>;
    using List = CfgList<
        TileCfg<8, 8, 4, 1, 3>,             //  1: 8 KiB tiles, 4 stages
        TileCfg<16, 8, 3, 1, 3>,            //  2: 16 KiB, 3 stages
        TileCfg<16, 16, 2, 1, 2>,           //  3: 32 KiB, 2 stages, 16 warps
        TileCfg<16, 8, 3, 1, 3, 1, 1, 4>,   //  4: = 2, 32-byte status slots
        TileCfg<16, 16, 2, 1, 2, 1, 1, 8>,  //  5: = 3, 64-byte slots
        TileCfg<16, 16, 2, 1, 2, 1, 1, 16>, //  6: = 3, 128-byte slots
        TileCfg<16, 8, 3, 1, 3, 1, 2, 4>,   //  7: = 4, runs of 2 tiles
        TileCfg<32, 8, 2, 1, 2, 1, 1, 8>,   //  8: 32 KiB, 8 warps, 2 stages
        TileCfg<16, 4, 4, 1, 4, 1, 1, 4>,   //  9: 8 KiB, 4 warps, 4 stages
        TileCfg<32, 4, 3, 1, 3, 1, 1, 4>,   // 10: 16 KiB, 4 warps, 3 stages
        TileCfg<16, 16, 3, 1, 1, 1, 1, 8>,  // 11: 32 KiB, 3 stages (1 CTA/SM)
        TileCfg<32, 16, 2, 1, 1, 1, 1, 8>,  // 12: 64 KiB tiles
        TileCfg<16, 8, 4, 1, 2, 1, 1, 4>,   // 13: 16 KiB, 4 stages
        TileCfg<16, 16, 2, 1, 2, 1, 2, 8>,  // 14: = 5, runs of 2 tiles
        TileCfg<32, 8, 3, 1, 1, 1, 1, 8>,   // 15: 32 KiB, 8 warps, 3 stages
        TileCfg<8, 16, 3, 1, 2, 1, 1, 4>,   // 16: 16 KiB, 16 warps, 3 stages
        TileCfg<32, 12, 3, 1, 1, 1, 1, 8>>; // 17: 48 KiB, 12 warps, 3 stages
};
template <>
struct Cfgs<8> {
    using G = TileCfg<4, 8, 4, 1, 3>;
    using List = CfgList<
        TileCfg<4, 8, 4, 1, 3>,
        TileCfg<8, 8, 3, 1, 3>,
        TileCfg<8, 16, 2, 1, 2>,
        TileCfg<8, 8, 3, 1, 3, 1, 1, 4>,
        TileCfg<8, 16, 2, 1, 2, 1, 1, 8>,
        TileCfg<8, 16, 2, 1, 2, 1, 1, 16>,
        TileCfg<8, 8, 3, 1, 3, 1, 2, 4>,
        TileCfg<16, 8, 2, 1, 2, 1, 1, 8>,
        TileCfg<8, 4, 4, 1, 4, 1, 1, 4>,
        TileCfg<16, 4, 3, 1, 3, 1, 1, 4>,
        TileCfg<8, 16, 3, 1, 1, 1, 1, 8>,
        TileCfg<16, 16, 2, 1, 1, 1, 1, 8>,
        TileCfg<8, 8, 4, 1, 2, 1, 1, 4>,
        TileCfg<8, 16, 2, 1, 2, 1, 2, 8>,
        TileCfg<16, 8, 3, 1, 1, 1, 1, 8>,
        TileCfg<4, 16, 3, 1, 2, 1, 1, 4>,
        TileCfg<16, 12, 3, 1, 1, 1, 1, 8>>;
};
// bf16: twice the items for the same bytes.  Items stay <= 32 (a thread's
// segment-head bits fit one word), so where the 4-byte entry has 32 items
// the bf16 entry doubles the warps instead, or (entries 8, 10, 15) takes
// the same tile bytes with another slot width or run; entry 12 (64 KiB of
// 4-byte input) is 56 KiB of bf16, the largest tile whose 28 consumer warps
// and 3 service warps fit one 1024-thread CTA.
template <>
struct Cfgs<2> {
    using G = TileCfg<16, 8, 4, 1, 3>;
    using List = CfgList<
        TileCfg<16, 8, 4, 1, 3>,              //  1: 8 KiB
        TileCfg<32, 8, 3, 1, 2>,              //  2: 16 KiB
        TileCfg<32, 16, 2, 1, 1>,             //  3: 32 KiB
        TileCfg<32, 8, 3, 1, 2, 1, 1, 4>,     //  4: 16 KiB, 32-byte slots
        TileCfg<32, 16, 2, 1, 1, 1, 1, 8>,    //  5: 32 KiB, 64-byte slots
        TileCfg<32, 16, 2, 1, 1, 1, 1, 16>,   //  6: 32 KiB, 128-byte slots
        TileCfg<32, 8, 3, 1, 2, 1, 2, 4>,     //  7: 16 KiB, runs of 2
        TileCfg<32, 16, 2, 1, 1, 1, 2, 16>,   //  8: 32 KiB, runs of 2
        TileCfg<32, 4, 4, 1, 4, 1, 1, 4>,     //  9: 8 KiB, 4 warps
        TileCfg<32, 8, 3, 1, 2, 1, 1, 8>,     // 10: 16 KiB, 64-byte slots
        TileCfg<32, 16, 3, 1, 1, 1, 1, 8>,    // 11: 32 KiB, 3 stages
        TileCfg<32, 28, 2, 1, 1, 1, 1, 8>,    // 12: 56 KiB, 28 warps
        TileCfg<32, 8, 4, 1, 2, 1, 1, 4>,     // 13: 16 KiB, 4 stages
        TileCfg<32, 16, 2, 1, 1, 1, 2, 8>,    // 14: 32 KiB, runs of 2
        TileCfg<32, 16, 3, 1, 1, 1, 1, 16>,   // 15: 32 KiB, 3 stages, 128 B
        TileCfg<16, 16, 3, 1, 2, 1, 1, 4>,    // 16: 16 KiB, 16 warps
        TileCfg<32, 24, 3, 1, 1, 1, 1, 8>>;   // 17: 48 KiB, 24 warps, 3 stages
};
// flags of a stream compaction: 4096 flags per tile, 16 per thread, whose
// values are loaded early and held in registers (2 CTAs/SM leave room for
// them; a 6-stage ring keeps 12 tiles per SM in flight); one output buffer
// in which each tile's kept values are compacted before a coalesced copy
template <>
struct Cfgs<1> {
    using G = TileCfg<16, 8, 6, 1, 2>;
    using C1 = TileCfg<16, 8, 6, 1, 2>;
};
// stream compaction with its values staged in the ring beside the flags:
// 16384-element tiles (a quarter of the carry hops of 4096-element tiles),
// 2 slots, 64-byte status slots, one CTA per SM (2- and 4-byte values: 80
// KiB per slot for 4-byte values plus the 64 KiB output tile); 8-byte values
// take 8192-element tiles to fit
template <int VSZ>
struct SelStagedCfg {
    using C = TileCfg<32, 16, 2, 1, 1, 1, 1, 8>;
};
template <>
struct SelStagedCfg<8> {
    using C = TileCfg<16, 16, 2, 1, 1, 1, 1, 8>;
};

// shared memory one CTA may use (sm_100 family: 227 KiB)
constexpr int kMaxSmemPerCta = 227 * 1024;

// the configuration with S tile slots instead of Cfg's
template <class Cfg, int S>
using WithStages = TileCfg<Cfg::ITEMS, Cfg::CWARPS, S, Cfg::OSTAGES, Cfg::MINB, Cfg::NCARRY,
                           Cfg::RUN, Cfg::SLOTW>;

// A configuration names the tile; where a kind's shared memory (wider
// output staging, e.g. bf16 in, fp32 out) does not fit one CTA with Cfg's
// tile slots, the entry takes one slot fewer, down to two.
template <class K, class Cfg, int MODE, bool TMA>
void fill_entry(int kind, int variant) {
    using L = Layout<K, Cfg, MODE, TMA>;
    if constexpr (L::bytes > kMaxSmemPerCta) {
        if constexpr (Cfg::STAGES > 2 && (Cfg::STAGES - 1) % Cfg::NCARRY == 0)
            fill_entry<K, WithStages<Cfg, Cfg::STAGES - 1>, MODE, TMA>(kind, variant);
    } else {
        KernelEntry &e = g_kernels[kind][MODE][variant];
        e.fn = reinterpret_cast<const void *>(&lscan_kernel<K, Cfg, MODE, TMA>);
        e.threads = kernel_threads<K, Cfg, MODE, TMA>();
        e.smem = L::bytes;
        e.tile = Cfg::TILE;
        e.items = Cfg::ITEMS;
        e.cwarps = Cfg::CWARPS;
        e.stages = Cfg::STAGES;
        e.run = Cfg::RUN;
        static_assert(status_slot_words<K, Cfg>() <= kMaxSlotWords, "status slot");
        e.car_words = status_slot_words<K, Cfg>();  // status words per tile
        e.in_size = int(sizeof(typename K::In));
        e.out_size = int(sizeof(typename K::Out));
        using S = Swz<K, Cfg, MODE, TMA>;
        e.swz_in = S::IN ? S::RBI : 0;
        e.swz_out = S::OUT ? S::RBO : 0;
    }
}

// configuration number V of a mode: batched modes take the first kMultiCfg
// (the others are not instantiated for them)
template <class K, class Cfg, int MODE, int V>
void fill_numbered(int kind) {
    if constexpr (MODE == MODE_SINGLE || V <= kMultiCfg)
        fill_entry<K, Cfg, MODE, true>(kind, V);
}

template <class K, int MODE, class... Cs, size_t... I>
void fill_list(int kind, CfgList<Cs...>, std::index_sequence<I...>) {
    static_assert(sizeof...(Cs) == kNumTmaCfg, "one entry per configuration number");
    (fill_numbered<K, Cs, MODE, int(I) + 1>(kind), ...);
}

template <class K, int MODE>
void fill_mode(int kind) {
    using C = Cfgs<int(sizeof(typename K::In))>;
    fill_entry<K, typename C::G, MODE, false>(kind, 0);
    fill_list<K, MODE>(kind, typename C::List{}, std::make_index_sequence<kNumTmaCfg>{});
}

// stream compaction: single arrays only, plain-load and one bulk-copy variant
template <class K>
void fill_select(int kind) {
    using C = Cfgs<1>;
    fill_entry<K, typename C::G, MODE_SINGLE, false>(kind, 0);
    fill_entry<K, typename C::C1, MODE_SINGLE, true>(kind, 1);
    using V = typename K::Out;
    fill_entry<KSelectStaged<V>, typename SelStagedCfg<int(sizeof(V))>::C, MODE_SINGLE, true>(kind,
                                                                                           2);
}

template <class K>
void fill_kind(int kind) {
    g_tiny_kernels[kind] = reinterpret_cast<const void *>(&lscan_tiny_kernel<K>);
    g_reduce_kernels[kind] = reinterpret_cast<const void *>(&lscan_reduce_kernel<K>);
    g_carry_bytes[kind] = int(sizeof(typename K::Car));
    fill_mode<K, MODE_SINGLE>(kind);
    fill_mode<K, MODE_SEGMENTED>(kind);
    fill_mode<K, MODE_LIST>(kind);
}

}  // namespace lscan
