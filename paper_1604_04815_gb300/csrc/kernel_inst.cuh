// kernel_inst.cuh -- explicit instantiation of the scan kernel for one kind.
#pragma once
#include "kernel_table.h"
#include "scan_kernel.cuh"
#include "tiny_kernel.cuh"

namespace lscan {

// Tile configurations by input element size: <items/thread, consumer warps,
// ring stages, output staging buffers, CTAs per SM the registers must fit>.
// Variant 0 (G) loads straight from global memory; C1..C3 stream 8, 16 and
// 32 KiB input tiles through the bulk-copy ring (for every element size).
template <int ISZ>
struct Cfgs;
template <>
struct Cfgs<4> {
    using G = TileCfg<8, 8, 4, 1, 3>;
    using C1 = TileCfg<8, 8, 4, 1, 3>;
    using C2 = TileCfg<16, 8, 3, 1, 3>;
    using C3 = TileCfg<16, 16, 2, 1, 2>;
};
template <>
struct Cfgs<8> {
    using G = TileCfg<4, 8, 4, 1, 3>;
    using C1 = TileCfg<4, 8, 4, 1, 3>;
    using C2 = TileCfg<8, 8, 3, 1, 3>;
    using C3 = TileCfg<8, 16, 2, 1, 2>;
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
template <>
struct Cfgs<2> {
    using G = TileCfg<16, 8, 4, 1, 3>;
    using C1 = TileCfg<16, 8, 4, 1, 3>;
    using C2 = TileCfg<32, 8, 3, 1, 2>;
    using C3 = TileCfg<32, 16, 2, 1, 1>;
};

template <class K, class Cfg, int MODE, bool TMA>
void fill_entry(int kind, int variant) {
    using L = Layout<K, Cfg, MODE, TMA>;
    KernelEntry &e = g_kernels[kind][MODE][variant];
    e.fn = reinterpret_cast<const void *>(&lscan_kernel<K, Cfg, MODE, TMA>);
    e.threads = Cfg::THREADS;
    e.smem = L::bytes;
    e.tile = Cfg::TILE;
    e.items = Cfg::ITEMS;
    e.cwarps = Cfg::CWARPS;
    e.stages = Cfg::STAGES;
    static_assert(status_slot_words<K, Cfg::TILE>() <= kMaxSlotWords, "status slot");
    e.car_words = status_slot_words<K, Cfg::TILE>();  // status words per tile
    e.in_size = int(sizeof(typename K::In));
    e.out_size = int(sizeof(typename K::Out));
}

template <class K, int MODE>
void fill_mode(int kind) {
    using C = Cfgs<int(sizeof(typename K::In))>;
    fill_entry<K, typename C::G, MODE, false>(kind, 0);
    fill_entry<K, typename C::C1, MODE, true>(kind, 1);
    fill_entry<K, typename C::C2, MODE, true>(kind, 2);
    fill_entry<K, typename C::C3, MODE, true>(kind, 3);
}

// stream compaction: single arrays only, plain-load and one bulk-copy variant
template <class K>
void fill_select(int kind) {
    using C = Cfgs<1>;
    fill_entry<K, typename C::G, MODE_SINGLE, false>(kind, 0);
    fill_entry<K, typename C::C1, MODE_SINGLE, true>(kind, 1);
}

template <class K>
void fill_kind(int kind) {
    g_tiny_kernels[kind] = reinterpret_cast<const void *>(&lscan_tiny_kernel<K>);
    fill_mode<K, MODE_SINGLE>(kind);
    fill_mode<K, MODE_SEGMENTED>(kind);
    fill_mode<K, MODE_LIST>(kind);
}

}  // namespace lscan
