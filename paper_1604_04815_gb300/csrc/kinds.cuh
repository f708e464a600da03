// kinds.cuh -- operator / element-type traits of the scan kernels.
//
// A "kind" fixes: storage types In/Out, the in-tile accumulation type Acc,
// the inter-tile carry type Car (what the status words carry), and CarA, the
// form in which a tile applies its carry to its elements; car_of_out reads a
// caller's carry-in (one output element) as a carry.  The operator is
// always combined as op(earlier, later), so the code never relies on
// commutativity even though add and max are commutative (Section 1 only asks
// for associativity).
//
//   int32 add  : wrapping uint32 arithmetic (two's complement mod 2^32)
//   int32 max  : signed compare, identity INT32_MIN
//   fp32/bf16 max : b > a ? b : a  (a tie keeps the earlier element's bits),
//                identity -inf; bf16 widened exactly to fp32 and narrowed
//                back exactly
//   fp32/bf16 add, four precision paths for the carry chain:
//     Plain : fp32 in tile, fp32 carry
//     F64   : fp32 in tile, FP64 carry; the carry is split once per tile into
//             an fp32 (hi, lo) pair and applied with fp32 two-sum arithmetic,
//             so no per-element FP64 work is done
//     DF    : fp32 in tile, double-float carry: a normalised fp32 (hi, lo)
//             pair (48-bit significand) combined with two-sum arithmetic, so
//             the carry path has no FP64 instruction (GB300's FP64 pipe is
//             narrow and its latency sits on the carry chain)
//     Comp  : compensated in tile (each element enters through an exact
//             two-sum into an unnormalised (hi, lo) pair), double-float
//             carry, each output rounded from hi + lo
//
// Two-sum (Knuth, TAOCP vol. 2, 4.2.2) is written with __fadd_rn / __fsub_rn
// so the compiler cannot contract or reassociate it.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

namespace lscan {

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ float bf16_bits_to_f32(uint16_t b) {
    return __uint_as_float(static_cast<uint32_t>(b) << 16);
}
// exact when f came from a bf16 (low 16 bits zero)
__device__ __forceinline__ uint16_t f32_to_bf16_bits_exact(float f) {
    return static_cast<uint16_t>(__float_as_uint(f) >> 16);
}
__device__ __forceinline__ uint16_t f32_to_bf16_bits_rn(float f) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}
// Two fp32 values rounded to bf16 (to nearest, ties to even) and packed in
// one instruction: lo in bits 0..15, hi in bits 16..31.
__device__ __forceinline__ uint32_t f32x2_to_bf16x2_rn(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// s + e == a + b exactly (Knuth two-sum)
__device__ __forceinline__ float2 two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
// double-float addition (hi, lo) + (hi, lo), normalised result (hi the
// rounded sum, lo its exact remainder).  The only roundings are those of the
// low parts, so the absolute error is at most 2u (|s.y| + |a.y| + |b.y|):
// O(u^2 (|a| + |b|)) for normalised inputs.  It ends in a two-sum rather than
// Dekker's fast-two-sum, so inputs need not be normalised (the in-tile pairs
// of the compensated path are not).
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float2 s = two_sum(a.x, b.x);
    float e = __fadd_rn(s.y, __fadd_rn(a.y, b.y));
    return two_sum(s.x, e);
}
// FP64 value -> fp32 (hi, lo) with hi + lo == d to ~2^-48 |d|
__device__ __forceinline__ float2 split_f64(double d) {
    float h = __double2float_rn(d);
    float l = __double2float_rn(__dsub_rn(d, static_cast<double>(h)));
    return make_float2(h, l);
}

template <class T>
__device__ __forceinline__ T max_keep_left(T a, T b) {
    return (b > a) ? b : a;
}

// ----------------------------------------------------------------- kinds
struct KI32Add {
    static constexpr bool kTieOrdered = false;
    using In = int32_t;
    using Out = int32_t;
    using Acc = uint32_t;
    using Car = uint32_t;
    using CarA = uint32_t;
    __device__ static Acc ident() { return 0u; }
    __device__ static Acc load(In v) { return static_cast<uint32_t>(v); }
    __device__ static Acc op(Acc a, Acc b) { return a + b; }
    __device__ static Car cident() { return 0u; }
    __device__ static Car to_car(Acc a) { return a; }
    __device__ static Car cop(Car a, Car b) { return a + b; }
    __device__ static CarA to_apply(Car c) { return c; }
    __device__ static CarA base(CarA c, Acc tb) { return c + tb; }
    __device__ static CarA base_local(Acc tb) { return tb; }
    __device__ static Out fin(CarA b, Acc v) {
        return static_cast<int32_t>(b + v);
    }
    __device__ static Car car_of_out(Out o) { return static_cast<uint32_t>(o); }
};

struct KI32Max {
    static constexpr bool kTieOrdered = false;  // equal ints have equal bits
    using In = int32_t;
    using Out = int32_t;
    using Acc = int32_t;
    using Car = int32_t;
    using CarA = int32_t;
    __device__ static Acc ident() { return INT32_MIN; }
    __device__ static Acc load(In v) { return v; }
    __device__ static Acc op(Acc a, Acc b) { return max_keep_left(a, b); }
    __device__ static Car cident() { return INT32_MIN; }
    __device__ static Car to_car(Acc a) { return a; }
    __device__ static Car cop(Car a, Car b) { return max_keep_left(a, b); }
    __device__ static CarA to_apply(Car c) { return c; }
    __device__ static CarA base(CarA c, Acc tb) { return max_keep_left(c, tb); }
    __device__ static CarA base_local(Acc tb) { return tb; }
    __device__ static Out fin(CarA b, Acc v) { return max_keep_left(b, v); }
    __device__ static Car car_of_out(Out o) { return o; }
};

template <class InT>
struct FloatIn;
template <>
struct FloatIn<float> {
    __device__ static float load(float v) { return v; }
};
template <>
struct FloatIn<uint16_t> {
    __device__ static float load(uint16_t v) { return bf16_bits_to_f32(v); }
};

template <class OutT>
struct FloatOut;
template <>
struct FloatOut<float> {
    __device__ static float cvt(float v) { return v; }
    __device__ static float cvt_exact(float v) { return v; }
};
template <>
struct FloatOut<uint16_t> {
    __device__ static uint16_t cvt(float v) { return f32_to_bf16_bits_rn(v); }
    __device__ static uint16_t cvt_exact(float v) {
        return f32_to_bf16_bits_exact(v);
    }
};

// fp32 / bf16 max (InT = float or uint16_t bf16 bits; Out = In)
template <class InT>
struct KFMax {
    static constexpr bool kTieOrdered = true;  // +0 / -0 compare equal
    // a tile's maximum may be found on the raw bits (raw_float_max_tile)
    static constexpr bool kRawMax = true;
    // strict "greater" of the operator (tie-ordered folds; +0 == -0)
    __device__ static bool gt(float a, float b) { return a > b; }
    using In = InT;
    using Out = InT;
    using Acc = float;
    using Car = float;
    using CarA = float;
    __device__ static Acc ident() { return __uint_as_float(0xff800000u); }
    __device__ static Acc load(In v) { return FloatIn<InT>::load(v); }
    __device__ static Acc op(Acc a, Acc b) { return max_keep_left(a, b); }
    __device__ static Car cident() { return __uint_as_float(0xff800000u); }
    __device__ static Car to_car(Acc a) { return a; }
    __device__ static Car cop(Car a, Car b) { return max_keep_left(a, b); }
    __device__ static CarA to_apply(Car c) { return c; }
    __device__ static CarA base(CarA c, Acc tb) { return max_keep_left(c, tb); }
    __device__ static CarA base_local(Acc tb) { return tb; }
    __device__ static Out fin(CarA b, Acc v) {
        return FloatOut<InT>::cvt_exact(max_keep_left(b, v));
    }
    __device__ static Car car_of_out(Out o) { return FloatIn<InT>::load(o); }
};

// float add, plain fp32 carry
template <class InT, class OutT>
struct KFAddPlain {
    static constexpr bool kTieOrdered = false;
    using In = InT;
    using Out = OutT;
    using Acc = float;
    using Car = float;
    using CarA = float;
    __device__ static Acc ident() { return 0.0f; }
    __device__ static Acc load(In v) { return FloatIn<InT>::load(v); }
    __device__ static Acc op(Acc a, Acc b) { return __fadd_rn(a, b); }
    __device__ static Car cident() { return 0.0f; }
    __device__ static Car to_car(Acc a) { return a; }
    __device__ static Car cop(Car a, Car b) { return __fadd_rn(a, b); }
    __device__ static CarA to_apply(Car c) { return c; }
    __device__ static CarA base(CarA c, Acc tb) { return __fadd_rn(c, tb); }
    __device__ static CarA base_local(Acc tb) { return tb; }
    // the output before its rounding to Out (fp32)
    __device__ static float fin_f(CarA b, Acc v) { return __fadd_rn(b, v); }
    __device__ static Out fin(CarA b, Acc v) { return FloatOut<OutT>::cvt(fin_f(b, v)); }
    __device__ static Car car_of_out(Out o) { return FloatIn<OutT>::load(o); }
};

// float add, fp32 in tile, FP64 carry applied as an fp32 (hi, lo) pair
template <class InT, class OutT>
struct KFAddF64 {
    static constexpr bool kTieOrdered = false;
    using In = InT;
    using Out = OutT;
    using Acc = float;
    using Car = double;
    using CarA = float2;
    __device__ static Acc ident() { return 0.0f; }
    __device__ static Acc load(In v) { return FloatIn<InT>::load(v); }
    __device__ static Acc op(Acc a, Acc b) { return __fadd_rn(a, b); }
    __device__ static Car cident() { return 0.0; }
    __device__ static Car to_car(Acc a) { return static_cast<double>(a); }
    __device__ static Car cop(Car a, Car b) { return __dadd_rn(a, b); }
    __device__ static CarA to_apply(Car c) { return split_f64(c); }
    __device__ static CarA base(CarA c, Acc tb) {
        float2 s = two_sum(c.x, tb);
        return make_float2(s.x, __fadd_rn(s.y, c.y));
    }
    __device__ static CarA base_local(Acc tb) { return make_float2(tb, 0.0f); }
    __device__ static float fin_f(CarA b, Acc v) { return __fadd_rn(b.x, __fadd_rn(v, b.y)); }
    __device__ static Out fin(CarA b, Acc v) { return FloatOut<OutT>::cvt(fin_f(b, v)); }
    __device__ static Car car_of_out(Out o) {
        return static_cast<double>(FloatIn<OutT>::load(o));
    }
};

// float add, fp32 in tile, double-float carry: the carry chain runs on
// normalised fp32 (hi, lo) pairs (a 48-bit significand, FP64-class) with
// two-sum arithmetic, so no FP64 instruction is on the carry path
template <class InT, class OutT>
struct KFAddDF {
    static constexpr bool kTieOrdered = false;
    using In = InT;
    using Out = OutT;
    using Acc = float;
    using Car = float2;
    using CarA = float2;
    __device__ static Acc ident() { return 0.0f; }
    __device__ static Acc load(In v) { return FloatIn<InT>::load(v); }
    __device__ static Acc op(Acc a, Acc b) { return __fadd_rn(a, b); }
    __device__ static Car cident() { return make_float2(0.0f, 0.0f); }
    __device__ static Car to_car(Acc a) { return make_float2(a, 0.0f); }
    __device__ static Car cop(Car a, Car b) { return df_add(a, b); }
    __device__ static CarA to_apply(Car c) { return c; }
    __device__ static CarA base(CarA c, Acc tb) {
        float2 s = two_sum(c.x, tb);
        return make_float2(s.x, __fadd_rn(s.y, c.y));
    }
    __device__ static CarA base_local(Acc tb) { return make_float2(tb, 0.0f); }
    __device__ static float fin_f(CarA b, Acc v) { return __fadd_rn(b.x, __fadd_rn(v, b.y)); }
    __device__ static Out fin(CarA b, Acc v) { return FloatOut<OutT>::cvt(fin_f(b, v)); }
    __device__ static Car car_of_out(Out o) {
        return make_float2(FloatIn<OutT>::load(o), 0.0f);
    }
};

// float add, compensated in tile, double-float carry.
// Per element (op_step, b a fresh element (x, 0)): (s, e) = two-sum(hi, x),
// hi = s, lo += e -- hi + lo keeps every rounding error of the running sum;
// only the additions into lo round, O(K u^2 S) over K elements.  Pairs
// (thread totals, warp and tile totals, carries) combine with df_add.  The
// output y = fl(fl(b.hi + hi) + fl(b.lo + lo)) rounds twice, so
// |y_j - sum| <= 2u S_j + O(u^2 S_j), within the 2.5e-7 S_j (~4.2u) bound.
template <class InT, class OutT>
struct KFAddComp {
    static constexpr bool kTieOrdered = false;
    // several reducer warps fold a tile's parts where one CTA runs per SM
    // (a compensated fold per element is as much arithmetic as the
    // consumers' scan: one reducer warp on one SM sub-partition carries
    // twice the load of the others)
    static constexpr bool kSplitReduce = true;
    using In = InT;
    using Out = OutT;
    using Acc = float2;
    using Car = float2;
    using CarA = float2;
    __device__ static Acc ident() { return make_float2(0.0f, 0.0f); }
    __device__ static Acc load(In v) {
        return make_float2(FloatIn<InT>::load(v), 0.0f);
    }
    __device__ static Acc op(Acc a, Acc b) { return df_add(a, b); }
    // a (+) b where b is one element (b.y == 0)
    __device__ static Acc op_step(Acc a, Acc b) {
        const float2 s = two_sum(a.x, b.x);
        return make_float2(s.x, __fadd_rn(a.y, s.y));
    }
    __device__ static Car cident() { return make_float2(0.0f, 0.0f); }
    __device__ static Car to_car(Acc a) { return df_add(a, make_float2(0.0f, 0.0f)); }
    __device__ static Car cop(Car a, Car b) { return df_add(a, b); }
    __device__ static CarA to_apply(Car c) { return c; }
    __device__ static CarA base(CarA c, Acc tb) { return df_add(c, tb); }
    __device__ static CarA base_local(Acc tb) { return tb; }
    __device__ static float fin_f(CarA b, Acc v) {
        return __fadd_rn(__fadd_rn(b.x, v.x), __fadd_rn(b.y, v.y));
    }
    __device__ static Out fin(CarA b, Acc v) { return FloatOut<OutT>::cvt(fin_f(b, v)); }
    __device__ static Car car_of_out(Out o) {
        return make_float2(FloatIn<OutT>::load(o), 0.0f);
    }
};

// Step of a left fold that adds one freshly loaded element: K::op_step where
// a kind has a cheaper form for that case, K::op otherwise.
template <class K, class = void>
struct has_op_step : std::false_type {};
template <class K>
struct has_op_step<K, std::void_t<decltype(K::op_step(typename K::Acc{}, typename K::Acc{}))>>
    : std::true_type {};
template <class K>
__device__ __forceinline__ typename K::Acc op_step(typename K::Acc a, typename K::Acc b) {
    if constexpr (has_op_step<K>::value) {
        return K::op_step(a, b);
    } else {
        return K::op(a, b);
    }
}

// 64-bit integers and doubles (the paper's other two types, Table 2)
struct KI64Add {
    static constexpr bool kTieOrdered = false;
    using In = int64_t;
    using Out = int64_t;
    using Acc = uint64_t;  // wrapping mod 2^64
    using Car = uint64_t;
    using CarA = uint64_t;
    __device__ static Acc ident() { return 0ull; }
    __device__ static Acc load(In v) { return static_cast<uint64_t>(v); }
    __device__ static Acc op(Acc a, Acc b) { return a + b; }
    __device__ static Car cident() { return 0ull; }
    __device__ static Car to_car(Acc a) { return a; }
    __device__ static Car cop(Car a, Car b) { return a + b; }
    __device__ static CarA to_apply(Car c) { return c; }
    __device__ static CarA base(CarA c, Acc tb) { return c + tb; }
    __device__ static CarA base_local(Acc tb) { return tb; }
    __device__ static Out fin(CarA b, Acc v) { return static_cast<int64_t>(b + v); }
    __device__ static Car car_of_out(Out o) { return static_cast<uint64_t>(o); }
};

struct KI64Max {
    static constexpr bool kTieOrdered = false;  // equal ints have equal bits
    using In = int64_t;
    using Out = int64_t;
    using Acc = int64_t;
    using Car = int64_t;
    using CarA = int64_t;
    __device__ static Acc ident() { return INT64_MIN; }
    __device__ static Acc load(In v) { return v; }
    __device__ static Acc op(Acc a, Acc b) { return max_keep_left(a, b); }
    __device__ static Car cident() { return INT64_MIN; }
    __device__ static Car to_car(Acc a) { return a; }
    __device__ static Car cop(Car a, Car b) { return max_keep_left(a, b); }
    __device__ static CarA to_apply(Car c) { return c; }
    __device__ static CarA base(CarA c, Acc tb) { return max_keep_left(c, tb); }
    __device__ static CarA base_local(Acc tb) { return tb; }
    __device__ static Out fin(CarA b, Acc v) { return max_keep_left(b, v); }
    __device__ static Car car_of_out(Out o) { return o; }
};

// double max on order-preserving int64 keys: GB300's FP64 pipe is narrow,
// and a key comparison runs on the integer ALUs.  key(bits) flips the
// magnitude bits of negative values, so signed key order is the order of
// the doubles, except that -0 (key -1) sits just below +0 (key 0); gt()
// treats that one pair as equal, as the floating-point comparison does.
// The mapping is an involution (key(key(b)) == b).  NaN is out of contract.
struct KF64Max {
    static constexpr bool kTieOrdered = true;  // +0 / -0 compare equal
    using In = double;
    using Out = double;
    using Acc = int64_t;  // key
    using Car = int64_t;
    using CarA = int64_t;
    __device__ static int64_t key(int64_t b) {
        return b ^ static_cast<int64_t>(static_cast<uint64_t>(b >> 63) >> 1);
    }
    __device__ static bool gt(int64_t a, int64_t b) { return a > b && !(b == -1 && a == 0); }
    __device__ static int64_t mx(int64_t a, int64_t b) { return gt(b, a) ? b : a; }
    __device__ static Acc ident() { return key(static_cast<int64_t>(0xfff0000000000000ull)); }
    __device__ static Acc load(In v) { return key(__double_as_longlong(v)); }
    __device__ static Acc op(Acc a, Acc b) { return mx(a, b); }
    __device__ static Car cident() { return ident(); }
    __device__ static Car to_car(Acc a) { return a; }
    __device__ static Car cop(Car a, Car b) { return mx(a, b); }
    __device__ static CarA to_apply(Car c) { return c; }
    __device__ static CarA base(CarA c, Acc tb) { return mx(c, tb); }
    __device__ static CarA base_local(Acc tb) { return tb; }
    __device__ static Out fin(CarA b, Acc v) { return __longlong_as_double(key(mx(b, v))); }
    __device__ static Car car_of_out(Out o) { return load(o); }
};

// double add: double in tile and in the carry chain
struct KF64Add {
    static constexpr bool kTieOrdered = false;
    using In = double;
    using Out = double;
    using Acc = double;
    using Car = double;
    using CarA = double;
    __device__ static Acc ident() { return 0.0; }
    __device__ static Acc load(In v) { return v; }
    __device__ static Acc op(Acc a, Acc b) { return __dadd_rn(a, b); }
    __device__ static Car cident() { return 0.0; }
    __device__ static Car to_car(Acc a) { return a; }
    __device__ static Car cop(Car a, Car b) { return __dadd_rn(a, b); }
    __device__ static CarA to_apply(Car c) { return c; }
    __device__ static CarA base(CarA c, Acc tb) { return __dadd_rn(c, tb); }
    __device__ static CarA base_local(Acc tb) { return tb; }
    __device__ static Out fin(CarA b, Acc v) { return __dadd_rn(b, v); }
    __device__ static Car car_of_out(Out o) { return o; }
};

// Stream compaction (a consumer of the scan, not in the paper): the scanned
// input is a byte of flags per element (nonzero = keep), the scan counts
// kept elements (uint32 in a tile, uint64 across tiles), and the output
// stage writes each kept value of type V to its index.  Out = V.
template <class V>
struct KSelect {
    static constexpr bool kTieOrdered = false;
    static constexpr bool kSelect = true;
    using In = uint8_t;
    using Out = V;
    using Acc = uint32_t;
    using Car = uint64_t;
    using CarA = uint64_t;
    __device__ static Acc ident() { return 0u; }
    __device__ static Acc load(In f) { return f != 0 ? 1u : 0u; }
    __device__ static Acc op(Acc a, Acc b) { return a + b; }
    __device__ static Car cident() { return 0ull; }
    __device__ static Car to_car(Acc a) { return a; }
    __device__ static Car cop(Car a, Car b) { return a + b; }
    __device__ static CarA to_apply(Car c) { return c; }
    __device__ static CarA base(CarA c, Acc tb) { return c + tb; }
    __device__ static CarA base_local(Acc tb) { return tb; }
    __device__ static Out fin(CarA, Acc) { return Out{}; }  // not used
    __device__ static Car car_of_out(Out) { return 0ull; }  // no carry-in
};

template <class K, class = void>
struct has_raw_max : std::false_type {};
template <class K>
struct has_raw_max<K, std::void_t<decltype(K::kRawMax)>> : std::bool_constant<K::kRawMax> {};

template <class K, class = void>
struct is_select : std::false_type {};
template <class K>
struct is_select<K, std::void_t<decltype(K::kSelect)>> : std::bool_constant<K::kSelect> {};

// kinds whose output is a rounding of an fp32 value (K::fin_f): a bf16
// output pair is rounded and packed by one conversion
template <class K, class = void>
struct has_fin_f : std::false_type {};
template <class K>
struct has_fin_f<K, std::void_t<decltype(K::fin_f(typename K::CarA{}, typename K::Acc{}))>>
    : std::true_type {};

template <class K, class = void>
struct has_split_reduce : std::false_type {};
template <class K>
struct has_split_reduce<K, std::void_t<decltype(K::kSplitReduce)>>
    : std::bool_constant<K::kSplitReduce> {};

// stream compaction whose values travel through the bulk-copy ring with the
// flags (both arrays 16-byte aligned), instead of loads into registers
template <class V>
struct KSelectStaged : KSelect<V> {
    static constexpr bool kStagedValues = true;
};
template <class K, class = void>
struct is_staged_select : std::false_type {};
template <class K>
struct is_staged_select<K, std::void_t<decltype(K::kStagedValues)>>
    : std::bool_constant<K::kStagedValues> {};

// ------------------------------------------------- kind ids (host + device)
enum KindId : int {
    KIND_I32_ADD = 0,
    KIND_I32_MAX,
    KIND_F32_MAX,
    KIND_BF16_MAX,
    KIND_F32_ADD_PLAIN,
    KIND_F32_ADD_F64,
    KIND_F32_ADD_COMP,
    KIND_BF16_ADD_PLAIN_F32,
    KIND_BF16_ADD_F64_F32,
    KIND_BF16_ADD_COMP_F32,
    KIND_BF16_ADD_PLAIN_BF16,
    KIND_BF16_ADD_F64_BF16,
    KIND_BF16_ADD_COMP_BF16,
    KIND_I64_ADD,
    KIND_I64_MAX,
    KIND_F64_MAX,
    KIND_F64_ADD,
    KIND_F32_ADD_DF,  // float add with the double-float carry
    KIND_BF16_ADD_DF_F32,
    KIND_BF16_ADD_DF_BF16,
    KIND_SEL16,  // stream compaction of 2-, 4- and 8-byte values
    KIND_SEL32,
    KIND_SEL64,
    KIND_COUNT
};

}  // namespace lscan
