"""Seeded synthetic inputs shared by the tests, the smoke check and bench.py.

This module only draws random numbers; it contains none of the scan's
arithmetic.  The paper evaluates on synthetic arrays described only by N and
dtype (Section 5: N from 32M to 512M, add operator); the shapes below follow
that and the workload list of this library:

  small_i32      : int32, N = 2^20, uniform integers in [-1000, 1000], seed 0
  large_i32_add  : int32, N = 2^28, uniform in [-2^15, 2^15], seed 1
  large_i32_max  : int32, N = 2^28, uniform over the full int32 range, seed 2
  large_f32_add  : fp32,  N = 2^28, uniform in [0, 1), seed 3
  precision      : N = 2^26, x = s * exp(2 Z), Z ~ N(0,1), s = +-1 (p = 1/2),
                   drawn in FP64, rounded to fp32 (round-to-nearest-even) and
                   from that fp32 to bf16 (round-to-nearest-even), seed 4
  batched        : 4096 segment lengths round(2^(20 U)), U ~ U[0,1), clamped
                   to [1, 2^20]; int32 values as large_i32_add, fp32 values
                   uniform in [0, 1), seed 5
  serving        : Poisson arrivals, sizes round(2^(10 + 14 U)), dtype
                   int32/fp32/bf16 at 50/35/15 %, op add/max at 50/50, seed 6
  radix_keys     : uint32 keys, N = 2^28, uniform over all 2^32 values (the
                   usual radix-sort benchmark input), seed 7

bf16 arrays are carried as uint16 bit patterns.
"""
import numpy as np

SEEDS = {
    "small_i32": 0,
    "large_i32_add": 1,
    "large_i32_max": 2,
    "large_f32_add": 3,
    "precision": 4,
    "batched": 5,
    "serving": 6,
    "radix_keys": 7,
}


def f32_to_bf16_bits(x):
    """Round fp32 values to the nearest bf16 (ties to even); uint16 bits."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    lsb = (u >> np.uint32(16)) & np.uint32(1)
    r = (u + np.uint32(0x7FFF) + lsb) >> np.uint32(16)
    return r.astype(np.uint16)


def bf16_bits_to_f32(b):
    """Exact widening of bf16 bit patterns to fp32."""
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32)
            << np.uint32(16)).view(np.float32)


def small_i32(n=1 << 20, seed=SEEDS["small_i32"]):
    rng = np.random.default_rng(seed)
    return rng.integers(-1000, 1001, size=n, dtype=np.int32)


def large_i32_add(n=1 << 28, seed=SEEDS["large_i32_add"]):
    rng = np.random.default_rng(seed)
    return rng.integers(-(1 << 15), (1 << 15) + 1, size=n, dtype=np.int32)


def large_i32_max(n=1 << 28, seed=SEEDS["large_i32_max"]):
    rng = np.random.default_rng(seed)
    return rng.integers(-(1 << 31), 1 << 31, size=n, dtype=np.int32)


def large_f32_add(n=1 << 28, seed=SEEDS["large_f32_add"]):
    rng = np.random.default_rng(seed)
    return rng.random(size=n, dtype=np.float32)


def radix_keys(n=1 << 28, seed=SEEDS["radix_keys"]):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2 ** 32, size=n, dtype=np.uint32)


def precision(n=1 << 26, seed=SEEDS["precision"]):
    """Returns (fp32 array, bf16 bit array) of the cancellation-heavy mix."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(size=n)
    s = np.where(rng.random(size=n) < 0.5, -1.0, 1.0)
    x64 = s * np.exp(2.0 * z)
    x32 = x64.astype(np.float32)  # numpy casts with round-to-nearest-even
    return x32, f32_to_bf16_bits(x32)


def batched_lengths(n_seg=4096, max_log2=20, seed=SEEDS["batched"]):
    rng = np.random.default_rng(seed)
    u = rng.random(size=n_seg)
    lens = np.rint(np.exp2(max_log2 * u)).astype(np.int64)
    return np.clip(lens, 1, 1 << max_log2)


def offsets_from_lengths(lens):
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(np.asarray(lens, dtype=np.int64), out=off[1:])
    return off


def batched(dtype, n_seg=4096, max_log2=20, seed=SEEDS["batched"]):
    """Returns (values, offsets[n_seg+1]) for the batched workload."""
    lens = batched_lengths(n_seg, max_log2, seed)
    off = offsets_from_lengths(lens)
    rng = np.random.default_rng(seed + 1000)
    total = int(off[-1])
    if dtype == "i32":
        x = rng.integers(-(1 << 15), (1 << 15) + 1, size=total, dtype=np.int32)
    elif dtype == "f32":
        x = rng.random(size=total, dtype=np.float32)
    elif dtype == "bf16":
        x = f32_to_bf16_bits(rng.random(size=total, dtype=np.float32))
    else:
        raise ValueError(dtype)
    return x, off


def random_array(dtype, n, rng, kind="uniform"):
    """Generic test input of a given dtype (bf16 as uint16 bits; i64/f64 for
    the 64-bit kinds)."""
    if dtype == "i32":
        if kind == "full":
            return rng.integers(-(1 << 31), 1 << 31, size=n, dtype=np.int32)
        return rng.integers(-1000, 1001, size=n, dtype=np.int32)
    if dtype == "i64":
        if kind == "full":
            return rng.integers(-(1 << 63), (1 << 63) - 1, size=n, dtype=np.int64,
                                endpoint=True)
        return rng.integers(-(1 << 40), (1 << 40) + 1, size=n, dtype=np.int64)
    if dtype == "f64":
        if kind == "intval":
            return rng.integers(-8, 9, size=n).astype(np.float64)
        if kind == "signed":
            return rng.random(size=n) * 2 - 1
        return rng.random(size=n)
    if kind == "intval":
        # integer-valued floats: fp32 prefixes stay exact below 2^24
        f = rng.integers(-8, 9, size=n).astype(np.float32)
    elif kind == "signed":
        f = (rng.random(size=n, dtype=np.float32) * 2 - 1).astype(np.float32)
    else:
        f = rng.random(size=n, dtype=np.float32)
    if dtype == "f32":
        return f
    if dtype == "bf16":
        return f32_to_bf16_bits(f)
    raise ValueError(dtype)


def ties_array(dtype, n, rng, pattern="zeros", first_zero=0, p_zero=0.02):
    """Tie-heavy input for the float max scans (fp32, bf16 bits, double),
    drawn from small pools.  Under max, equal values differ in their bits only
    for +0 and -0, so these arrays make the first-occurrence rule observable:
      "zeros"      : -1, -2.5 and -inf (the identity's value), with +0 or -0
                     (random sign) at rate p_zero from index first_zero on;
                     before it only negatives, so the running maximum is a
                     zero whose sign is that of the first zero
      "all_zeros"  : +0 or -0 only (random signs)
      "repeated"   : 0.5, 0.25, -1 and +-0 at similar rates (repeated maxima)
    """
    if pattern == "all_zeros":
        f = np.where(rng.random(size=n) < 0.5, -0.0, 0.0)
    elif pattern == "repeated":
        f = rng.choice(np.array([0.5, 0.25, -1.0, 0.0, -0.0]), size=n)
    elif pattern == "zeros":
        f = rng.choice(np.array([-1.0, -2.5, -np.inf]), size=n)
        z = np.where(rng.random(size=n) < 0.5, -0.0, 0.0)
        put = rng.random(size=n) < p_zero
        put[:first_zero] = False
        if 0 <= first_zero < n:
            put[first_zero] = True
        f = np.where(put, z, f)
    else:
        raise ValueError(pattern)
    if dtype == "f64":
        return f.astype(np.float64)
    f32 = f.astype(np.float32)
    if dtype == "f32":
        return f32
    if dtype == "bf16":
        return f32_to_bf16_bits(f32)
    raise ValueError(dtype)


def serving_requests(n_req, seed=SEEDS["serving"], min_log2=10, max_log2=24):
    """Request mix: list of dicts (size, dtype, op); arrival gaps drawn later."""
    rng = np.random.default_rng(seed)
    u = rng.random(size=n_req)
    sizes = np.rint(np.exp2(min_log2 + (max_log2 - min_log2) * u)).astype(
        np.int64)
    d = rng.random(size=n_req)
    dtypes = np.where(d < 0.50, "i32", np.where(d < 0.85, "f32", "bf16"))
    ops = np.where(rng.random(size=n_req) < 0.5, "add", "max")
    return [dict(n=int(sizes[i]), dtype=str(dtypes[i]), op=str(ops[i]))
            for i in range(n_req)]


def poisson_gaps(n_req, rate_per_s, seed=SEEDS["serving"] + 1):
    """Exponential inter-arrival gaps (seconds) for a Poisson stream."""
    rng = np.random.default_rng(seed)
    return rng.exponential(1.0 / rate_per_s, size=n_req)
