"""Pins for the CPU oracle (no GPU).

The oracle is the authority the GPU path is checked against, so it is pinned
here to things other than itself: hand-computed fixtures (tests/golden), closed
forms, the inclusive/exclusive relation stated in LightScan Section 1, brute
force with Python's exact integers and fractions, and independent library
routines (numpy cumsum / maximum.accumulate) on the special cases where they
are exact.  A dropped term, a wrong identity, an off-by-one between inclusive
and exclusive, a truncation instead of a wrap, or a float accumulator in place
of FP64 each fails at least one test here.
"""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

from conftest import golden

I32_MIN = -(1 << 31)


def wrap32(v):
    v &= 0xFFFFFFFF
    return v - (1 << 32) if v >= (1 << 31) else v


def f32_from_hex(h):
    return np.array([int(h, 16)], dtype=np.uint32).view(np.float32)[0]


# ----------------------------------------------------------------- fixtures
def test_golden_i32_small(oracle_mod):
    g = golden("scan_i32_small.txt")
    x = np.array(g["x"], dtype=np.int32)
    for op in ("add", "max"):
        for incl, key in ((True, "inclusive"), (False, "exclusive")):
            want = np.array(g[f"{op}_{key}"], dtype=np.int64)
            got = oracle_mod.scan(op, "i32", x, inclusive=incl)
            assert got.dtype == np.int32
            np.testing.assert_array_equal(got.astype(np.int64), want)


def test_golden_i32_wrap(oracle_mod):
    g = golden("scan_i32_wrap.txt")
    x = np.array(g["x"], dtype=np.int32)
    np.testing.assert_array_equal(
        oracle_mod.scan("add", "i32", x, True).astype(np.int64),
        np.array(g["add_inclusive"], dtype=np.int64))
    np.testing.assert_array_equal(
        oracle_mod.scan("add", "i32", x, False).astype(np.int64),
        np.array(g["add_exclusive"], dtype=np.int64))


def test_golden_f32_max_ties_bits(oracle_mod):
    g = golden("scan_f32_maxties_bits.txt")
    for xs, ys, incl in (("x", "max_inclusive", True),
                         ("x2", "max_inclusive2", True),
                         ("x3", "max_inclusive3", True),
                         ("x3", "max_exclusive3", False)):
        x = np.array([int(h, 16) for h in g[xs]], dtype=np.uint32).view(
            np.float32)
        want = np.array([int(h, 16) for h in g[ys]], dtype=np.uint32)
        got = oracle_mod.scan("max", "f32", x, incl).view(np.uint32)
        np.testing.assert_array_equal(got, want)


def test_golden_f32_add_fp64_reference(oracle_mod):
    g = golden("scan_f32_add_exact.txt")
    x = np.array(g["x"], dtype=np.float32)
    np.testing.assert_array_equal(oracle_mod.scan("add", "f32", x, True),
                                  np.array(g["add_inclusive"], dtype=float))
    np.testing.assert_array_equal(oracle_mod.scan("add", "f32", x, False),
                                  np.array(g["add_exclusive"], dtype=float))
    x2 = np.array(g["x2"], dtype=np.float32)
    np.testing.assert_array_equal(oracle_mod.scan("add", "f32", x2, True),
                                  np.array(g["add_inclusive2"], dtype=float))


def _parse_value(s):
    if s.startswith("2^"):
        return 2.0 ** int(s[2:])
    return float(s)


def test_golden_bf16(oracle_mod):
    g = golden("bf16_decode.txt")
    for b, v in zip(g["bits"], g["values"]):
        got = oracle_mod.bf16_to_double(int(b, 16))
        want = _parse_value(v)
        assert got == want and math.copysign(1, got) == math.copysign(1, want)
    x = np.array([int(h, 16) for h in g["x"]], dtype=np.uint16)
    np.testing.assert_array_equal(oracle_mod.scan("add", "bf16", x, True),
                                  np.array(g["add_inclusive"], dtype=float))
    np.testing.assert_array_equal(oracle_mod.scan("add", "bf16", x, False),
                                  np.array(g["add_exclusive"], dtype=float))
    np.testing.assert_array_equal(
        oracle_mod.scan("max", "bf16", x, True),
        np.array([int(h, 16) for h in g["max_inclusive"]], dtype=np.uint16))
    np.testing.assert_array_equal(
        oracle_mod.scan("max", "bf16", x, False),
        np.array([int(h, 16) for h in g["max_exclusive"]], dtype=np.uint16))


def test_golden_segscan(oracle_mod):
    g = golden("segscan_i32.txt")
    off = np.array(g["offsets"], dtype=np.int64)
    x = np.array(g["x"], dtype=np.int32)
    for op in ("add", "max"):
        for incl, key in ((True, "inclusive"), (False, "exclusive")):
            got = oracle_mod.segscan(op, "i32", x, off, incl)
            np.testing.assert_array_equal(
                got.astype(np.int64),
                np.array(g[f"{op}_{key}"], dtype=np.int64))


# ------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [1, 2, 7, 1000, 100003])
def test_closed_form_all_ones(oracle_mod, n):
    x = np.ones(n, dtype=np.int32)
    np.testing.assert_array_equal(oracle_mod.scan("add", "i32", x),
                                  np.arange(1, n + 1, dtype=np.int32))
    np.testing.assert_array_equal(oracle_mod.scan("add", "i32", x, False),
                                  np.arange(0, n, dtype=np.int32))
    xf = np.ones(n, dtype=np.float32)
    np.testing.assert_array_equal(oracle_mod.scan("add", "f32", xf),
                                  np.arange(1, n + 1, dtype=np.float64))


@pytest.mark.parametrize("n", [5, 4097, 200001])
def test_closed_form_triangular(oracle_mod, n):
    # x_i = i  ->  y_j = j (j + 1) / 2, taken mod 2^32 for int32
    x = np.arange(n, dtype=np.int64)
    tri = x * (x + 1) // 2
    want = ((tri + (1 << 31)) % (1 << 32) - (1 << 31)).astype(np.int32)
    np.testing.assert_array_equal(
        oracle_mod.scan("add", "i32", x.astype(np.int32)), want)
    # the same in the float reference: exact while below 2^53
    xf = np.arange(min(n, 4097), dtype=np.float32)
    j = np.arange(min(n, 4097), dtype=np.float64)
    np.testing.assert_array_equal(oracle_mod.scan("add", "f32", xf),
                                  j * (j + 1) / 2)


def test_closed_form_max_monotone(oracle_mod):
    rng = np.random.default_rng(11)
    inc = np.sort(rng.integers(-10**9, 10**9, size=5000)).astype(np.int32)
    np.testing.assert_array_equal(oracle_mod.scan("max", "i32", inc), inc)
    dec = inc[::-1].copy()
    np.testing.assert_array_equal(oracle_mod.scan("max", "i32", dec),
                                  np.full_like(dec, dec[0]))
    f = np.sort(rng.standard_normal(3000).astype(np.float32))
    np.testing.assert_array_equal(oracle_mod.scan("max", "f32", f), f)
    np.testing.assert_array_equal(oracle_mod.scan("max", "f32", f[::-1].copy()),
                                  np.full_like(f, f[-1]))


def test_empty_and_single(oracle_mod):
    for op in ("add", "max"):
        for dt, arr in (("i32", np.array([], np.int32)),
                        ("f32", np.array([], np.float32)),
                        ("bf16", np.array([], np.uint16))):
            assert oracle_mod.scan(op, dt, arr).shape == (0,)
    assert oracle_mod.scan("add", "i32", np.array([-7], np.int32))[0] == -7
    assert oracle_mod.scan("add", "i32", np.array([-7], np.int32), False)[0] == 0
    assert oracle_mod.scan("max", "i32", np.array([-7], np.int32),
                           False)[0] == I32_MIN


# ---------------------------------------- inclusive / exclusive relation (S1)
@pytest.mark.parametrize("dtype", ["i32", "f32", "bf16"])
@pytest.mark.parametrize("op", ["add", "max"])
def test_inclusive_exclusive_relation(oracle_mod, op, dtype):
    from paper_1604_04815_gb300.workloads import random_array
    rng = np.random.default_rng(3)
    x = random_array(dtype, 3001, rng, kind="signed" if dtype != "i32" else
                     "full")
    inc = oracle_mod.scan(op, dtype, x, True)
    exc = oracle_mod.scan(op, dtype, x, False)
    ident = oracle_mod.identity(op, dtype)
    assert exc[0] == ident
    np.testing.assert_array_equal(exc[1:], inc[:-1])
    # excl_j (+) x_j == incl_j
    if op == "add" and dtype == "i32":
        np.testing.assert_array_equal(
            (exc.astype(np.int64) + x) % (1 << 32),
            inc.astype(np.int64) % (1 << 32))
    elif op == "add":
        xv = (x.astype(np.float64) if dtype == "f32" else
              np.array([oracle_mod.bf16_to_double(b) for b in x]))
        np.testing.assert_array_equal(exc + xv, inc)


# --------------------------------------------------------------- brute force
def _brute(op, vals):
    """O(n^2) recomputation with Python exact arithmetic."""
    inc = []
    for j in range(len(vals)):
        pre = vals[: j + 1]
        if op == "add":
            inc.append(sum(pre, Fraction(0)) if isinstance(pre[0], Fraction)
                       else sum(pre))
        else:
            m = pre[0]
            for v in pre[1:]:
                if v > m:
                    m = v
            inc.append(m)
    return inc


@pytest.mark.parametrize("n", [1, 2, 3, 17, 33, 64])
def test_brute_force_int32(oracle_mod, n):
    rng = np.random.default_rng(100 + n)
    x = rng.integers(-(1 << 31), 1 << 31, size=n, dtype=np.int32)
    vals = [int(v) for v in x]
    add = [wrap32(v) for v in _brute("add", vals)]
    mx = _brute("max", vals)
    np.testing.assert_array_equal(oracle_mod.scan("add", "i32", x).astype(
        np.int64), add)
    np.testing.assert_array_equal(oracle_mod.scan("max", "i32", x).astype(
        np.int64), mx)
    np.testing.assert_array_equal(oracle_mod.scan("add", "i32", x, False)
                                  .astype(np.int64), [0] + add[:-1])
    np.testing.assert_array_equal(oracle_mod.scan("max", "i32", x, False)
                                  .astype(np.int64), [I32_MIN] + mx[:-1])


@pytest.mark.parametrize("n", [1, 5, 31, 64])
def test_brute_force_f32_exact_within_fp64(oracle_mod, n):
    """FP64 reference vs the exact rational prefix: |err| <= n 2^-53 S_j."""
    rng = np.random.default_rng(200 + n)
    x = ((rng.random(n) * 2 - 1) * np.exp2(rng.integers(-20, 20, n))).astype(
        np.float32)
    exact = _brute("add", [Fraction(float(v)) for v in x])
    got = oracle_mod.scan("add", "f32", x)
    s = np.cumsum(np.abs(x.astype(np.float64)))
    for j in range(n):
        err = abs(Fraction(float(got[j])) - exact[j])
        assert err <= Fraction(n) * Fraction(2) ** -53 * Fraction(float(s[j]))


@pytest.mark.parametrize("n", [1, 5, 31, 64])
def test_brute_force_bf16_add_exact_within_fp64(oracle_mod, n):
    """bf16 add: the FP64 reference of the decoded inputs against the exact
    rational prefix of (bits << 16) read as IEEE singles."""
    rng = np.random.default_rng(250 + n)
    b = rng.integers(0, 1 << 16, size=n, dtype=np.uint16)
    b = b[((b >> 7) & 0xFF) != 0xFF]  # no Inf/NaN
    vals = [struct.unpack("<f", struct.pack("<I", int(v) << 16))[0] for v in b]
    exact = _brute("add", [Fraction(v) for v in vals])
    got = oracle_mod.scan("add", "bf16", b)
    s = np.cumsum(np.abs(np.array(vals, dtype=np.float64)))
    for j in range(len(vals)):
        err = abs(Fraction(float(got[j])) - exact[j])
        assert err <= Fraction(len(vals)) * Fraction(2) ** -53 * Fraction(float(s[j]))


@pytest.mark.parametrize("n", [1, 9, 64])
def test_brute_force_max_first_occurrence(oracle_mod, n):
    """Max-scan bits are those of the FIRST occurrence of the prefix max."""
    rng = np.random.default_rng(300 + n)
    pool = np.array([0.0, -0.0, 1.5, -2.0, 1.5, -0.0], dtype=np.float32)
    x = pool[rng.integers(0, len(pool), n)]
    got = oracle_mod.scan("max", "f32", x).view(np.uint32)
    xb = x.view(np.uint32)
    for j in range(n):
        m = max(float(v) for v in x[: j + 1])
        first = next(i for i in range(j + 1) if float(x[i]) == m)
        assert got[j] == xb[first]
    b = np.array([0x3F80, 0x8000, 0x0000, 0x3F80, 0xC000], dtype=np.uint16)
    xb16 = b[rng.integers(0, len(b), n)]
    got16 = oracle_mod.scan("max", "bf16", xb16)
    for j in range(n):
        vals = [oracle_mod.bf16_to_double(v) for v in xb16[: j + 1]]
        m = max(vals)
        first = next(i for i in range(j + 1) if vals[i] == m)
        assert got16[j] == xb16[first]


# ------------------------------------------- independent library cross-checks
def test_numpy_cumsum_small_magnitude(oracle_mod):
    """No wrap possible -> int32 add equals numpy's int64 cumsum exactly."""
    rng = np.random.default_rng(5)
    x = rng.integers(-1000, 1001, size=1 << 20, dtype=np.int32)
    np.testing.assert_array_equal(oracle_mod.scan("add", "i32", x),
                                  np.cumsum(x, dtype=np.int64).astype(np.int32))
    np.testing.assert_array_equal(oracle_mod.scan("max", "i32", x),
                                  np.maximum.accumulate(x))


def test_numpy_cumsum_integer_valued_float(oracle_mod):
    """Integer-valued fp32 inputs: FP64 prefix is exact, equals float64 cumsum."""
    rng = np.random.default_rng(6)
    x = rng.integers(-8, 9, size=200000).astype(np.float32)
    np.testing.assert_array_equal(oracle_mod.scan("add", "f32", x),
                                  np.cumsum(x.astype(np.float64)))


def test_bf16_decode_matches_struct(oracle_mod):
    """bf16 -> double equals decoding (bits << 16) as an IEEE single."""
    rng = np.random.default_rng(7)
    for b in rng.integers(0, 1 << 16, size=2000):
        w = int(b) << 16
        exp = (w >> 23) & 0xFF
        if exp == 0xFF and (w & 0x7FFFFF):
            continue  # NaN: outside the contract
        want = struct.unpack("<f", struct.pack("<I", w))[0]
        assert oracle_mod.bf16_to_double(int(b)) == want


# ------------------------------------------------------------ segmented scans
def test_segscan_matches_per_segment_and_brute(oracle_mod):
    rng = np.random.default_rng(8)
    lens = [0, 1, 0, 5, 33, 0, 2, 64, 1]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    x = rng.integers(-(1 << 31), 1 << 31, size=int(off[-1]), dtype=np.int32)
    for op in ("add", "max"):
        for incl in (True, False):
            got = oracle_mod.segscan(op, "i32", x, off, incl).astype(np.int64)
            for s in range(len(lens)):
                a, b = off[s], off[s + 1]
                if a == b:
                    continue
                vals = [int(v) for v in x[a:b]]
                br = _brute(op, vals)
                if op == "add":
                    br = [wrap32(v) for v in br]
                if not incl:
                    br = [0 if op == "add" else I32_MIN] + br[:-1]
                np.testing.assert_array_equal(got[a:b], br)


def test_segscan_rejects_bad_offsets(oracle_mod):
    x = np.zeros(4, np.int32)
    with pytest.raises(ValueError):
        oracle_mod.segscan("add", "i32", x, np.array([0, 3, 2, 4]))
    with pytest.raises(ValueError):
        oracle_mod.segscan("add", "i32", x, np.array([0, 3]))


# --------------------------------------------------------- error-bound helper
def test_abs_prefix_properties(oracle_mod):
    rng = np.random.default_rng(9)
    x = (rng.random(5000, dtype=np.float32) * 2 - 1).astype(np.float32)
    s = oracle_mod.abs_prefix("f32", x)
    y = oracle_mod.scan("add", "f32", x)
    assert np.all(np.abs(y) <= s * (1 + 1e-12))          # triangle inequality
    assert np.all(np.diff(s) >= 0)
    xp = np.abs(x)
    np.testing.assert_array_equal(oracle_mod.abs_prefix("f32", xp),
                                  oracle_mod.scan("add", "f32", xp))
    se = oracle_mod.abs_prefix("f32", x, inclusive=False)
    assert se[0] == 0.0
    np.testing.assert_array_equal(se[1:], s[:-1])
    off = np.array([0, 10, 10, 5000], dtype=np.int64)
    ss = oracle_mod.abs_segprefix("f32", x, off)
    np.testing.assert_array_equal(ss[:10], s[:10])
    np.testing.assert_array_equal(ss[10:], oracle_mod.abs_prefix("f32", x[10:]))


def test_golden_abs_prefix_bf16_and_i32(oracle_mod):
    """The bf16 branch decodes bit patterns and the int32 branch widens
    before taking |x| (|INT32_MIN| = 2^31)."""
    g = golden("abs_prefix.txt")
    xb = np.array([int(v, 16) for v in g["bf16_x"]], dtype=np.uint16)
    for incl, key in ((True, "bf16_inclusive"), (False, "bf16_exclusive")):
        want = np.array([float(v) for v in g[key]])
        assert np.array_equal(oracle_mod.abs_prefix("bf16", xb, incl), want)
    xi = np.array([int(v) for v in g["i32_x"]], dtype=np.int32)
    for incl, key in ((True, "i32_inclusive"), (False, "i32_exclusive")):
        want = np.array([float(v) for v in g[key]])
        assert np.array_equal(oracle_mod.abs_prefix("i32", xi, incl), want)


@pytest.mark.parametrize("n", [1, 17, 300])
def test_abs_prefix_bf16_i32_brute_force(oracle_mod, n):
    """Exact rational / integer sums of |x_i| with an independent decode
    (struct) of the bf16 bits; every partial sum here is exact in FP64."""
    import struct
    from fractions import Fraction
    rng = np.random.default_rng(n)
    # random signs and mantissas, biased exponents 120..135: the sums span
    # fewer than 53 bits, so each FP64 partial sum is exact
    sign = rng.integers(0, 2, size=n) << 15
    expo = rng.integers(120, 136, size=n) << 7
    mant = rng.integers(0, 128, size=n)
    xb = (sign | expo | mant).astype(np.uint16)
    vals = [abs(Fraction(struct.unpack(">f", struct.pack(">I", int(b) << 16))[0]))
            for b in xb]
    got = oracle_mod.abs_prefix("bf16", xb)
    acc = Fraction(0)
    for j, v in enumerate(vals):
        acc += v
        assert Fraction(got[j]) == acc
    xi = rng.integers(-(1 << 31), 1 << 31, size=n, dtype=np.int32)
    xi[0] = -(1 << 31)
    got = oracle_mod.abs_prefix("i32", xi, inclusive=False)
    acc = 0
    for j, v in enumerate(xi.tolist()):
        assert got[j] == acc
        acc += abs(v)


# ------------------------------------------------------ int64 and double
def test_golden_i64_wrap(oracle_mod):
    g = golden("scan_i64_wrap.txt")
    x = np.array([int(v) for v in g["x"]], dtype=np.int64)
    for key, incl in (("add_inclusive", True), ("add_exclusive", False)):
        want = np.array([int(v) for v in g[key]], dtype=np.int64)
        assert np.array_equal(oracle_mod.scan("add", "i64", x, incl), want)
    x2 = np.array([int(v) for v in g["x2"]], dtype=np.int64)
    want2 = np.array([int(v) for v in g["add_inclusive2"]], dtype=np.int64)
    assert np.array_equal(oracle_mod.scan("add", "i64", x2, True), want2)


def test_golden_f64_add_double_double(oracle_mod):
    g = golden("scan_f64_add_dd.txt")
    for xk, keys in (("x", (("add_inclusive", True), ("add_exclusive", False))),
                     ("x2", (("add_inclusive2", True),))):
        x = np.array([float(v) for v in g[xk]], dtype=np.float64)
        for key, incl in keys:
            want = np.array([float(v) for v in g[key]], dtype=np.float64)
            got = oracle_mod.scan("add", "f64", x, incl)
            assert np.array_equal(got, want), (xk, key, got, want)


@pytest.mark.parametrize("n", [1, 2, 17, 64])
def test_brute_force_int64_mod_2_64(oracle_mod, n):
    rng = np.random.default_rng(640 + n)
    x = rng.integers(-2**63, 2**63, size=n, dtype=np.int64)
    for incl in (True, False):
        want = []
        for j in range(n):
            acc = sum(int(v) for v in x[: j + 1 if incl else j]) % 2**64
            want.append(acc - 2**64 if acc >= 2**63 else acc)
        assert np.array_equal(oracle_mod.scan("add", "i64", x, incl),
                              np.array(want, dtype=np.int64))


@pytest.mark.parametrize("n", [1, 3, 40, 200])
def test_brute_force_f64_add_vs_exact_rationals(oracle_mod, n):
    """Each output is the exact prefix sum (Python Fractions) rounded to
    double, to within one unit in the last place; magnitudes spread over
    2^-40 .. 2^40 with both signs so that double accumulation would lose
    many digits."""
    from fractions import Fraction
    rng = np.random.default_rng(641 + n)
    x = (rng.choice([-1.0, 1.0], size=n) *
         np.ldexp(rng.random(n) + 0.5, rng.integers(-40, 41, size=n)))
    for incl in (True, False):
        got = oracle_mod.scan("add", "f64", x, incl)
        acc = Fraction(0)
        for j in range(n):
            if incl:
                acc += Fraction(float(x[j]))
            exact = float(acc)
            tol = np.spacing(abs(exact)) if exact != 0 else 0.0
            assert abs(got[j] - exact) <= tol, (j, got[j], exact)
            if not incl:
                acc += Fraction(float(x[j]))


@pytest.mark.parametrize("dtype", ["i64", "f64"])
def test_brute_force_max_64bit_first_occurrence(oracle_mod, dtype):
    rng = np.random.default_rng(642)
    if dtype == "i64":
        x = rng.integers(-5, 5, size=50, dtype=np.int64) * (2**40)
    else:
        x = rng.integers(-3, 3, size=50).astype(np.float64)
        x[rng.random(50) < 0.3] = 0.0
        x[rng.random(50) < 0.3] = -0.0
    ident = oracle_mod.identity("max", dtype)
    for incl in (True, False):
        got = oracle_mod.scan("max", dtype, x, incl)
        for j in range(50):
            best = ident
            for i in range(j + 1 if incl else j):
                if x[i] > best:
                    best = x[i]
            assert np.array(got[j]).tobytes() == np.array(
                best, dtype=x.dtype).tobytes(), (j, got[j], best)


@pytest.mark.parametrize("op,dtype", [("add", "i64"), ("max", "i64"),
                                      ("add", "f64"), ("max", "f64")])
def test_inclusive_exclusive_relation_64bit(oracle_mod, op, dtype):
    rng = np.random.default_rng(643)
    if dtype == "i64":
        x = rng.integers(-2**40, 2**40, size=300, dtype=np.int64)
    else:
        x = rng.standard_normal(300) * 1e3
    inc = oracle_mod.scan(op, dtype, x, True)
    exc = oracle_mod.scan(op, dtype, x, False)
    assert np.array_equal(exc[1:], inc[:-1])
    if op == "max":
        assert exc[0] == oracle_mod.identity(op, dtype)
    else:
        assert exc[0] == 0


def test_abs_prefix_f64(oracle_mod):
    x = np.array([1.5, -2.25, 0.0, -0.125])
    assert np.array_equal(oracle_mod.abs_prefix("f64", x, True),
                          [1.5, 3.75, 3.75, 3.875])
    assert np.array_equal(oracle_mod.abs_prefix("f64", x, False),
                          [0.0, 1.5, 3.75, 3.75])


# ------------------------------------------------------- stream compaction
def test_golden_select_flagged(oracle_mod):
    g = golden("select_flagged.txt")
    x = np.array([int(v) for v in g["x"]], dtype=np.int32)
    f = np.array([int(v) for v in g["flags"]], dtype=np.uint8)
    assert np.array_equal(oracle_mod.select_flagged(x, f),
                          np.array([int(v) for v in g["selected"]], np.int32))
    # output index = exclusive scan of the 0/1 flags (the oracle's own scan)
    pos = oracle_mod.scan("add", "i32", (f != 0).astype(np.int32), False)
    assert np.array_equal(pos, [int(v) for v in g["positions"]])


@pytest.mark.parametrize("dtype", [np.int16, np.int32, np.float32, np.int64,
                                   np.float64])
@pytest.mark.parametrize("p_keep", [0.0, 0.03, 0.5, 1.0])
def test_select_flagged_matches_mask_and_keeps_bits(oracle_mod, dtype, p_keep):
    rng = np.random.default_rng(int(p_keep * 100) + np.dtype(dtype).itemsize)
    n = 1000
    x = rng.integers(-1000, 1000, size=n).astype(dtype)
    f = (rng.random(n) < p_keep).astype(np.uint8) * rng.integers(1, 256, n,
                                                                 dtype=np.uint8)
    got = oracle_mod.select_flagged(x, f)
    want = x[f != 0]
    assert got.dtype == x.dtype and np.array_equal(got.view(np.uint8),
                                                   want.view(np.uint8))
    assert got.shape[0] == int(np.count_nonzero(f))


# ------------------------------------------------- radix-sort digit offsets
def _digit(k, p, b):
    return (int(k) >> (p * b)) & ((1 << b) - 1)


def test_golden_radix_offsets(oracle_mod):
    g = golden("radix_offsets.txt")
    keys = np.array([int(v, 16) for v in g["keys"]], dtype=np.uint32)
    got = oracle_mod.radix_offsets(keys, 8)
    assert got.shape == (4, 256)
    at = [int(v) for v in g["at_v"]]
    for p in range(4):
        assert [int(got[p, v]) for v in at] == [int(v) for v in g[f"p{p}"]]


@pytest.mark.parametrize("kdt", [np.uint32, np.uint64])
@pytest.mark.parametrize("b", [1, 3, 4, 5, 8])
def test_radix_offsets_brute_force(oracle_mod, kdt, b):
    """The definition itself, key by key: how many keys have a smaller
    digit p than v (no histogram, no running sum)."""
    rng = np.random.default_rng(b * 10 + np.dtype(kdt).itemsize)
    kb = 8 * np.dtype(kdt).itemsize
    keys = rng.integers(0, 2 ** kb, size=37, dtype=kdt)
    got = oracle_mod.radix_offsets(keys, b)
    P = -(-kb // b)
    assert got.shape == (P, 1 << b)
    for p in range(P):
        digits = [_digit(k, p, b) for k in keys]
        for v in range(1 << b):
            assert got[p, v] == sum(1 for d in digits if d < v), (p, v)


@pytest.mark.parametrize("b", [2, 5, 8])
def test_radix_offsets_closed_form_identity_keys(oracle_mod, b):
    """keys 0 .. 2^m - 1: the w = clamp(m - p b, 0, b) low bits of digit p
    take every value equally often, so offsets[p][v] = min(v, 2^w) 2^(m-w)."""
    m = 13
    n = 1 << m
    got = oracle_mod.radix_offsets(np.arange(n, dtype=np.uint32), b)
    for p in range(got.shape[0]):
        w = min(max(m - p * b, 0), b)
        want = [min(v, 1 << w) * (n >> w) for v in range(1 << b)]
        assert got[p].tolist() == want, p


def test_radix_offsets_equal_keys_and_empty(oracle_mod):
    k = np.uint64(0xDEADBEEF01234567)
    got = oracle_mod.radix_offsets(np.full(100, k, dtype=np.uint64), 8)
    for p in range(8):
        d = _digit(k, p, 8)
        assert got[p].tolist() == [0] * (d + 1) + [100] * (255 - d)
    assert not oracle_mod.radix_offsets(np.zeros(0, np.uint32), 4).any()


@pytest.mark.parametrize("kdt", [np.uint32, np.uint64])
def test_radix_offsets_place_a_stable_counting_sort(oracle_mod, kdt):
    """Scattering each key to offsets[p][digit] + (keys with the same digit
    before it) must give numpy's stable sort by that digit, for every p."""
    rng = np.random.default_rng(7)
    kb = 8 * np.dtype(kdt).itemsize
    keys = rng.integers(0, 2 ** kb, size=5000, dtype=kdt)
    b = 6
    off = oracle_mod.radix_offsets(keys, b)
    for p in range(off.shape[0]):
        d = ((keys >> kdt(p * b)) & kdt((1 << b) - 1)).astype(np.int64)
        nxt = off[p].copy()
        out = np.empty_like(keys)
        for j in range(keys.shape[0]):
            out[nxt[d[j]]] = keys[j]
            nxt[d[j]] += 1
        assert np.array_equal(out, keys[np.argsort(d, kind="stable")]), p


def test_radix_offsets_rejects_bad_arguments(oracle_mod):
    with pytest.raises(TypeError):
        oracle_mod.radix_offsets(np.zeros(4, np.int32), 8)
    for b in (0, 9):
        with pytest.raises(ValueError):
            oracle_mod.radix_offsets(np.zeros(4, np.uint32), b)
