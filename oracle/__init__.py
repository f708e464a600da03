"""Sequential CPU scan oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  The GPU
library never calls it and has no CPU fallback.

Definition (LightScan, Section 1): inclusive y_j = x_0 (+) ... (+) x_j,
exclusive y_j = x_0 (+) ... (+) x_{j-1} with y_0 the identity.  The C code in
``scan_oracle.c`` is that definition as one sequential loop; accumulation is
int64-wrapping for int32 add and FP64 for float add (see scan_oracle.h).

Python API (numpy in, numpy out):
    scan(op, dtype, x, inclusive=True)            -> np.ndarray
    segscan(op, dtype, x, offsets, inclusive=True) -> np.ndarray
    abs_prefix(dtype, x, inclusive=True)           -> np.ndarray (float64)
    abs_segprefix(dtype, x, offsets, inclusive=True)
    bf16_to_double(bits)                           -> float
    select_flagged(x, flags)                       -> x[flags != 0] in order
    radix_offsets(keys, digit_bits)                -> int64 [P, 2^digit_bits]
op in {"add", "max"}; dtype in {"i32", "f32", "bf16", "i64", "f64"}; bf16
data are uint16 bit patterns.  Output dtype: i32 add/max -> int32, f32/bf16
add -> float64 (the FP64 reference), f32 max -> float32, bf16 max -> uint16
bits, i64 add/max -> int64, f64 add -> float64 (double-double sum rounded
to double), f64 max -> float64 (selected element's bits).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_OPS = {"add": 0, "max": 1}
_DTYPES = {"i32": 0, "f32": 1, "bf16": 2, "i64": 3, "f64": 4}
_IN_NP = {"i32": np.int32, "f32": np.float32, "bf16": np.uint16,
          "i64": np.int64, "f64": np.float64}

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64 = ctypes.c_int64
        vp = ctypes.c_void_p
        lib.oracle_scan.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, i64,
                                    ctypes.c_int]
        lib.oracle_segscan.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp,
                                       i64, ctypes.c_int]
        lib.oracle_abs_prefix.argtypes = [ctypes.c_int, vp, vp, i64,
                                          ctypes.c_int]
        lib.oracle_abs_segprefix.argtypes = [ctypes.c_int, vp, vp, vp, i64,
                                             ctypes.c_int]
        lib.oracle_select_flagged.argtypes = [vp, vp, vp, i64, ctypes.c_int]
        lib.oracle_select_flagged.restype = i64
        lib.oracle_radix_offsets.argtypes = [vp, ctypes.c_int, i64,
                                             ctypes.c_int, vp]
        lib.oracle_radix_offsets.restype = ctypes.c_int
        lib.oracle_bf16_to_double.argtypes = [ctypes.c_uint16]
        lib.oracle_bf16_to_double.restype = ctypes.c_double
        for f in (lib.oracle_scan, lib.oracle_segscan, lib.oracle_abs_prefix,
                  lib.oracle_abs_segprefix):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def out_dtype(op, dtype):
    """numpy dtype of the oracle's output for (op, dtype)."""
    if op == "add":
        if dtype in ("i32", "i64"):
            return _IN_NP[dtype]
        return np.float64
    return _IN_NP[dtype]


def _prep(dtype, x):
    x = np.ascontiguousarray(x)
    if x.dtype != _IN_NP[dtype]:
        raise TypeError(f"oracle: {dtype} input must be {_IN_NP[dtype]}, "
                        f"got {x.dtype}")
    return x


def scan(op, dtype, x, inclusive=True):
    """Sequential inclusive/exclusive scan of a 1-D array (Section 1)."""
    x = _prep(dtype, x)
    y = np.empty(x.shape[0], dtype=out_dtype(op, dtype))
    rc = _load().oracle_scan(_OPS[op], _DTYPES[dtype], x.ctypes.data,
                             y.ctypes.data, x.shape[0], int(bool(inclusive)))
    if rc != 0:
        raise ValueError("oracle_scan rejected its arguments")
    return y


def segscan(op, dtype, x, offsets, inclusive=True):
    """Each segment [offsets[s], offsets[s+1]) scanned independently."""
    x = _prep(dtype, x)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    if off.shape[0] < 1 or off[-1] != x.shape[0]:
        raise ValueError("offsets must end at len(x)")
    y = np.empty(x.shape[0], dtype=out_dtype(op, dtype))
    rc = _load().oracle_segscan(_OPS[op], _DTYPES[dtype], x.ctypes.data,
                                y.ctypes.data, off.ctypes.data,
                                off.shape[0] - 1, int(bool(inclusive)))
    if rc != 0:
        raise ValueError("oracle_segscan rejected its arguments")
    return y


def abs_prefix(dtype, x, inclusive=True):
    """S_j = sum of |x_i| over the scanned prefix, in FP64."""
    x = _prep(dtype, x)
    s = np.empty(x.shape[0], dtype=np.float64)
    rc = _load().oracle_abs_prefix(_DTYPES[dtype], x.ctypes.data,
                                   s.ctypes.data, x.shape[0],
                                   int(bool(inclusive)))
    if rc != 0:
        raise ValueError("oracle_abs_prefix rejected its arguments")
    return s


def abs_segprefix(dtype, x, offsets, inclusive=True):
    """Segmented S_j (restarts at each segment head)."""
    x = _prep(dtype, x)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    s = np.empty(x.shape[0], dtype=np.float64)
    rc = _load().oracle_abs_segprefix(_DTYPES[dtype], x.ctypes.data,
                                      s.ctypes.data, off.ctypes.data,
                                      off.shape[0] - 1, int(bool(inclusive)))
    if rc != 0:
        raise ValueError("oracle_abs_segprefix rejected its arguments")
    return s


def select_flagged(x, flags):
    """Stream compaction: the elements of x whose flag is nonzero, in order
    (a consumer of the scan: each output index is the exclusive prefix sum of
    the flags)."""
    x = np.ascontiguousarray(x)
    f = np.ascontiguousarray(flags, dtype=np.uint8)
    if f.shape[0] != x.shape[0] or x.ndim != 1:
        raise ValueError("x and flags must be 1-D arrays of the same length")
    y = np.empty_like(x)
    k = _load().oracle_select_flagged(x.ctypes.data, f.ctypes.data,
                                      y.ctypes.data, x.shape[0], x.itemsize)
    if k < 0:
        raise ValueError("oracle_select_flagged rejected its arguments")
    return y[:k]


def radix_offsets(keys, digit_bits):
    """Radix-sort digit offsets (a consumer of the scan): for unsigned keys
    (uint32 or uint64), out[p, v] = number of keys whose digit p (digit_bits
    wide, lowest first) is below v -- the exclusive scan of the digit-p
    histogram, where bucket v starts in a counting-sort pass on digit p."""
    k = np.ascontiguousarray(keys)
    if k.dtype not in (np.uint32, np.uint64) or k.ndim != 1:
        raise TypeError("keys must be a 1-D uint32 or uint64 array")
    kb = k.dtype.itemsize
    P = -(-8 * kb // int(digit_bits)) if 1 <= digit_bits <= 8 else 0
    out = np.empty((max(P, 1), 1 << max(0, min(int(digit_bits), 8))),
                   dtype=np.int64)
    rc = _load().oracle_radix_offsets(k.ctypes.data, kb, k.shape[0],
                                      int(digit_bits), out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_radix_offsets rejected its arguments")
    return out


def bf16_to_double(bits):
    """Exact decode of one bf16 bit pattern."""
    return _load().oracle_bf16_to_double(int(bits) & 0xFFFF)


def identity(op, dtype):
    """Identity element of the operator, in the oracle's output dtype."""
    if op == "add":
        return 0
    if dtype == "i32":
        return np.iinfo(np.int32).min
    if dtype == "i64":
        return np.iinfo(np.int64).min
    if dtype == "f32":
        return np.float32(-np.inf)
    if dtype == "f64":
        return np.float64(-np.inf)
    return np.uint16(0xFF80)
