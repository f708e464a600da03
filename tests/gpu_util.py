"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare it element by element with the CPU oracle."""
import numpy as np
import torch

import oracle
import paper_1604_04815_gb300 as lscan
from paper_1604_04815_gb300 import _lib

DTYPES = {"i32": torch.int32, "f32": torch.float32, "bf16": torch.bfloat16,
          "i64": torch.int64, "f64": torch.float64}
LDT = {"i32": _lib.LSCAN_I32, "f32": _lib.LSCAN_F32, "bf16": _lib.LSCAN_BF16,
       "i64": _lib.LSCAN_I64, "f64": _lib.LSCAN_F64}
LOP = {"add": _lib.LSCAN_ADD, "max": _lib.LSCAN_MAX}

# device wait limit used by the GPU tests (a hang-free failure in ~0.2 s)
TEST_WAIT_NS = 200_000_000

# |y_j - ref_j| <= c * S_j for float add, per precision path
BOUND = {"plain": 1e-5, "f64": 1e-5, "df": 1e-5, "comp": 2.5e-7}
# double add (double in tile and carry): |y_j - ref_j| <= 1e-12 * S_j
# (~9000 units of double roundoff: the worst case (K + 11 + carry hops) u S_j
# of a double-in-tile, double-carry scan stays below it up to ~9000 hops)
BOUND_F64_ADD = 1e-12
PREC_CODE = {"plain": _lib.LSCAN_PREC_F32_CARRY, "f64": _lib.LSCAN_PREC_F64_CARRY,
             "comp": _lib.LSCAN_PREC_COMPENSATED, "df": _lib.LSCAN_PREC_DF_CARRY}


def to_device(x_np, dtype, pad_front=0):
    """Upload a numpy array (bf16 as uint16 bits); pad_front > 0 returns a
    view that starts pad_front elements into its allocation (unaligned)."""
    if dtype == "bf16":
        t = torch.from_numpy(x_np.view(np.int16).copy()).view(torch.bfloat16)
    else:
        t = torch.from_numpy(np.ascontiguousarray(x_np))
    t = t.cuda()
    if pad_front:
        buf = torch.empty(t.shape[0] + pad_front, dtype=t.dtype, device="cuda")
        buf[pad_front:] = t
        t = buf[pad_front:]
    return t


def to_host(y):
    if y.dtype == torch.bfloat16:
        return y.view(torch.int16).cpu().numpy().view(np.uint16)
    return y.cpu().numpy()


def out_torch_dtype(op, dtype, out_bf16=False):
    if op == "add" and dtype == "bf16":
        return torch.bfloat16 if out_bf16 else torch.float32
    return DTYPES[dtype]


def run_c_abi(op, dtype, x_dev, inclusive=True, prec=None, carry=0, config=0,
              out_bf16=False, y_dev=None, check_status=True):
    """One call of lscan_scan through the C ABI on torch's current stream."""
    n = x_dev.shape[0]
    if y_dev is None:
        y_dev = torch.empty(n, dtype=out_torch_dtype(op, dtype, out_bf16),
                            device="cuda")
    opts = _lib.make_options(
        out_dtype=_lib.LSCAN_BF16 if out_bf16 else 0,
        precision=PREC_CODE[prec] if prec else 0, carry=carry, config=config)
    stream = torch.cuda.current_stream().cuda_stream
    st = _lib.lscan_scan(LOP[op], LDT[dtype], int(inclusive), x_dev.data_ptr(),
                         y_dev.data_ptr(), n, opts, stream)
    assert st == _lib.LSCAN_OK, _lib.strerror(st)
    if check_status:
        st = _lib.lscan_stream_status(stream)
        assert st == _lib.LSCAN_OK, _lib.strerror(st)
    return y_dev


def assert_matches(op, dtype, x_np, got, inclusive=True, prec="f64",
                   out_bf16=False, offsets=None, bound=None):
    """Bit-exact for int and max; S_j-relative bound for float add."""
    if offsets is None:
        want = oracle.scan(op, dtype, x_np, inclusive)
    else:
        want = oracle.segscan(op, dtype, x_np, offsets, inclusive)
    if op == "max" or dtype in ("i32", "i64"):
        if dtype == "f32":
            got_b, want_b = got.view(np.uint32), want.view(np.uint32)
        elif dtype == "f64":
            got_b, want_b = got.view(np.uint64), want.view(np.uint64)
        else:
            got_b, want_b = got, want
        if not np.array_equal(got_b, want_b):
            bad = np.flatnonzero(got_b != want_b)
            j = int(bad[0])
            raise AssertionError(
                f"{op}/{dtype} mismatch at {j} ({len(bad)} bad): "
                f"got {got[j]!r} want {want[j]!r}")
        return 0.0
    if offsets is None:
        s = oracle.abs_prefix(dtype, x_np, inclusive)
    else:
        s = oracle.abs_segprefix(dtype, x_np, offsets, inclusive)
    if out_bf16:
        from paper_1604_04815_gb300.workloads import bf16_bits_to_f32
        g = bf16_bits_to_f32(got).astype(np.float64)
    else:
        g = got.astype(np.float64)
    err = np.abs(g - want)
    c = BOUND[prec] if bound is None else bound
    if dtype == "f64" and bound is None:
        c = BOUND_F64_ADD
    lim = c * s
    if out_bf16:
        lim = lim + 2.0 ** -8 * np.abs(want)
    ok = err <= lim
    if not np.all(ok):
        j = int(np.flatnonzero(~ok)[0])
        raise AssertionError(
            f"{op}/{dtype}/{prec} bound broken at {j}: |err| {err[j]:.3e} > "
            f"{lim[j]:.3e} (S_j {s[j]:.3e}, ratio {err[j] / max(s[j], 1e-300):.3e})")
    pos = s > 0
    return float(np.max(err[pos] / s[pos])) if np.any(pos) else 0.0
