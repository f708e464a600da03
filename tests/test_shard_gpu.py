"""Sharded scan on the GPU: 2-4 contiguous shards of one array scanned on
one device through the same C ABI calls a multi-GPU run makes (lscan_reduce
per shard, lscan_carry_combine of the lower shards' totals, lscan_scan with
that offset as a carry-type carry-in), minus only the collective that
would carry the 4- or 8-byte totals between devices.  The stitched result
must match the oracle's scan of the whole array: bit-exact for integers and
max, within each precision path's bound for float add.  The reduction alone
is checked against the oracle's total."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import (BOUND, BOUND_F64_ADD, LDT, LOP, PREC_CODE, TEST_WAIT_NS,
                      assert_matches, to_device, to_host)
from paper_1604_04815_gb300 import _lib
from paper_1604_04815_gb300.workloads import random_array, ties_array

pytestmark = pytest.mark.gpu

KINDS = [("add", "i32", None), ("max", "i32", None), ("max", "f32", None),
         ("max", "bf16", None), ("add", "f32", "plain"), ("add", "f32", "f64"),
         ("add", "f32", "df"), ("add", "f32", "comp"), ("add", "bf16", "df"),
         ("add", "bf16", "comp"), ("add", "i64", None), ("max", "i64", None),
         ("max", "f64", None), ("add", "f64", None)]
IDS = [f"{o}-{d}-{p or 'exact'}" for o, d, p in KINDS]
TDT = {"i32": torch.int32, "f32": torch.float32, "bf16": torch.bfloat16,
       "i64": torch.int64, "f64": torch.float64}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_04815_gb300 import build
    build.build()
    _lib.load()
    _lib.lscan_set_wait_limit_ns(TEST_WAIT_NS)


def _input(op, dtype, n, seed):
    rng = np.random.default_rng(seed)
    if op == "max" and dtype in ("f32", "bf16", "f64"):
        return ties_array(dtype, n, rng, "zeros", first_zero=n // 3,
                          p_zero=0.001)
    if dtype in ("i32", "i64"):
        return random_array(dtype, n, rng, kind="full")
    return random_array(dtype, n, rng, kind="signed")


def _sharded(op, dtype, prec, x, bounds, inclusive, config=0):
    """Scan x as len(bounds) - 1 shards; returns the stitched output."""
    s = torch.cuda.current_stream().cuda_stream
    opts = _lib.make_options(precision=PREC_CODE[prec] if prec else 0)
    nb = _lib.lscan_carry_bytes(LOP[op], LDT[dtype], opts)
    assert nb in (4, 8)
    xd = to_device(x, dtype)
    totals = []
    for g in range(len(bounds) - 1):          # 1. reduce each shard
        a, b = bounds[g], bounds[g + 1]
        t = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        assert _lib.lscan_reduce(LOP[op], LDT[dtype],
                                 xd.data_ptr() + a * xd.element_size(), b - a,
                                 opts, t.data_ptr(), s) == _lib.LSCAN_OK
        totals.append(t.cpu().numpy().tobytes())   # 2. (the all-gather)
    odt = torch.float32 if (op == "add" and dtype == "bf16") else TDT[dtype]
    y = torch.empty(x.shape[0], dtype=odt, device="cuda")
    for g in range(len(bounds) - 1):          # 3. offset, scan with carry-in
        a, b = bounds[g], bounds[g + 1]
        st, off = _lib.lscan_carry_combine(LOP[op], LDT[dtype],
                                           b"".join(totals[:g]), g, opts)
        assert st == _lib.LSCAN_OK
        cin = torch.frombuffer(bytearray(off), dtype=torch.uint8).cuda()
        so = _lib.make_options(precision=PREC_CODE[prec] if prec else 0,
                               carry_in=cin.data_ptr(), carry_in_type=1,
                               config=config)
        st = _lib.lscan_scan(LOP[op], LDT[dtype], int(inclusive),
                             xd.data_ptr() + a * xd.element_size(),
                             y.data_ptr() + a * y.element_size(), b - a, so, s)
        assert st == _lib.LSCAN_OK
        torch.cuda.synchronize()                   # cin stays alive
    assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
    return to_host(y)


@pytest.mark.parametrize("inclusive", [True, False], ids=["incl", "excl"])
@pytest.mark.parametrize("kind", KINDS, ids=IDS)
def test_sharded_matches_oracle(kind, inclusive):
    op, dtype, prec = kind
    n = 3 * 65536 + 4099
    for bounds in ([0, n // 2 + 7, n],                        # 2 shards
                   [0, 1000, 1000, 70001, n],                 # tiny, empty
                   [0, 4096, 12289, 100000, n]):              # 4 shards
        x = _input(op, dtype, n, seed=len(bounds) + n % 17)
        got = _sharded(op, dtype, prec, x, bounds, inclusive)
        assert_matches(op, dtype, x, got, inclusive, prec or "df")


def test_sharded_every_config_int32():
    """The carry-type carry-in through every tile configuration."""
    n = 5 * 16384 + 77
    x = _input("add", "i32", n, seed=5)
    for config in range(1, _lib.lscan_num_configs() + 1):
        got = _sharded("add", "i32", None, x, [0, 12345, n], True, config)
        assert np.array_equal(got, oracle.scan("add", "i32", x, True))


@pytest.mark.parametrize("kind", KINDS, ids=IDS)
def test_reduce_matches_oracle_total(kind):
    """lscan_reduce against the oracle's total: exact for integers and max
    (first occurrence of a zero maximum), within the bound for float add;
    unaligned starts and n = 0 (the identity)."""
    op, dtype, prec = kind
    s = torch.cuda.current_stream().cuda_stream
    opts = _lib.make_options(precision=PREC_CODE[prec] if prec else 0)
    nb = _lib.lscan_carry_bytes(LOP[op], LDT[dtype], opts)
    for n, pad in ((1, 0), (7, 1), (4097, 0), (1 << 20, 3), ((1 << 22) + 5, 0)):
        x = _input(op, dtype, n, seed=n)
        xd = to_device(x, dtype, pad_front=pad)
        t = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        assert _lib.lscan_reduce(LOP[op], LDT[dtype], xd.data_ptr(), n, opts,
                                 t.data_ptr(), s) == _lib.LSCAN_OK
        b = t.cpu().numpy().tobytes()
        want = oracle.scan(op, dtype, x, True)[-1]
        if op == "max" or dtype in ("i32", "i64"):
            w = np.array([want])
            if dtype == "f64":      # the carry is the order-preserving key
                k = int(np.frombuffer(b, dtype=np.int64)[0])
                bits = k ^ (0x7FFFFFFFFFFFFFFF if k < 0 else 0)
                assert bits == int(w.view(np.int64)[0])
            elif dtype == "f32":
                assert b == w.astype(np.float32).tobytes()
            elif dtype == "bf16":   # carried widened to fp32
                assert b == (w.astype(np.uint32) << 16).tobytes()
            else:                   # wrapping sums as unsigned, maxima signed
                assert b == w.astype(np.int32 if dtype == "i32" else
                                     np.int64).tobytes()
        else:
            if nb == 4:
                v = float(np.frombuffer(b, dtype=np.float32)[0])
            elif prec in ("f64",) or dtype == "f64":
                v = float(np.frombuffer(b, dtype=np.float64)[0])
            else:
                hi, lo = np.frombuffer(b, dtype=np.float32)
                v = float(hi) + float(lo)
            S = oracle.abs_prefix(dtype, x, True)[-1]
            c = BOUND_F64_ADD if dtype == "f64" else BOUND[prec]
            assert abs(v - float(want)) <= c * S + 1e-30, (n, v, want)
    # n = 0: the identity
    t = torch.full((nb,), 0x5A, dtype=torch.uint8, device="cuda")
    assert _lib.lscan_reduce(LOP[op], LDT[dtype], 0, 0, opts, t.data_ptr(),
                             s) == _lib.LSCAN_OK
    st, ident = _lib.lscan_carry_combine(LOP[op], LDT[dtype], b"", 0, opts)
    assert t.cpu().numpy().tobytes() == ident
