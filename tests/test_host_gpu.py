"""GPU parity of lscan_scan_host (arrays in host memory, scanned in chunks
that pass through device slots): every kind, inclusive and exclusive, chunk
sizes that split tiles and a ragged last chunk, chunks small enough for the
single-CTA kernel, in-place, pageable host memory, a carry-in and repeated
calls that grow the slots -- all against the CPU oracle, with the same
bounds as the device-resident scans (the chunk totals are handed on in the
carry type, so chunking adds no rounding)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import (DTYPES, LDT, LOP, PREC_CODE, TEST_WAIT_NS, assert_matches,
                      out_torch_dtype)
from paper_1604_04815_gb300 import _lib
from paper_1604_04815_gb300.workloads import random_array

pytestmark = pytest.mark.gpu

KINDS = [
    ("add", "i32", None, False),
    ("max", "i32", None, False),
    ("max", "f32", None, False),
    ("max", "bf16", None, False),
    ("add", "f32", "plain", False),
    ("add", "f32", "f64", False),
    ("add", "f32", "comp", False),
    ("add", "bf16", "f64", False),
    ("add", "bf16", "comp", False),
    ("add", "bf16", "f64", True),
    ("add", "i64", None, False),
    ("max", "i64", None, False),
    ("max", "f64", None, False),
    ("add", "f64", None, False),
]
KIND_IDS = [f"{o}-{d}-{p or 'exact'}{'-bf16out' if b else ''}"
            for o, d, p, b in KINDS]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_04815_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    _lib.load()
    _lib.lscan_set_wait_limit_ns(TEST_WAIT_NS)
    yield


def _input(op, dtype, n, seed):
    rng = np.random.default_rng(seed)
    if dtype in ("i32", "i64"):
        return random_array(dtype, n, rng, kind="full" if op == "max" else "uniform")
    return random_array(dtype, n, rng, kind="signed")


def _host_tensor(x_np, dtype, pinned=True):
    if dtype == "bf16":
        t = torch.from_numpy(x_np.view(np.int16).copy()).view(torch.bfloat16)
    else:
        t = torch.from_numpy(np.ascontiguousarray(x_np).copy())
    return t.pin_memory() if pinned else t


def _to_np(t):
    if t.dtype == torch.bfloat16:
        return t.view(torch.int16).numpy().view(np.uint16)
    return t.numpy()


def _scan_host(op, dtype, prec, ob, hx, hy, inclusive, chunk, carry_in=None):
    n = hx.shape[0]
    opts = _lib.make_options(out_dtype=_lib.LSCAN_BF16 if ob else 0,
                             precision=PREC_CODE[prec] if prec else 0,
                             carry_in=carry_in)
    s = torch.cuda.current_stream().cuda_stream
    st = _lib.lscan_scan_host(LOP[op], LDT[dtype], int(inclusive), hx.data_ptr(),
                              hy.data_ptr(), n, opts, chunk, s)
    assert st == _lib.LSCAN_OK, _lib.strerror(st)
    torch.cuda.current_stream().synchronize()
    assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK


@pytest.mark.parametrize("inclusive", [True, False], ids=["incl", "excl"])
@pytest.mark.parametrize("kind", KINDS, ids=KIND_IDS)
def test_chunked_matches_oracle(kind, inclusive):
    op, dtype, prec, ob = kind
    # (n, chunk): chunks that split tiles with a ragged last chunk, chunks
    # for the single-CTA kernel, one chunk larger than n, and the default
    # schedule (one chunk, then chunks ramping up from 2^20 and down again)
    for i, (n, chunk) in enumerate([(47123, 10000), (10001, 3000), (777, 5000),
                                    (1, 0), (65537, 0),
                                    (3 * 2 ** 20 + 12345, 0)]):
        x = _input(op, dtype, n, seed=900 + i)
        hx = _host_tensor(x, dtype)
        hy = torch.empty(n, dtype=out_torch_dtype(op, dtype, ob)).pin_memory()
        _scan_host(op, dtype, prec, ob, hx, hy, inclusive, chunk)
        assert_matches(op, dtype, x, _to_np(hy), inclusive, prec or "f64",
                       out_bf16=ob)


@pytest.mark.parametrize("kind", [("add", "i32"), ("max", "f32"), ("add", "f64")])
def test_in_place_host(kind):
    op, dtype = kind
    n = 100003
    x = _input(op, dtype, n, seed=31)
    h = _host_tensor(x, dtype)
    _scan_host(op, dtype, None, False, h, h, True, 16384)
    assert_matches(op, dtype, x, _to_np(h), True, "f64")


def test_pageable_host_memory():
    n = 50000
    x = _input("add", "i32", n, seed=32)
    hx = _host_tensor(x, "i32", pinned=False)
    hy = torch.empty(n, dtype=torch.int32)
    _scan_host("add", "i32", None, False, hx, hy, False, 8192)
    assert_matches("add", "i32", x, hy.numpy(), False)


@pytest.mark.parametrize("inclusive", [True, False], ids=["incl", "excl"])
def test_carry_in_starts_chunk_zero(inclusive):
    n = 30000
    x = _input("add", "i32", n, seed=33)
    c = np.int32(-123456789)
    cdev = torch.tensor([int(c)], dtype=torch.int32, device="cuda")
    hx = _host_tensor(x, "i32")
    hy = torch.empty(n, dtype=torch.int32).pin_memory()
    _scan_host("add", "i32", None, False, hx, hy, inclusive, 7000,
               carry_in=cdev.data_ptr())
    want = (oracle.scan("add", "i32", x, inclusive).view(np.uint32) +
            np.uint32(int(c) % 2**32)).view(np.int32)
    assert np.array_equal(hy.numpy(), want)


def test_repeated_calls_grow_slots_and_keep_order():
    """Several calls back to back on one stream, with chunk sizes and element
    sizes that make the device slots grow between calls, and no
    synchronisation in between: each result must still be its own scan."""
    s = torch.cuda.current_stream().cuda_stream
    jobs = []
    for i, (op, dtype, n, chunk) in enumerate([("add", "i32", 40000, 4096),
                                               ("max", "i64", 90000, 30000),
                                               ("add", "i32", 200000, 65536),
                                               ("add", "f32", 120000, 20000)]):
        x = _input(op, dtype, n, seed=40 + i)
        hx = _host_tensor(x, dtype)
        hy = torch.empty(n, dtype=DTYPES[dtype]).pin_memory()
        st = _lib.lscan_scan_host(LOP[op], LDT[dtype], 1, hx.data_ptr(),
                                  hy.data_ptr(), n, None, chunk, s)
        assert st == _lib.LSCAN_OK
        jobs.append((op, dtype, x, hx, hy))
    torch.cuda.current_stream().synchronize()
    assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
    for op, dtype, x, _, hy in jobs:
        assert_matches(op, dtype, x, hy.numpy(), True, "f64")


def test_work_queued_after_sees_the_output():
    """A copy queued on the stream after the call reads the finished host
    output (the call joins its copy-outs back into the stream)."""
    n = 300000
    x = _input("add", "i32", n, seed=50)
    hx = _host_tensor(x, "i32")
    hy = torch.empty(n, dtype=torch.int32).pin_memory()
    s = torch.cuda.current_stream().cuda_stream
    st = _lib.lscan_scan_host(LOP["add"], LDT["i32"], 1, hx.data_ptr(),
                              hy.data_ptr(), n, None, 32768, s)
    assert st == _lib.LSCAN_OK
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    d.copy_(hy, non_blocking=True)
    got = d.cpu().numpy()
    assert np.array_equal(got, oracle.scan("add", "i32", x, True))


def test_torch_front_scan_host():
    """paper_1604_04815_gb300.scan_host: CPU tensors in and out, bf16 add
    writing fp32, and the in-place form."""
    import paper_1604_04815_gb300 as lscan
    n = 70001
    xb = _input("add", "bf16", n, seed=60)
    hb = _host_tensor(xb, "bf16")
    yb = lscan.scan_host(hb, chunk=20000)
    assert yb.dtype == torch.float32 and not yb.is_cuda
    assert_matches("add", "bf16", xb, yb.numpy(), True, "f64")
    xi = _input("max", "i32", n, seed=61)
    hi = _host_tensor(xi, "i32")
    out = lscan.scan_host(hi, op="max", inclusive=False, out=hi, chunk=9000)
    assert out.data_ptr() == hi.data_ptr()
    assert_matches("max", "i32", xi, hi.numpy(), False)
    with pytest.raises(TypeError):
        lscan.scan_host(hi.cuda())
