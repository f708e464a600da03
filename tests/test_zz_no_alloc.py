"""lscan_scan_noalloc: the scan entry point for callers that cannot allocate
device memory at the moment they scan (an allocator or memory pool servicing
a request, a framework that forbids allocations outside its pool, a latency-
critical path).  Its results must match the oracle and lscan_scan, call after
call, using only the fixed scratch array compiled into the library; it must
not change the device's free memory; its size limit must sit exactly where
include/lscan.h puts it; and a device wait that ran out must be reported by
lscan_noalloc_status.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process (each test
makes its own set-up call first)."""
import threading

import numpy as np
import pytest
import torch

import oracle
from gpu_util import (BOUND, LDT, LOP, TEST_WAIT_NS, assert_matches,
                      to_device, to_host)
from paper_1604_04815_gb300 import _lib
from paper_1604_04815_gb300.workloads import random_array

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_04815_gb300 import build
    build.build()
    _lib.load()
    _lib.lscan_set_wait_limit_ns(TEST_WAIT_NS)


def _stream_ptr(stream=None):
    return (stream or torch.cuda.current_stream()).cuda_stream


def _regular(op, dtype, xd, inclusive, stream=None):
    y = torch.empty_like(xd)
    s = _stream_ptr(stream)
    st = _lib.lscan_scan(LOP[op], LDT[dtype], int(inclusive), xd.data_ptr(),
                         y.data_ptr(), xd.shape[0], None, s)
    assert st == _lib.LSCAN_OK
    assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
    return y


def _noalloc(op, dtype, xd, inclusive, y=None, stream=None):
    y = torch.empty_like(xd) if y is None else y
    s = _stream_ptr(stream)
    st = _lib.lscan_scan_noalloc(LOP[op], LDT[dtype], int(inclusive),
                                 xd.data_ptr(), y.data_ptr(), xd.shape[0], s)
    assert st == _lib.LSCAN_OK, _lib.strerror(st)
    assert _lib.lscan_noalloc_status(s) == _lib.LSCAN_OK
    return y


def _input(op, dtype, n, seed):
    rng = np.random.default_rng(seed)
    return random_array(dtype, n, rng, kind="full" if dtype in ("i32", "i64")
                        else "signed")


@pytest.mark.parametrize("op,dtype,n", [("add", "i32", (1 << 22) + 5),
                                        ("max", "i32", 100003),
                                        ("add", "f32", (1 << 21) + 9),
                                        ("add", "i64", (1 << 20) + 77),
                                        ("max", "f32", 4096),     # one CTA
                                        ("add", "i32", 1000)])    # one CTA
def test_noalloc_matches_oracle_and_regular_twice(op, dtype, n):
    x = _input(op, dtype, n, seed=40 + n % 97)
    xd = to_device(x, dtype)
    for inclusive in (True, False):
        ref = to_host(_regular(op, dtype, xd, inclusive))
        for _ in range(2):  # two calls in a row share the fixed scratch
            got = to_host(_noalloc(op, dtype, xd, inclusive))
            assert_matches(op, dtype, x, got, inclusive, "df")
            if op == "max" or dtype in ("i32", "i64"):
                assert np.array_equal(got, ref)
            else:
                s = oracle.abs_prefix(dtype, x, inclusive)
                err = np.abs(got.astype(np.float64) - ref.astype(np.float64))
                assert np.all(err <= 2 * BOUND["df"] * s)


def test_noalloc_leaves_free_device_memory_unchanged():
    """After the documented set-up call, a call on a stream that never saw a
    scan allocates nothing: the device's free bytes are the same before and
    after (the regular entry point would allocate that stream's scratch)."""
    n = (1 << 22) + 3
    x = _input("add", "i32", n, seed=7)
    xd = to_device(x, "i32")
    y = torch.empty_like(xd)
    _noalloc("add", "i32", xd, True, y=y)        # set-up call (this kernel)
    fresh = torch.cuda.Stream()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        st = _lib.lscan_scan_noalloc(LOP["add"], LDT["i32"], 1, xd.data_ptr(),
                                     y.data_ptr(), n, fresh.cuda_stream)
        assert st == _lib.LSCAN_OK
    fresh.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert _lib.lscan_noalloc_status(fresh.cuda_stream) == _lib.LSCAN_OK
    assert_matches("add", "i32", x, to_host(y))


def test_noalloc_accepts_the_exact_limit():
    """2^29 int32 elements: 131072 tiles of 4096 with 2 status words each,
    exactly the 262144 words of the fixed array."""
    n = 1 << 29
    x = _input("add", "i32", n, seed=11)
    xd = to_device(x, "i32")
    y = _noalloc("add", "i32", xd, True)
    want = oracle.scan("add", "i32", x, True)
    assert np.array_equal(to_host(y), want)


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch():
    """2^40 int32 elements need far more status words than the array holds:
    refused on the host before the (never allocated) pointers are used.  The
    exact limits by type and alignment are checked without a GPU
    (tests/test_abi.py)."""
    s = _stream_ptr()
    assert _lib.lscan_scan_noalloc(LOP["add"], LDT["i32"], 1, 1 << 20, 1 << 50,
                                   1 << 40, s) == _lib.LSCAN_ERR_INVALID
    assert _lib.lscan_scan_noalloc(LOP["add"], LDT["i32"], 1, 0, 0, 0,
                                   s) == _lib.LSCAN_OK


def test_noalloc_status_reports_a_wait_that_ran_out():
    """A tile that never publishes (injected on the host): its successors'
    bounded waits run out, the call's launch ends, lscan_noalloc_status
    reports the timeout once, and the next call is correct."""
    s = _stream_ptr()
    n = 64 * 4096
    x = _input("add", "i32", n, seed=3)
    xd = to_device(x, "i32")
    y = torch.empty_like(xd)
    _noalloc("add", "i32", xd, True, y=y)        # set-up call
    assert _lib.lscan_set_wait_limit_ns(20_000_000) == _lib.LSCAN_OK
    try:
        _lib.lscan_debug_skip_publish(3)
        st = _lib.lscan_scan_noalloc(LOP["add"], LDT["i32"], 1, xd.data_ptr(),
                                     y.data_ptr(), n, s)
        assert st == _lib.LSCAN_OK
        assert _lib.lscan_noalloc_status(s) == _lib.LSCAN_ERR_TIMEOUT
        assert _lib.lscan_noalloc_status(s) == _lib.LSCAN_OK   # cleared
    finally:
        _lib.lscan_set_wait_limit_ns(TEST_WAIT_NS)
        _lib.lscan_debug_skip_publish(-1)
    y = _noalloc("add", "i32", xd, True, y=y)
    assert_matches("add", "i32", x, to_host(y))


def test_noalloc_beside_regular_calls_on_other_host_threads():
    """One host thread loops on lscan_scan_noalloc (one stream) while another
    loops on lscan_scan on a second stream: both share the library's launch
    caches; every result matches the oracle."""
    n = (1 << 20) + 11
    xa = _input("add", "i32", n, seed=21)
    xb = _input("max", "f32", n, seed=22)
    want_a = oracle.scan("add", "i32", xa, True)
    want_b = oracle.scan("max", "f32", xb, True)
    xad, xbd = to_device(xa, "i32"), to_device(xb, "f32")
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    ya = [torch.empty_like(xad) for _ in range(20)]
    yb = [torch.empty_like(xbd) for _ in range(20)]
    torch.cuda.synchronize()
    errors = []

    def run_noalloc():
        try:
            for y in ya:
                st = _lib.lscan_scan_noalloc(LOP["add"], LDT["i32"], 1,
                                             xad.data_ptr(), y.data_ptr(), n,
                                             sa.cuda_stream)
                assert st == _lib.LSCAN_OK
        except Exception as e:  # reported on the main thread
            errors.append(e)

    def run_regular():
        try:
            for y in yb:
                st = _lib.lscan_scan(LOP["max"], LDT["f32"], 1, xbd.data_ptr(),
                                     y.data_ptr(), n, None, sb.cuda_stream)
                assert st == _lib.LSCAN_OK
        except Exception as e:
            errors.append(e)

    ts = [threading.Thread(target=run_noalloc), threading.Thread(target=run_regular)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    assert _lib.lscan_noalloc_status(sa.cuda_stream) == _lib.LSCAN_OK
    assert _lib.lscan_stream_status(sb.cuda_stream) == _lib.LSCAN_OK
    for y in ya:
        assert np.array_equal(to_host(y), want_a)
    for y in yb:
        assert np.array_equal(to_host(y).view(np.uint32), want_b.view(np.uint32))
