"""lscan_scan_noalloc: the scan entry point for callers that cannot allocate
device memory at the moment they scan (an allocator or memory pool servicing
a request, a framework that forbids allocations outside its pool, a latency-
critical path).  It must give the same results as lscan_scan, call after
call, using only the fixed scratch array compiled into the library.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process (its first
call then performs the one-time set-up)."""
import numpy as np
import pytest
import torch

from gpu_util import BOUND, LDT, LOP, to_device, to_host
from paper_1604_04815_gb300 import _lib
from paper_1604_04815_gb300.workloads import random_array

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_04815_gb300 import build
    build.build()
    _lib.load()


def _regular(op, dtype, xd, inclusive):
    y = torch.empty_like(xd)
    s = torch.cuda.current_stream().cuda_stream
    st = _lib.lscan_scan(LOP[op], LDT[dtype], int(inclusive), xd.data_ptr(),
                         y.data_ptr(), xd.shape[0], None, s)
    assert st == _lib.LSCAN_OK
    assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
    return to_host(y)


def _noalloc(op, dtype, xd, inclusive):
    y = torch.empty_like(xd)
    s = torch.cuda.current_stream().cuda_stream
    st = _lib.lscan_scan_noalloc(LOP[op], LDT[dtype], int(inclusive),
                                 xd.data_ptr(), y.data_ptr(), xd.shape[0], s)
    assert st == _lib.LSCAN_OK, _lib.strerror(st)
    torch.cuda.synchronize()
    return to_host(y)


@pytest.mark.parametrize("op,dtype,n", [("add", "i32", (1 << 22) + 5),
                                        ("max", "i32", 100003),
                                        ("add", "f32", (1 << 21) + 9)])
def test_noalloc_matches_regular_twice(op, dtype, n):
    import oracle
    rng = np.random.default_rng(40 + n % 97)
    x = random_array(dtype, n, rng,
                     kind="full" if dtype == "i32" else "signed")
    xd = to_device(x, dtype)
    for inclusive in (True, False):
        ref = _regular(op, dtype, xd, inclusive)
        for _ in range(2):  # two calls in a row share the fixed scratch
            got = _noalloc(op, dtype, xd, inclusive)
            if dtype == "i32":
                assert np.array_equal(got, ref)
            else:
                s = oracle.abs_prefix(dtype, x, inclusive)
                err = np.abs(got.astype(np.float64) - ref.astype(np.float64))
                assert np.all(err <= 2 * BOUND["f64"] * s)


def test_noalloc_rejects_sizes_beyond_fixed_scratch():
    # 2^40 int32 elements need far more status words than the array holds;
    # the call must refuse before touching the (never allocated) pointers.
    s = torch.cuda.current_stream().cuda_stream
    big = 1 << 40
    st = _lib.lscan_scan_noalloc(_lib.LSCAN_ADD, _lib.LSCAN_I32, 1, 1 << 20,
                                 1 << 50, big, s)
    assert st == _lib.LSCAN_ERR_INVALID
    assert _lib.lscan_scan_noalloc(_lib.LSCAN_ADD, _lib.LSCAN_I32, 1, 0, 0, 0,
                                   s) == _lib.LSCAN_OK
