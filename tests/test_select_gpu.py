"""Stream compaction (lscan_select_flagged): the fused scan consumer against
the oracle's plain loop, bit for bit, with the count."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import DTYPES, LDT, to_device, to_host
from paper_1604_04815_gb300 import _lib
from paper_1604_04815_gb300.workloads import random_array

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_04815_gb300 import build
    build.build()
    _lib.load()


def _run(dtype, x_dev, f_dev, y_dev, n):
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    st = _lib.lscan_select_flagged(LDT[dtype], x_dev.data_ptr(),
                                   f_dev.data_ptr(), y_dev.data_ptr(), n,
                                   cnt.data_ptr(), s)
    assert st == _lib.LSCAN_OK, _lib.strerror(st)
    assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
    return int(cnt.item())


def _flags(n, p_keep, rng):
    keep = rng.random(n) < p_keep
    return (keep * rng.integers(1, 256, size=n)).astype(np.uint8)


@pytest.mark.parametrize("p_keep", [0.0, 0.03, 0.5, 1.0])
@pytest.mark.parametrize("dtype", ["i32", "f32", "bf16", "i64", "f64"])
def test_select_matches_oracle(dtype, p_keep):
    rng = np.random.default_rng(int(p_keep * 1000) + len(dtype))
    for n in (1, 1000, 4095, 4096, 4097, 10 * 4096 + 123, (1 << 20) + 7):
        x = random_array(dtype, n, rng, kind="full" if dtype in ("i32", "i64")
                         else "signed")
        f = _flags(n, p_keep, rng)
        want = oracle.select_flagged(x, f)
        xd = to_device(x, dtype)
        fd = torch.from_numpy(f).cuda()
        yd = torch.empty_like(xd)
        k = _run(dtype, xd, fd, yd, n)
        assert k == want.shape[0], (n, k, want.shape[0])
        got = to_host(yd)[:k]
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), n


def test_select_unaligned_and_empty():
    rng = np.random.default_rng(5)
    n = 3 * 4096 + 77
    x = random_array("f32", n, rng, kind="signed")
    f = _flags(n, 0.4, rng)
    want = oracle.select_flagged(x, f)
    xd = to_device(x, "f32", pad_front=1)            # values not 16-B aligned
    fb = torch.empty(n + 3, dtype=torch.uint8, device="cuda")
    fb[3:] = torch.from_numpy(f)
    fd = fb[3:]                                      # flags not 16-B aligned
    yb = torch.empty(n + 1, dtype=torch.float32, device="cuda")
    k = _run("f32", xd, fd, yb[1:], n)
    assert k == want.shape[0]
    assert np.array_equal(to_host(yb[1:])[:k].view(np.uint32),
                          want.view(np.uint32))
    # n = 0 writes a zero count and launches nothing
    before = _lib.lscan_launch_count()
    assert _run("f32", xd, fd, yb, 0) == 0
    assert _lib.lscan_launch_count() == before
    # y may not overlap x or the flags
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    assert _lib.lscan_select_flagged(LDT["f32"], xd.data_ptr(), fd.data_ptr(),
                                     xd.data_ptr(), n, cnt.data_ptr(),
                                     None) == _lib.LSCAN_ERR_INVALID


def test_select_torch_front():
    import paper_1604_04815_gb300 as lscan
    x = torch.arange(100000, dtype=torch.int64, device="cuda")
    flags = (x % 3 == 0)
    out, count = lscan.select_flagged(x, flags)
    k = int(count.item())
    assert k == 33334
    assert torch.equal(out[:k], x[x % 3 == 0])


@pytest.mark.parametrize("dtype", ["i32", "bf16", "i64"])
def test_select_each_load_variant(dtype):
    """Flags and values each 16-byte aligned or not: plain loads (flags
    unaligned), flags by bulk copy with values loaded into registers (values
    unaligned), and both through the bulk-copy ring (both aligned), with a
    ragged last tile whose values are copied by the lanes."""
    rng = np.random.default_rng(17)
    esz = np.dtype(np.uint16 if dtype == "bf16" else
                   np.int32 if dtype == "i32" else np.int64).itemsize
    for n in (4096 + 5, 16384 + 5, 5 * 16384 + 13, (1 << 18) + 3):
        x = random_array(dtype, n, rng, kind="full" if dtype != "bf16" else "signed")
        f = _flags(n, 0.45, rng)
        want = oracle.select_flagged(x, f)
        for f_pad in (0, 5):
            for x_pad in (0, 1):
                xd = to_device(x, dtype, pad_front=x_pad)
                assert (xd.data_ptr() % 16 == 0) == (x_pad == 0) or esz * x_pad % 16 == 0
                fb = torch.empty(n + f_pad, dtype=torch.uint8, device="cuda")
                fb[f_pad:] = torch.from_numpy(f)
                yd = torch.empty_like(xd)
                k = _run(dtype, xd, fb[f_pad:], yd, n)
                assert k == want.shape[0], (n, f_pad, x_pad)
                got = to_host(yd)[:k]
                assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (n, f_pad, x_pad)
