"""The inter-block carry chain as a primitive (tile_chain.cuh): epoch-tagged
status slots, decoupled look-back and bounded waits, shared by the scan
kernel (and its stream-compaction kinds) and by the reduction of sharded
scans (lscan_reduce, whose CTAs' partials meet through the same slots).

The bounded wait is made to run out on the host's request: a block that
never publishes (lscan_debug_skip_publish), so the block that looks back
past it waits until the limit, the launch ends, the stream reports
LSCAN_ERR_TIMEOUT, and the next launch on the stream is correct."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import LDT, LOP, TEST_WAIT_NS, to_device, to_host, assert_matches
from paper_1604_04815_gb300 import _lib
from paper_1604_04815_gb300.workloads import random_array

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_04815_gb300 import build
    build.build()
    _lib.load()
    _lib.lscan_set_wait_limit_ns(TEST_WAIT_NS)
    yield
    _lib.lscan_set_wait_limit_ns(TEST_WAIT_NS)
    _lib.lscan_debug_skip_publish(-1)


def _reduce(x_dev, op, dtype, stream):
    t = torch.zeros(8, dtype=torch.uint8, device="cuda")
    st = _lib.lscan_reduce(LOP[op], LDT[dtype], x_dev.data_ptr(), x_dev.shape[0],
                           None, t.data_ptr(), stream)
    assert st == _lib.LSCAN_OK
    return t


@pytest.mark.parametrize("skip", [0, 1, 5])
def test_reduce_wait_runs_out_and_recovers(skip):
    """Block `skip` of the reduction never publishes its partial: the last
    block's look-back gives up after the wait limit."""
    s = torch.cuda.current_stream().cuda_stream
    x = random_array("i32", (1 << 22) + 3, np.random.default_rng(skip))
    xd = to_device(x, "i32")
    want = np.int32(oracle.scan("add", "i32", x, True)[-1]).view(np.uint32)
    assert _lib.lscan_set_wait_limit_ns(20_000_000) == _lib.LSCAN_OK
    try:
        _lib.lscan_debug_skip_publish(skip)
        _reduce(xd, "add", "i32", s)
        assert _lib.lscan_stream_status(s) == _lib.LSCAN_ERR_TIMEOUT
        assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK   # cleared
    finally:
        _lib.lscan_set_wait_limit_ns(TEST_WAIT_NS)
        _lib.lscan_debug_skip_publish(-1)
    t = _reduce(xd, "add", "i32", s)
    assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
    assert np.frombuffer(t.cpu().numpy().tobytes()[:4], dtype=np.uint32)[0] == want


def test_reduce_and_scan_share_the_stream_chain():
    """Reductions and scans alternate on one stream: both use its control
    block and status slots, each launch re-arms them for the next."""
    s = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(3)
    for i in range(6):
        n = int(rng.integers(1 << 16, 1 << 21))
        x = random_array("i32", n, rng, kind="full")
        xd = to_device(x, "i32")
        t = _reduce(xd, "add", "i32", s)
        y = torch.empty_like(xd)
        assert _lib.lscan_scan(LOP["add"], LDT["i32"], 1, xd.data_ptr(),
                               y.data_ptr(), n, None, s) == _lib.LSCAN_OK
        assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
        got = to_host(y)
        assert_matches("add", "i32", x, got)
        assert np.frombuffer(t.cpu().numpy().tobytes()[:4], dtype=np.int32)[0] == got[-1]


def test_scan_and_compaction_wait_runs_out_and_recovers():
    """The scan template's users of the chain: a tile that never publishes
    makes a scan and a stream compaction report the timeout; both are
    correct on the next launch."""
    import paper_1604_04815_gb300 as lscan
    s = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(9)
    n = 64 * 4096
    x = random_array("i32", n, rng, kind="full")
    flags = (rng.random(n) < 0.5).astype(np.uint8)
    xd = to_device(x, "i32")
    fd = torch.from_numpy(flags).cuda()
    assert _lib.lscan_set_wait_limit_ns(20_000_000) == _lib.LSCAN_OK
    try:
        _lib.lscan_debug_skip_publish(2)
        y = torch.empty_like(xd)
        _lib.lscan_scan(LOP["add"], LDT["i32"], 1, xd.data_ptr(), y.data_ptr(), n,
                        None, s)
        assert _lib.lscan_stream_status(s) == _lib.LSCAN_ERR_TIMEOUT
        _lib.lscan_debug_skip_publish(2)
        lscan.select_flagged(xd, fd)
        assert _lib.lscan_stream_status(s) == _lib.LSCAN_ERR_TIMEOUT
    finally:
        _lib.lscan_set_wait_limit_ns(TEST_WAIT_NS)
        _lib.lscan_debug_skip_publish(-1)
    y = torch.empty_like(xd)
    assert _lib.lscan_scan(LOP["add"], LDT["i32"], 1, xd.data_ptr(), y.data_ptr(),
                           n, None, s) == _lib.LSCAN_OK
    assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
    assert_matches("add", "i32", x, to_host(y))
    out, count = lscan.select_flagged(xd, fd)
    lscan.stream_status()
    k = int(count.item())
    assert np.array_equal(to_host(out)[:k], oracle.select_flagged(x, flags))
