"""Parity at the full single-array sizes (N = 2^28) in the launch
configuration bench.py times (default tuned tile configuration, decoupled
look-back, FP64 carry for fp32 add): every output element is compared with the
oracle, which finishes a 2^28 scan in about a second."""
import numpy as np
import pytest
import torch

from gpu_util import assert_matches, run_c_abi, to_device, to_host
from paper_1604_04815_gb300 import workloads

pytestmark = pytest.mark.gpu

N = 1 << 28


@pytest.mark.parametrize("case", ["i32_add", "i32_max", "f32_add"])
def test_full_size(case):
    from paper_1604_04815_gb300 import build
    build.build()
    if case == "i32_add":
        op, dtype, x = "add", "i32", workloads.large_i32_add(N)
    elif case == "i32_max":
        op, dtype, x = "max", "i32", workloads.large_i32_max(N)
    else:
        op, dtype, x = "add", "f32", workloads.large_f32_add(N)
    xd = to_device(x, dtype)
    y = run_c_abi(op, dtype, xd, True)
    got = to_host(y)
    del xd, y
    torch.cuda.empty_cache()
    ratio = assert_matches(op, dtype, x, got, True, "f64")
    if op == "add" and dtype == "f32":
        print(f"fp32 add N=2^28 max err/S_j = {ratio:.3e}")


@pytest.mark.parametrize("case", ["i32_add", "i32_max", "f32_add"])
def test_full_size_from_host(case):
    """The same arrays from pinned host memory through lscan_scan_host with
    the default chunking, as bench.py's end-to-end leg runs them."""
    from paper_1604_04815_gb300 import _lib, build
    from gpu_util import LDT, LOP
    build.build()
    if case == "i32_add":
        op, dtype, x = "add", "i32", workloads.large_i32_add(N)
    elif case == "i32_max":
        op, dtype, x = "max", "i32", workloads.large_i32_max(N)
    else:
        op, dtype, x = "add", "f32", workloads.large_f32_add(N)
    hx = torch.from_numpy(x).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    s = torch.cuda.current_stream().cuda_stream
    st = _lib.lscan_scan_host(LOP[op], LDT[dtype], 1, hx.data_ptr(),
                              hy.data_ptr(), N, None, 0, s)
    assert st == _lib.LSCAN_OK
    torch.cuda.current_stream().synchronize()
    assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
    got = hy.numpy().copy()
    del hx, hy
    assert_matches(op, dtype, x, got, True, "f64")


@pytest.mark.parametrize("dtype", ["i32", "f32"])
def test_full_size_batched_graph(dtype):
    """The batched workload bench.py times: 4096 arrays with log-uniform
    lengths in [1, 2^20] (3.1e8 elements) in one persistent segmented launch
    replayed from a CUDA graph; every element against the oracle after the
    second replay (each replay re-arms its own scratch)."""
    import paper_1604_04815_gb300 as lscan
    x, off = workloads.batched(dtype)
    xd = torch.from_numpy(x).cuda()
    od = torch.from_numpy(off).cuda()
    yd = torch.empty_like(xd)
    g = lscan.Graph.batched(xd, od, yd)
    for _ in range(2):
        g.launch()
    torch.cuda.synchronize()
    g.status()
    got = yd.cpu().numpy()
    g.close()
    del xd, od, yd
    torch.cuda.empty_cache()
    assert_matches("add", dtype, x, got, True, "f64", offsets=off)


def test_full_size_select():
    """Stream compaction as bench.py times it: 2^28 int32 values, byte flags,
    about half kept; compared with the oracle's compaction."""
    import oracle
    import paper_1604_04815_gb300 as lscan
    rng = np.random.default_rng(11)
    x = rng.integers(-1000, 1001, size=N, dtype=np.int32)
    f = (rng.random(N) < 0.5).astype(np.uint8)
    xd = torch.from_numpy(x).cuda()
    fd = torch.from_numpy(f).cuda()
    out, count = lscan.select_flagged(xd, fd)
    k = int(count.item())
    lscan.stream_status()
    want = oracle.select_flagged(x, f)
    assert k == want.shape[0]
    assert np.array_equal(out[:k].cpu().numpy(), want)
