"""Parity at the full single-array sizes (N = 2^28) in the launch
configuration bench.py times (default tuned tile configuration, decoupled
look-back, double-float carry for fp32 add): every output element is compared
with the oracle, which finishes a 2^28 scan in about a second.  Beyond 2^31
elements, where a 32-bit element index would overflow, the outputs are
checked on the device against properties that hold at any size."""
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


@pytest.mark.parametrize("op", ["add", "max"])
def test_beyond_2_31_elements(op):
    """N = 2^31 + 4099 int32 elements (about 8.6 GB per array): the add-scan
    of all ones is y_j = j + 1 modulo 2^32 (it passes 2^31 and wraps), and
    the max-scan of a non-decreasing array is the array itself.  Every
    element is compared on the device."""
    from paper_1604_04815_gb300 import build
    build.build()
    n = (1 << 31) + 4099
    if op == "add":
        xd = torch.ones(n, dtype=torch.int32, device="cuda")
        want = torch.arange(1, n + 1, dtype=torch.int64, device="cuda")
        want = want.to(torch.int32)  # two's-complement wrap, as modulo 2^32
    else:
        want = (torch.arange(n, dtype=torch.int64, device="cuda") // 3).to(torch.int32)
        xd = want.clone()
    y = run_c_abi(op, "i32", xd, True)
    assert torch.equal(y, want)
    del xd, y, want
    torch.cuda.empty_cache()
