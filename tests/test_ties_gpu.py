"""GPU parity of the max tie rule: max(a, b) = b > a ? b : a with a the
earlier element, so a tie keeps the earlier element's bits, and +0 and -0
compare equal (the paper leaves ties open; the definition of scan in
Section 1 only needs an associative operator, and this rule is one).

Under max, equal values differ in their bits only for +0 and -0, so every
input here is drawn from small pools in which the running maximum is a zero
for long stretches (workloads.ties_array): the output bits then show whether
the kernel kept the first zero.  The kernels carry tile and element indices
through the reducer and the look-back only for this rule; these tests put
the deciding zeros on both sides of tile boundaries, across many look-back
windows, through both carry protocols, every tile configuration, the
single-CTA kernel, batched segments, a carry-in and the server.  Every output
is compared bit for bit with the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1604_04815_gb300 as lscan
from gpu_util import (assert_matches, run_c_abi, to_device, to_host, LDT, LOP,
                      TEST_WAIT_NS)
from paper_1604_04815_gb300 import _lib
from paper_1604_04815_gb300.workloads import (f32_to_bf16_bits, ties_array,
                                              offsets_from_lengths)

pytestmark = pytest.mark.gpu

DTYPES = ["f32", "bf16", "f64"]
TDT = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_04815_gb300 import build
    build.build()
    _lib.load()
    _lib.lscan_set_wait_limit_ns(TEST_WAIT_NS)
    yield


def _bits(a):
    return a.view({2: np.uint16, 4: np.uint32, 8: np.uint64}[a.itemsize])


def _tile(config, dtype):
    return _lib.lscan_config_info(config, LDT[dtype])["tile"]


def _cases(tile, rng):
    """(pattern, n, first_zero): the first zero just before, at and after a
    tile boundary, deep in a long array, and zeros everywhere."""
    return [("zeros", tile - 1, tile - 2),
            ("zeros", tile, tile - 1),
            ("zeros", 2 * tile, tile),
            ("zeros", 7 * tile + 123, 3 * tile - 1),
            ("all_zeros", 7 * tile + 123, 0),
            ("repeated", 3 * tile + 5, 0),
            ("zeros", (1 << 22) + 17, int(rng.integers(1 << 21, 1 << 22)))]


@pytest.mark.parametrize("inclusive", [True, False], ids=["incl", "excl"])
@pytest.mark.parametrize("dtype", DTYPES)
def test_ties_every_config(dtype, inclusive):
    """Every tile configuration with the look-back, configuration 2 with
    the chained carry."""
    rng = np.random.default_rng(41)
    runs = [(c, _lib.LSCAN_CARRY_LOOKBACK)
            for c in range(1, _lib.lscan_num_configs() + 1)]
    runs.append((2, _lib.LSCAN_CARRY_CHAINED))
    for config, carry in runs:
        for pattern, n, fz in _cases(_tile(config, dtype), rng):
            if carry == _lib.LSCAN_CARRY_CHAINED and n > (1 << 20):
                continue
            # a low zero rate puts a few zeros in every tile, so that tile
            # aggregates with both signs meet in the look-back
            x = ties_array(dtype, n, rng, pattern, first_zero=fz,
                           p_zero=4.0 / _tile(config, dtype))
            y = run_c_abi("max", dtype, to_device(x, dtype), inclusive,
                          config=config, carry=carry)
            assert_matches("max", dtype, x, to_host(y), inclusive)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_ties_swizzled_tile_order(dtype):
    """Full tiles of a single array sit in shared memory with their 16-byte
    chunks swizzled by row (a row is one thread's elements), and the fp32 /
    bf16 max reducer searches a tile whose maximum is a zero for its first
    zero.  Here a -0 opens row 4 of tile 1 and a +0 sits in a later chunk of
    the same row that the swizzle places before it in shared memory: element
    order and shared-memory order disagree, and only element order gives -0
    as the tile's total and as every later output."""
    isz = 2 if dtype == "bf16" else 4
    epc = 16 // isz
    for config in range(1, _lib.lscan_num_configs() + 1):
        info = _lib.lscan_config_info(config, LDT[dtype])
        tile, items = info["tile"], info["items"]
        rb = items * isz                       # row bytes
        chunks = max(rb // 16, 1)              # 16-byte chunks per row

        def phys(b):                           # the 128-byte swizzle
            return b ^ (((b >> 7) & 7) << 4)
        base = 4 * rb                          # row 4
        ahead = [j for j in range(1, chunks) if phys(base + 16 * j) < phys(base)]
        later = ahead[0] if ahead else 1       # (16-byte rows: the next row)
        n = 3 * tile
        x = np.full(n, -1.0, dtype=np.float32)
        first = tile + 4 * items
        second = first + later * epc
        x[first] = -0.0
        x[second] = 0.0
        if dtype == "bf16":
            x = f32_to_bf16_bits(x)
        for inclusive in (True, False):
            y = run_c_abi("max", dtype, to_device(x, dtype), inclusive,
                          config=config)
            got = to_host(y)
            assert_matches("max", dtype, x, got, inclusive)
            # the zero after both is -0's bits
            assert _bits(got[-1:])[0] == _bits(_neg_zero(dtype))[0], (config, inclusive)


@pytest.mark.parametrize("dtype", DTYPES)
def test_ties_plain_load_path(dtype):
    """Unaligned x and y (the plain-load variant) on tie-heavy input."""
    rng = np.random.default_rng(42)
    n = 3 * 4096 + 77
    x = ties_array(dtype, n, rng, "zeros", first_zero=4095, p_zero=0.001)
    xd = to_device(x, dtype, pad_front=1)
    yb = torch.empty(n + 1, dtype=TDT[dtype], device="cuda")
    y = run_c_abi("max", dtype, xd, True, y_dev=yb[1:])
    assert_matches("max", dtype, x, to_host(y), True)


@pytest.mark.parametrize("dtype", DTYPES)
def test_ties_tiny_kernel(dtype):
    """The single-CTA kernel (n <= 4096, configuration left to the library)."""
    rng = np.random.default_rng(43)
    for pattern, n, fz in (("zeros", 1, 0), ("all_zeros", 2, 0),
                           ("zeros", 1000, 500), ("all_zeros", 4096, 0),
                           ("zeros", 4096, 4095), ("repeated", 3000, 0)):
        x = ties_array(dtype, n, rng, pattern, first_zero=fz, p_zero=0.01)
        for inclusive in (True, False):
            before = _lib.lscan_launch_count()
            y = run_c_abi("max", dtype, to_device(x, dtype), inclusive)
            assert _lib.lscan_launch_count() == before + 1
            assert_matches("max", dtype, x, to_host(y), inclusive)


@pytest.mark.parametrize("dtype", DTYPES)
def test_ties_batched_segments(dtype):
    """Segments whose first zeros sit on both sides of tile boundaries; the
    carry restarts at every segment head."""
    rng = np.random.default_rng(44)
    lens = [1, 0, 4095, 4096, 4097, 2, 30000, 0, 8191, 12345, 3]
    off = offsets_from_lengths(lens)
    n = int(off[-1])
    x = ties_array(dtype, n, rng, "zeros", first_zero=0, p_zero=0.002)
    xd = to_device(x, dtype)
    od = torch.from_numpy(off).cuda()
    s = torch.cuda.current_stream().cuda_stream
    for config in (1, 2, 3):
        for inclusive in (True, False):
            y = torch.empty(n, dtype=TDT[dtype], device="cuda")
            opts = _lib.make_options(config=config)
            st = _lib.lscan_batched(LOP["max"], LDT[dtype], int(inclusive),
                                    xd.data_ptr(), y.data_ptr(), od.data_ptr(),
                                    len(off) - 1, n, opts, s)
            assert st == _lib.LSCAN_OK
            assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
            assert_matches("max", dtype, x, to_host(y), inclusive,
                           offsets=off)


def _neg_zero(dtype):
    if dtype == "bf16":
        return np.array([0x8000], dtype=np.uint16)
    return np.array([-0.0], dtype=np.float32 if dtype == "f32" else np.float64)


def _pos_zero(dtype):
    if dtype == "bf16":
        return np.array([0x0000], dtype=np.uint16)
    return np.array([0.0], dtype=np.float32 if dtype == "f32" else np.float64)


@pytest.mark.parametrize("dtype", DTYPES)
def test_ties_carry_in(dtype):
    """A carry-in is an element placed in front of x_0: against a zero of
    the other sign it wins the tie, so the oracle's scan of [c] + x, first
    output dropped, is the expected result."""
    rng = np.random.default_rng(45)
    s = torch.cuda.current_stream().cuda_stream
    tile = _tile(2, dtype)
    for c in (_neg_zero(dtype), _pos_zero(dtype)):
        for pattern, n in (("all_zeros", 1), ("all_zeros", 3 * tile + 9),
                           ("zeros", 5 * tile + 1)):
            x = ties_array(dtype, n, rng, pattern, first_zero=0, p_zero=0.01)
            for config, carry in ((0, 0), (2, 0),
                                  (2, _lib.LSCAN_CARRY_CHAINED)):
                for inclusive in (True, False):
                    ca = c.view(np.int16) if dtype == "bf16" else c
                    cdev = torch.from_numpy(ca.copy()).cuda().view(TDT[dtype])
                    xd = to_device(x, dtype)
                    y = torch.empty(n, dtype=TDT[dtype], device="cuda")
                    opts = _lib.make_options(config=config, carry=carry,
                                             carry_in=cdev.data_ptr())
                    st = _lib.lscan_scan(LOP["max"], LDT[dtype],
                                         int(inclusive), xd.data_ptr(),
                                         y.data_ptr(), n, opts, s)
                    assert st == _lib.LSCAN_OK
                    assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
                    full = np.concatenate([c, x])
                    want = oracle.scan("max", dtype, full, inclusive)[1:]
                    if not inclusive:
                        # exclusive y_0 = the carry-in; y_j = c (+) x_0..x_{j-1}
                        want = oracle.scan("max", dtype, full, True)[:-1]
                    got = to_host(y)
                    assert np.array_equal(_bits(got), _bits(want)), \
                        (dtype, pattern, n, config, carry, inclusive)


def test_ties_server_mix():
    """Tie-heavy float max requests batched with other kinds by the server:
    each result equals the oracle bit for bit."""
    rng = np.random.default_rng(46)
    reqs = []
    for i in range(36):
        dtype = DTYPES[i % 3]
        n = int(rng.choice([1, 777, 4096, 4097, 20000, 70001]))
        pattern = ["zeros", "all_zeros", "repeated"][(i // 3) % 3]
        x = ties_array(dtype, n, rng, pattern, first_zero=int(n // 2),
                       p_zero=0.001)
        reqs.append((dtype, x, bool(i % 4)))
    # other kinds in the same burst
    fill = [("i32", rng.integers(-9, 9, size=50000, dtype=np.int32), True),
            ("f32", rng.random(size=30000, dtype=np.float32), True)]
    srv = lscan.Server(budget_bytes=1 << 30, n_streams=2)
    try:
        xs = [to_device(x, d) for d, x, _ in reqs]
        fx = [to_device(x, d) for d, x, _ in fill]
        ys = [torch.empty(x.shape[0], dtype=TDT[d], device="cuda")
              for d, x, _ in reqs]
        srv.hold(True)
        tks = [srv.submit(xd, "max", inc, out=y)
               for (d, x, inc), xd, y in zip(reqs, xs, ys)]
        ftk = [srv.submit(xd, "add", True) for xd in fx]
        srv.hold(False)
        stats = [srv.wait(tk) for tk in tks + ftk]
        assert all(st["status"] == 0 for st in stats)
        assert max(st["batch_requests"] for st in stats) > 1
        for (d, x, inc), y in zip(reqs, ys):
            assert_matches("max", d, x, to_host(y), inc)
        for tk in tks + ftk:
            srv.release(tk)
    finally:
        srv.close()
