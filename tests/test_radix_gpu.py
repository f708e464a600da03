"""GPU parity of lscan_radix_offsets (radix-sort digit offsets: the histogram
of every digit position and its exclusive scan, in one pass over the keys)
against the CPU oracle, bit-exact: 32- and 64-bit keys, digit widths 1..8,
ragged and tiny sizes, unaligned keys (plain loads), skewed keys (shared-
memory atomics on one bucket), back-to-back launches that reuse the
scratch, n = 0, and the 2^28-key workload bench.py times."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TEST_WAIT_NS
from paper_1604_04815_gb300 import _lib

pytestmark = pytest.mark.gpu

N_FULL = 1 << 28


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_04815_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    _lib.load()
    _lib.lscan_set_wait_limit_ns(TEST_WAIT_NS)
    yield


def _keys(kdt, n, seed, kind="uniform"):
    rng = np.random.default_rng(seed)
    bits = 8 * np.dtype(kdt).itemsize
    if kind == "uniform":
        return rng.integers(0, 2 ** bits, size=n, dtype=kdt)
    if kind == "equal":
        return np.full(n, kdt(0x9E3779B97F4A7C15 % 2 ** bits), dtype=kdt)
    # a few distinct keys
    pool = rng.integers(0, 2 ** bits, size=3, dtype=kdt)
    return pool[rng.integers(0, 3, size=n)]


def _run(keys_np, digit_bits, pad_front=0):
    kb = keys_np.dtype.itemsize
    tdt = torch.int32 if kb == 4 else torch.int64
    sdt = np.int32 if kb == 4 else np.int64
    t = torch.from_numpy(keys_np.view(sdt).copy())
    if pad_front:
        buf = torch.empty(t.shape[0] + pad_front, dtype=tdt)
        buf[pad_front:] = t
        d = buf.cuda()[pad_front:]
    else:
        d = t.cuda()
    P = -(-8 * kb // digit_bits)
    out = torch.full((P, 1 << digit_bits), -7, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    st = _lib.lscan_radix_offsets(d.data_ptr(), kb, keys_np.shape[0], digit_bits,
                                  out.data_ptr(), s)
    assert st == _lib.LSCAN_OK, _lib.strerror(st)
    return out.cpu().numpy()


@pytest.mark.parametrize("kdt", [np.uint32, np.uint64], ids=["u32", "u64"])
@pytest.mark.parametrize("b", [1, 3, 4, 5, 7, 8])
def test_matches_oracle(kdt, b):
    for i, n in enumerate([1, 17, 1000, 1000003, (1 << 22) + 5]):
        k = _keys(kdt, n, seed=100 * b + i)
        got = _run(k, b)
        assert np.array_equal(got, oracle.radix_offsets(k, b)), (b, n)


@pytest.mark.parametrize("kdt", [np.uint32, np.uint64], ids=["u32", "u64"])
@pytest.mark.parametrize("kind", ["equal", "few"])
def test_skewed_keys(kdt, kind):
    k = _keys(kdt, 3_000_017, seed=5, kind=kind)
    assert np.array_equal(_run(k, 8), oracle.radix_offsets(k, 8))


@pytest.mark.parametrize("kdt", [np.uint32, np.uint64], ids=["u32", "u64"])
def test_unaligned_keys(kdt):
    k = _keys(kdt, 123457, seed=9)
    assert np.array_equal(_run(k, 8, pad_front=1), oracle.radix_offsets(k, 8))


def test_back_to_back_launches_reuse_the_scratch():
    """Each launch leaves its counters and done word zeroed for the next one
    on the stream; run several sizes and widths without synchronising."""
    s = torch.cuda.current_stream().cuda_stream
    jobs = []
    for i, (n, b) in enumerate([(50000, 8), (7, 2), (2000000, 5), (64, 8)]):
        k = _keys(np.uint32, n, seed=40 + i)
        d = torch.from_numpy(k.view(np.int32).copy()).cuda()
        out = torch.empty((-(-32 // b), 1 << b), dtype=torch.int64, device="cuda")
        assert _lib.lscan_radix_offsets(d.data_ptr(), 4, n, b, out.data_ptr(), s) == 0
        jobs.append((k, b, d, out))
    torch.cuda.synchronize()
    for k, b, _, out in jobs:
        assert np.array_equal(out.cpu().numpy(), oracle.radix_offsets(k, b))


def test_empty_writes_zeros():
    out = torch.full((4, 256), 5, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert _lib.lscan_radix_offsets(None, 4, 0, 8, out.data_ptr(), s) == 0
    assert not out.cpu().numpy().any()


def test_torch_front():
    import paper_1604_04815_gb300 as lscan
    k = _keys(np.uint64, 300001, seed=12)
    d = torch.from_numpy(k.view(np.int64).copy()).cuda()
    got = lscan.radix_offsets(d, digit_bits=6)
    assert tuple(got.shape) == (11, 64)
    assert np.array_equal(got.cpu().numpy(), oracle.radix_offsets(k, 6))


def test_full_size_workload():
    """2^28 uniform uint32 keys, 8-bit digits: the bench.py configuration."""
    from paper_1604_04815_gb300 import workloads
    k = workloads.radix_keys(N_FULL)
    assert np.array_equal(_run(k, 8), oracle.radix_offsets(k, 8))


@pytest.mark.parametrize("kdt", [np.uint32, np.uint64], ids=["u32", "u64"])
@pytest.mark.parametrize("kind", ["equal", "few"])
def test_pair_histograms_with_many_guard_overflows(kdt, kind):
    """8-bit digits on 2^24 keys take the joint digit-pair histograms; with
    one to three distinct keys each CTA's bin passes its 15-bit count many
    times (the guard bit is cleared and 32768 counted globally each time)."""
    k = _keys(kdt, (1 << 24) + 3, seed=77, kind=kind)
    assert np.array_equal(_run(k, 8), oracle.radix_offsets(k, 8))


def test_pair_histograms_at_the_size_threshold():
    """Just below and at 2^20 keys (the smallest array the pair kernel takes)
    and unaligned keys there (plain loads in the pair kernel)."""
    for i, n in enumerate([(1 << 20) - 1, 1 << 20, (1 << 20) + 1]):
        k = _keys(np.uint32, n, seed=300 + i)
        assert np.array_equal(_run(k, 8), oracle.radix_offsets(k, 8)), n
        assert np.array_equal(_run(k, 8, pad_front=1), oracle.radix_offsets(k, 8)), n
