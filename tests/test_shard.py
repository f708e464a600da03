"""Sharded scan, host side, on CPU: two gloo ranks each hold a contiguous
shard of one array, exchange their shard totals (all-gather of 4- or 8-byte
carry values) and fold the totals of the lower ranks with the library's
host combine (lscan_carry_combine, no GPU involved).  Each rank then applies
its offset to the oracle's scan of its shard, the way the device scan
applies a carry-in, and the stitched result must equal the oracle's scan of
the whole array: bit for bit for int32 add and for float max (+0 / -0 ties
across the shard boundary), within the bound for fp32 add."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _global_array(case, n):
    rng = np.random.default_rng(31)
    if case == "i32_add":
        return rng.integers(-(1 << 31), 1 << 31, size=n, dtype=np.int32)
    if case == "f32_add":
        return (rng.random(size=n, dtype=np.float32) * 2 - 1).astype(np.float32)
    # f32 max: negatives and zeros of both signs, the first zero on rank 1
    x = rng.choice(np.array([-1.0, -2.5, -np.inf], dtype=np.float32), size=n)
    z = np.where(rng.random(size=n) < 0.5, np.float32(-0.0), np.float32(0.0))
    put = rng.random(size=n) < 0.01
    put[: n // 2 + 3] = False
    x = np.where(put, z, x).astype(np.float32)
    x[n // 2 + 3] = np.float32(-0.0)
    return x


def _shard_total(case, xs):
    """The shard's total in the kind's carry type, as bytes (the value the
    device reduction produces, from the oracle)."""
    import oracle
    if case == "i32_add":
        t = int(np.sum(xs.astype(np.int64))) & 0xFFFFFFFF
        return np.uint32(t).tobytes()
    if case == "f32_add":  # double-float pair of the FP64 total
        t = float(oracle.scan("add", "f32", xs, True)[-1]) if len(xs) else 0.0
        hi = np.float32(t)
        lo = np.float32(t - float(hi))
        return np.array([hi, lo], dtype=np.float32).tobytes()
    t = oracle.scan("max", "f32", xs, True)[-1] if len(xs) else np.float32(-np.inf)
    return np.float32(t).tobytes()


def _apply_offset(case, xs, off):
    """off (+) the oracle's inclusive scan of the shard."""
    import oracle
    if case == "i32_add":
        o = int(np.frombuffer(off, dtype=np.uint32)[0])
        y = oracle.scan("add", "i32", xs, True).astype(np.int64) + o
        return (y & 0xFFFFFFFF).astype(np.uint32).view(np.int32)
    if case == "f32_add":
        hi, lo = np.frombuffer(off, dtype=np.float32)
        return oracle.scan("add", "f32", xs, True) + (float(hi) + float(lo))
    o = np.frombuffer(off, dtype=np.float32)[0]
    p = oracle.scan("max", "f32", xs, True)
    return np.where(p > o, p, o).astype(np.float32)   # the carry is earlier


def _rank_main(rank, ws, port, case, n, bounds, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1604_04815_gb300 import _lib, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        x = _global_array(case, n)
        xs = x[bounds[rank]:bounds[rank + 1]]
        op = _lib.LSCAN_MAX if case == "f32_max" else _lib.LSCAN_ADD
        dt = _lib.LSCAN_I32 if case == "i32_add" else _lib.LSCAN_F32
        opts = _lib.make_options()   # default precision: double-float carry
        off, totals = shard.exchange_offset(_shard_total(case, xs), op, dt,
                                            opts)
        out.put((rank, _apply_offset(case, xs, off), len(totals)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", ["i32_add", "f32_add", "f32_max"])
def test_two_rank_exchange_and_offsets(case):
    import oracle
    n = 100_003
    bounds = [0, 37_001, n]            # uneven shards
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main,
                         args=(r, ws, port, case, n, bounds, q))
             for r in range(ws)]
    for p in procs:
        p.start()
    got = dict((r, (y, k)) for r, y, k in (q.get(timeout=180)
                                          for _ in range(ws)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(k == ws for _, k in got.values())
    stitched = np.concatenate([got[r][0] for r in range(ws)])
    x = _global_array(case, n)
    if case == "i32_add":
        assert np.array_equal(stitched, oracle.scan("add", "i32", x, True))
    elif case == "f32_max":
        want = oracle.scan("max", "f32", x, True)
        assert np.array_equal(stitched.view(np.uint32), want.view(np.uint32))
        assert np.signbit(stitched[-1])      # the first zero was -0
    else:
        want = oracle.scan("add", "f32", x, True)
        s = oracle.abs_prefix("f32", x, True)
        assert np.all(np.abs(stitched - want) <= 1e-12 * s + 1e-30)


def test_carry_combine_on_the_host():
    """The host fold of carry values, without a GPU: wrapping int32 adds,
    first-occurrence float max, the double-float pair sum, identities."""
    import sys
    sys.path.insert(0, ROOT)
    from paper_1604_04815_gb300 import _lib as L
    t = np.array([0x7FFFFFFF, 5, 0xFFFFFFFF], dtype=np.uint32).tobytes()
    st, r = L.lscan_carry_combine(L.LSCAN_ADD, L.LSCAN_I32, t, 3)
    assert st == L.LSCAN_OK
    assert np.frombuffer(r, dtype=np.uint32)[0] == (0x7FFFFFFF + 5 + 0xFFFFFFFF) % 2**32
    st, r = L.lscan_carry_combine(L.LSCAN_ADD, L.LSCAN_I32, t, 0)
    assert np.frombuffer(r, dtype=np.uint32)[0] == 0          # identity
    z = np.array([-0.0, 0.0, -1.0], dtype=np.float32).tobytes()
    st, r = L.lscan_carry_combine(L.LSCAN_MAX, L.LSCAN_F32, z, 3)
    v = np.frombuffer(r, dtype=np.float32)[0]
    assert v == 0 and np.signbit(v)                          # first zero: -0
    st, r = L.lscan_carry_combine(L.LSCAN_MAX, L.LSCAN_F32, z, 0)
    assert np.frombuffer(r, dtype=np.float32)[0] == -np.inf
    # double-float: 1 + 2^-30 + 2^-30 keeps the low part exactly
    d = np.array([1.0, 0.0, 2.0 ** -30, 0.0, 2.0 ** -30, 0.0],
                 dtype=np.float32).tobytes()
    st, r = L.lscan_carry_combine(L.LSCAN_ADD, L.LSCAN_F32, d, 3)
    hi, lo = np.frombuffer(r, dtype=np.float32)
    assert float(hi) + float(lo) == 1.0 + 2.0 ** -29
    assert L.lscan_carry_bytes(L.LSCAN_ADD, L.LSCAN_F32) == 8   # (hi, lo)
    assert L.lscan_carry_bytes(L.LSCAN_ADD, L.LSCAN_I32) == 4
    assert L.lscan_carry_bytes(
        L.LSCAN_ADD, L.LSCAN_F32,
        L.make_options(precision=L.LSCAN_PREC_F32_CARRY)) == 4
    # the FP64 carry and double add: plain double sums
    e = np.array([0.1, 0.2], dtype=np.float64).tobytes()
    st, r = L.lscan_carry_combine(
        L.LSCAN_ADD, L.LSCAN_F32, e, 2,
        L.make_options(precision=L.LSCAN_PREC_F64_CARRY))
    assert np.frombuffer(r, dtype=np.float64)[0] == 0.1 + 0.2
    assert L.lscan_carry_combine(L.LSCAN_ADD, L.LSCAN_I32, t, -1)[0] == \
        L.LSCAN_ERR_INVALID
