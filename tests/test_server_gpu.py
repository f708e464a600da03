"""Serving: continuous batching over the C ABI (lscan_server_*).

The central property: every request's result is the same whether it runs
alone or mixed with concurrent requests of other sizes, dtypes and operators
(bit-identical for int32 and max; within the float bound, and equal to its
solo run within that bound, for float add), and both agree with the oracle.
"""
import numpy as np
import pytest
import torch

import paper_1604_04815_gb300 as lscan
from gpu_util import assert_matches, to_device, to_host, BOUND
from paper_1604_04815_gb300 import _lib
from paper_1604_04815_gb300.workloads import random_array

pytestmark = pytest.mark.gpu

TDT = {"i32": torch.int32, "f32": torch.float32, "bf16": torch.bfloat16,
       "i64": torch.int64, "f64": torch.float64}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_04815_gb300 import build
    build.build()
    _lib.load()


def _mix(n_req, seed, max_log2=18):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n_req):
        n = int(np.rint(2.0 ** (rng.random() * max_log2)))
        if i % 17 == 0:
            n = 0 if i % 34 == 0 else 1
        d = rng.random()
        dtype = ("i32" if d < 0.45 else "f32" if d < 0.75 else
                 "bf16" if d < 0.9 else "i64" if d < 0.95 else "f64")
        op = "add" if rng.random() < 0.5 else "max"
        incl = bool(rng.random() < 0.8)
        kind = "full" if dtype in ("i32", "i64") else "signed"
        reqs.append(dict(n=n, dtype=dtype, op=op, incl=incl,
                         x=random_array(dtype, n, rng, kind=kind)))
    return reqs


def _out_like(r):
    dt = lscan.out_dtype_for(r["op"], TDT[r["dtype"]])
    return torch.empty(r["n"], dtype=dt, device="cuda")


def test_same_alone_and_in_the_mix():
    reqs = _mix(80, seed=1)
    srv = lscan.Server(budget_bytes=2 << 30, n_streams=4)
    try:
        xs = [to_device(r["x"], r["dtype"]) for r in reqs]
        # alone: one request in flight at a time
        alone = []
        for r, xd in zip(reqs, xs):
            y = _out_like(r)
            tk = srv.submit(xd, r["op"], r["incl"], out=y)
            st = srv.wait(tk)
            assert st["status"] == 0 and st["batch_requests"] == 1
            srv.release(tk)
            alone.append(to_host(y))
        # in the mix: everything queued while the server holds, then
        # launched together (batched by kind) and collected
        ys = [_out_like(r) for r in reqs]
        srv.hold(True)
        tks = [srv.submit(xd, r["op"], r["incl"], out=y)
               for r, xd, y in zip(reqs, xs, ys)]
        srv.hold(False)
        stats = [srv.wait(tk) for tk in tks]
        for tk in tks:
            srv.release(tk)
        assert max(s["batch_requests"] for s in stats) > 1  # really batched
        for r, a, y, st in zip(reqs, alone, ys, stats):
            assert st["status"] == 0
            m = to_host(y)
            assert_matches(r["op"], r["dtype"], r["x"], a, r["incl"])
            assert_matches(r["op"], r["dtype"], r["x"], m, r["incl"])
            if r["op"] == "max" or r["dtype"] in ("i32", "i64"):
                assert np.array_equal(a.view(np.uint8), m.view(np.uint8))
            else:
                import oracle
                from gpu_util import BOUND_F64_ADD
                s = oracle.abs_prefix(r["dtype"], r["x"], r["incl"])
                c = BOUND_F64_ADD if r["dtype"] == "f64" else BOUND["f64"]
                assert np.all(np.abs(a.astype(np.float64) - m) <= 2 * c * s)
    finally:
        srv.close()


def test_server_outputs_and_admission_under_a_small_budget():
    """Outputs allocated by the server from a pool far smaller than the
    total they need: requests wait for admission and all complete."""
    rng = np.random.default_rng(4)
    n = 1 << 20                      # 4 MiB output each
    reqs = [random_array("i32", n, rng, kind="full") for _ in range(24)]
    xs = [to_device(x, "i32") for x in reqs]
    # the launch slots reserve their scratch first (6 slots x ~8 MiB of
    # status words); the pool that remains (< 40 MiB) holds only a few of
    # the 24 outputs of 4 MiB at a time
    srv = lscan.Server(budget_bytes=88 << 20, n_streams=2)
    try:
        tks = [srv.submit(xd, "add", True) for xd in xs]     # out=None
        for x, tk in zip(reqs, tks):
            st = srv.wait(tk)
            assert st["status"] == 0
            assert st["submit_us"] <= st["admit_us"] <= st["launch_us"] <= \
                st["done_us"]
            y = srv.output(st, "add", torch.int32)
            assert_matches("add", "i32", x, to_host(y))
            srv.release(tk)
        # a request whose output can never fit is refused at once
        big = torch.empty(16 << 20, dtype=torch.int32, device="cuda")
        with pytest.raises(lscan.LscanError):
            srv.submit(big, "add", True)
    finally:
        srv.close()


def test_server_replay_open_loop():
    rng = np.random.default_rng(7)
    lake = to_device(random_array("i32", 1 << 22, rng, kind="full"), "i32")
    lakef = to_device(random_array("f32", 1 << 22, rng, kind="signed"), "f32")
    trace, t = [], 0.0
    for i in range(400):
        n = int(np.rint(2.0 ** (10 + 8 * rng.random())))
        off = int(rng.integers(0, (1 << 22) - n)) // 4 * 4
        src = lake if i % 2 == 0 else lakef
        t += float(rng.exponential(20.0))
        trace.append(("add" if i % 3 else "max", src.dtype, True,
                      src.data_ptr() + 4 * off, n, t))
    srv = lscan.Server(budget_bytes=512 << 20, n_streams=4)
    try:
        stats, wall = srv.replay(trace)
    finally:
        srv.close()
    assert wall > 0
    for s in stats:
        assert s["status"] == 0
        assert s["submit_us"] <= s["admit_us"] + 1e-6
        assert s["launch_us"] <= s["done_us"]
        assert s["done_us"] >= s["submit_us"]


def test_server_rejects_bad_requests():
    srv = lscan.Server(budget_bytes=64 << 20, n_streams=1)
    try:
        L = _lib.load()
        import ctypes
        tk = ctypes.c_uint64()
        assert L.lscan_server_submit(srv._h, 0, 0, 1, None, None, 10,
                                     ctypes.byref(tk)) == _lib.LSCAN_ERR_INVALID
        assert L.lscan_server_submit(srv._h, 0, 9, 1, 1 << 20, None, 10,
                                     ctypes.byref(tk)) == _lib.LSCAN_ERR_INVALID
        assert L.lscan_server_submit(srv._h, 0, 0, 1, 1 << 20, None, -1,
                                     ctypes.byref(tk)) == _lib.LSCAN_ERR_INVALID
        assert L.lscan_server_release(srv._h, 12345) == _lib.LSCAN_ERR_INVALID
    finally:
        srv.close()


def test_resident_lane_across_chunk_boundaries():
    """Small-lane requests scanned by the resident kernel, one CTA each, in
    chunks of 16384 elements of up to 4 bytes or 8192 of 8 bytes: sizes just
    below, at and above a chunk and over several chunks, so the running
    carry passes from chunk to chunk, for every kind the lane scans (int32
    add and max, fp32 and bf16 max, fp32 and bf16 add with the default
    carry, int64 and double add and max).  The lane bound is raised to 2^16
    so that requests of several chunks take it."""
    srv = lscan.Server(budget_bytes=1 << 30, n_streams=2)
    try:
        srv.set_lanes(small_max_elems=1 << 16, bulk_batch_tiles=8192, reserve_sms=4)
        rng = np.random.default_rng(44)
        cases = []
        for dtype in ("i32", "f32", "bf16", "i64", "f64"):
            chunk = 8192 if dtype in ("i64", "f64") else 16384
            for n in (chunk - 1, chunk, chunk + 1, 3 * chunk + 17, 1 << 16):
                for op in ("add", "max"):
                    incl = bool(rng.random() < 0.5)
                    kind = "full" if dtype in ("i32", "i64") else "signed"
                    cases.append((op, dtype, incl,
                                  random_array(dtype, n, rng, kind=kind)))
        xs = [to_device(x, d) for _, d, _, x in cases]
        ys = [torch.empty(x.shape[0], dtype=lscan.out_dtype_for(op, TDT[d]),
                          device="cuda") for op, d, _, x in cases]
        # queued while the server holds: the bulk lane would launch each
        # kind's five requests together, the resident lane retires them one
        # by one (batch_requests == 1 shows which lane took them)
        srv.hold(True)
        tks = [srv.submit(xd, op, incl, out=y)
               for (op, _, incl, _), xd, y in zip(cases, xs, ys)]
        srv.hold(False)
        for tk in tks:
            st = srv.wait(tk)
            assert st["status"] == 0 and st["batch_requests"] == 1
            srv.release(tk)
        for (op, d, incl, x), y in zip(cases, ys):
            assert_matches(op, d, x, to_host(y), incl)
    finally:
        srv.close()
