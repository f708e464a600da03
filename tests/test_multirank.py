"""bench.py's N > 1 path on CPU (gloo, world size 2): whole-job throughput
is every rank's bytes over the slowest rank's time, and under
torch.distributed.run only rank 0 prints the reference arm's line."""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location(
        "bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        b = _bench()
        b._barrier(ws)
        # rank r's timed region lasted 1 + r seconds
        emax, gbs = b._aggregate(step_bytes=3 * 10**9, steps=2,
                                 elapsed_s=1.0 + rank, ws=ws)
        out.put((rank, emax, gbs))
    finally:
        dist.destroy_process_group()


def test_aggregate_max_over_ranks_gloo():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q))
             for r in range(ws)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, emax, gbs in got:
        assert emax == 2.0                       # the slowest rank's time
        assert abs(gbs - 3 * 2 * 2 / 2.0) < 1e-9  # all ranks' bytes / max


def test_single_rank_aggregate_needs_no_process_group():
    b = _bench()
    emax, gbs = b._aggregate(step_bytes=8 * 10**9, steps=4, elapsed_s=2.0, ws=1)
    assert emax == 2.0 and gbs == 16.0


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
           "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "3", "--log2n", "16"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True,
                       timeout=240)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_traffic_reported_only_for_the_measured_sources_and_size(monkeypatch):
    """roofline.traffic is the ncu figure only for N = 2^28 and the kernel
    sources it was taken on; any other size or a changed source is null."""
    b = _bench()
    key = next(iter(b._TRAFFIC["bytes_per_launch"]))
    want = b._TRAFFIC["bytes_per_launch"][key]
    if b._kernel_source_hash() == b._TRAFFIC["kernel_source_hash"]:
        assert b._traffic_for(key[0], key[1], 1 << 28) == want
    assert b._traffic_for(key[0], key[1], 1 << 26) is None
    monkeypatch.setitem(b._TRAFFIC, "kernel_source_hash", "0" * 16)
    assert b._traffic_for(key[0], key[1], 1 << 28) is None
    assert "N=2^26" in b._workload(1 << 26)
