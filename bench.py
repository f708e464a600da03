"""Benchmark: single-pass scan throughput on one GB300 (and N replicas).

One step = one pass of the scan path over the single-array workload: an
inclusive int32 add-scan (uniform [-2^15, 2^15]), an inclusive int32
max-scan (full int32 range) and an inclusive fp32 add-scan (uniform [0, 1),
double-float carry), each over N = 2^28 elements already resident in HBM.
value = bytes moved (each element read once and written once) / time, summed
over ranks.  Inputs are 1 GiB per array, far above the 129 MB L2, so no L2
flush is needed between steps.

Also reported on the same line:
  roofline     dominant kernel's algorithmic GB/s vs the measured HBM copy peak
  e2e          the same scans from pinned HOST buffers through the C ABI's
               host entry point (lscan_scan_host: chunked copy-in, scan and
               copy-out overlapped), all copies inside the timed region, with
               the host link's own pinned-copy ceiling measured beside it
  cub          CUB's device scan on the same resident inputs (comparator)
  cpu_parallel a multi-threaded scan on all host cores (comparator)
  batched      4096 log-uniform arrays (lengths 1..2^20) in one persistent
               launch replayed from a CUDA graph, vs 4096 plain launches
  dtypes       add scans of the paper's types (int32, fp32, int64, double)
  precision    fp32 and bf16 add at 2^26 on log-normal input, every carry
               path, with the error against a float64 reference
  bf16         bf16 max and add (fp32 and bf16 output) at 2^28
  small        latency of an L2-resident 2^20 scan and of a 1000-element one
  select       stream compaction (a scan consumer), 2^28 int32, half kept
  radix        radix-sort digit offsets (a scan consumer), 2^28 uint32 keys
  serving      Poisson request streams through the scan server
  cpu_baseline the sequential CPU oracle timed on a bounded sample
  clocks       nvidia-smi samples taken during the timed region

--impl reference times the CPU oracle (the slow reference program) on the
same workload, one bounded sample per step.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = 1 << 28
METRIC = ("scan GB/s & % of HBM peak, batched vs per-array; "
          "p50/p99 served latency")
def _workload(n):
    return (f"single-array inclusive scans, N=2^{n.bit_length() - 1} each: "
            "int32 add (uniform [-2^15,2^15]), int32 max (full int32 range), "
            "fp32 add (uniform [0,1), double-float carry)")
CASES = [  # (name, op, dtype)
    ("i32_add", "add", "i32"),
    ("i32_max", "max", "i32"),
    ("f32_add", "add", "f32"),
]
ELEM_BYTES = {"i32": 4, "f32": 4, "bf16": 2}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _inputs(case, n):
    from paper_1604_04815_gb300 import workloads
    if case == "i32_add":
        return workloads.large_i32_add(n)
    if case == "i32_max":
        return workloads.large_i32_max(n)
    return workloads.large_f32_add(n)


# Sources that do not build or launch the bench's scan kernels: other
# kernels (radix offsets) and entry points the timed scans do not go through.
_NOT_SCAN_SOURCES = {"radix_offsets.cu", "lscan_host.cu", "lscan_server.cu",
                     "lscan_graph.cu", "lscan_noalloc.cu", "resident_kernel.cu",
                     "resident.h", "lscan_shard.cu"}


def _kernel_source_hash():
    """Hash of the sources of the bench's scan kernels and their launch
    path (kernel templates, kinds, instantiations, dispatch, tuning)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1604_04815_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cuh", ".cu", ".h")) and fn not in _NOT_SCAN_SOURCES:
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(fn.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the bench's kernels at N = 2^28, from one ncu capture of this bench's
# kernels (the summary and its command are kept with the profiles).  Valid
# only for the kernel sources it was taken on: any change to csrc/ makes the
# reported traffic null until it is measured again (files listed in
# _NOT_SCAN_SOURCES excepted).
_TRAFFIC = {
    "kernel_source_hash": "80fe94155156a710",
    "bytes_per_launch": {  # (case, tile configuration)
        ("i32_add", 6): 1077993216 + 1019572992,
        ("i32_max", 6): 1077990912 + 1016316160,
        ("f32_add", 6): 1078080512 + 1016428032,
        ("i32_add", 8): 1075898880 + 1019142656,
        ("i32_max", 8): 1075948800 + 1016191744,
        ("f32_add", 8): 1075965952 + 1016437504,
        ("i32_add", 17): 1075273472 + 1018695168,
        ("i32_max", 17): 1075228928 + 1015876352,
        ("f32_add", 17): 1075234304 + 1015827200,
    },
}


def _traffic_for(kernel_case, config, n):
    """DRAM bytes per launch measured on the current kernel sources, tile
    configuration and size (N = 2^28 only), or None."""
    if n != 1 << 28 or _TRAFFIC["kernel_source_hash"] != _kernel_source_hash():
        return None
    return _TRAFFIC["bytes_per_launch"].get((kernel_case, config))


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _reduce_max(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _aggregate(step_bytes, steps, elapsed_s, ws):
    """Whole-job throughput: the bytes of every rank's steps over the slowest
    rank's timed region.  Returns (max elapsed seconds, GB/s)."""
    elapsed_max = _reduce_max(elapsed_s, ws)
    return elapsed_max, step_bytes * steps * ws / elapsed_max / 1e9


# --------------------------------------------------------------- CPU oracle
def cpu_baseline(budget_s=12.0, n=N):
    """Times the sequential oracle on the step's three arrays (bounded)."""
    import oracle
    arrays = [(_inputs(c, n), op, dt) for c, op, dt in CASES]
    total_bytes, total_t, reps = 0, 0.0, 0
    while reps < 1 or (total_t < budget_s and reps < 5):
        for x, op, dt in arrays:
            t0 = time.perf_counter()
            oracle.scan(op, dt, x, True)
            total_t += time.perf_counter() - t0
            total_bytes += 2 * x.nbytes
        reps += 1
    return {"value": total_bytes / total_t / 1e9, "unit": "GB/s", "cores": 1,
            "kind": "oracle",
            "sample": f"{reps} pass(es) of the step's three 2^{n.bit_length()-1}"
                      f"-element arrays through the sequential C oracle"}


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    import oracle
    n = N
    arrays = [(_inputs(c, n), op, dt) for c, op, dt in CASES]
    # each step: one bounded sample = the three arrays' first 2^26 elements
    m = 1 << 26
    samples = [(x[:m].copy(), op, dt) for x, op, dt in arrays]
    for _ in range(args.warmup):
        for x, op, dt in samples:
            oracle.scan(op, dt, x, True)
    times = []
    nbytes = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for x, op, dt in samples:
            oracle.scan(op, dt, x, True)
        times.append(time.perf_counter() - t0)
    nbytes = sum(2 * x.nbytes for x, _, _ in samples)
    tot = sum(times)
    value = nbytes * args.steps / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32/f32",
        "data": "synthetic",
        "config": {"workload": _workload(N), "n": N,
                   "sample": "first 2^26 elements of each array per step"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1,
                         "kind": "oracle",
                         "sample": "first 2^26 elements of each of the three "
                                   "2^28 arrays, per step"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU path
def run_gpu(args, ws, rank, local):
    import torch

    import paper_1604_04815_gb300 as lscan
    from paper_1604_04815_gb300 import _lib, build

    if ws > 1:
        torch.cuda.set_device(local)
    dev = torch.device("cuda", torch.cuda.current_device())
    build.build()
    _lib.load()
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    peak, peak_src = _peaks()

    host = {c: _inputs(c, N) for c, _, _ in CASES}
    xs = {c: torch.from_numpy(host[c]).to(dev) for c in host}
    ys = {c: torch.empty_like(xs[c]) for c in host}
    torch.cuda.synchronize()
    step_bytes = sum(2 * N * ELEM_BYTES[dt] for _, _, dt in CASES)

    def launch(case, op, dt):
        if args.sharded and ws > 1:
            # this rank's 2^k elements are shard `rank` of one array of
            # ws * 2^k: reduce, all-gather of the totals, carry-in scan
            lscan.shard.sharded_scan(xs[case], op, True, out=ys[case],
                                     stream=stream)
            return
        st = _lib.lscan_scan(_lib.LSCAN_ADD if op == "add" else _lib.LSCAN_MAX,
                             _lib.LSCAN_I32 if dt == "i32" else _lib.LSCAN_F32,
                             1, xs[case].data_ptr(), ys[case].data_ptr(), N,
                             _lib.make_options(config=args.config,
                                               carry=args.carry), sp)
        if st != _lib.LSCAN_OK:
            raise RuntimeError(_lib.strerror(st))

    # autotune the tile configuration of each scan on its own buffers
    tuned = {}
    if args.config == 0:
        for c, op, dt in CASES:
            st, res = _lib.lscan_autotune(
                _lib.LSCAN_ADD if op == "add" else _lib.LSCAN_MAX,
                _lib.LSCAN_I32 if dt == "i32" else _lib.LSCAN_F32, 1,
                xs[c].data_ptr(), ys[c].data_ptr(), N,
                opts=_lib.make_options(carry=args.carry), reps=args.tune_reps,
                stream=sp)
            _lib.check(st, "lscan_autotune")
            best = res["config"]
            info = _lib.lscan_config_info(best, _lib.LSCAN_I32)
            tuned[c] = {"config": best, "items": info["items"],
                        "threads": info["threads"], "tile": info["tile"],
                        "stages": info["stages"],
                        "tuned_ms": round(res["ms"], 4),
                        "default_config": res["default_config"],
                        "default_ms": round(res["default_ms"], 4),
                        "gain_vs_default": round(
                            res["default_ms"] / res["ms"], 4),
                        "configs_timed": res["n_timed"]}
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            for c, op, dt in CASES:
                launch(c, op, dt)
    _lib.check(_lib.lscan_stream_status(sp), "warm-up")

    ev = {c: [(torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)] for c, _, _ in CASES}
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev.index) if rank == 0 else None
    _barrier(ws)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    launches0 = _lib.lscan_launch_count()
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for k in range(args.steps):
            for c, op, dt in CASES:
                ev[c][k][0].record(stream)
                launch(c, op, dt)
                ev[c][k][1].record(stream)
        t_end.record(stream)
    stream.synchronize()
    launches = _lib.lscan_launch_count() - launches0
    torch.cuda.synchronize()
    _barrier(ws)
    clk = clocks.stop() if clocks else None
    _lib.check(_lib.lscan_stream_status(sp), "timed region")
    elapsed = t_start.elapsed_time(t_end) / 1e3
    elapsed_max, value = _aggregate(step_bytes, args.steps, elapsed, ws)

    per_kernel = {}
    for c, op, dt in CASES:
        ms = [a.elapsed_time(b) for a, b in ev[c]]
        avg = sum(ms) / len(ms) / 1e3
        per_kernel[c] = {"avg_us": avg * 1e6,
                         "gbs": 2 * N * ELEM_BYTES[dt] / avg / 1e9}
    dom = max(per_kernel, key=lambda c: per_kernel[c]["avg_us"])
    achieved = per_kernel[dom]["gbs"]
    roofline = {"bound": "hbm", "achieved": round(achieved, 1),
                "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": _traffic_for(
                    dom, args.config or tuned.get(dom, {}).get("config"), N),
                "kernel": dom,
                "peak_source": peak_src,
                "algorithmic_bytes_per_launch": 2 * N * 4}

    # ---- e2e: pinned host buffers, copies inside the timed region ----
    e2e = None
    if not args.no_e2e:
        hx = {c: torch.from_numpy(host[c]).pin_memory() for c in host}
        hy = {c: torch.empty_like(hx[c]).pin_memory() for c in host}
        torch.cuda.synchronize()

        e2e_opts = _lib.make_options(config=args.config, carry=args.carry)

        def e2e_step():
            # the public host-buffer entry point: chunked copy-in, scan and
            # copy-out, overlapped inside the library
            for c, op, dt in CASES:
                st = _lib.lscan_scan_host(
                    _lib.LSCAN_ADD if op == "add" else _lib.LSCAN_MAX,
                    _lib.LSCAN_I32 if dt == "i32" else _lib.LSCAN_F32, 1,
                    hx[c].data_ptr(), hy[c].data_ptr(), N, e2e_opts,
                    args.e2e_chunk, sp)
                if st != _lib.LSCAN_OK:
                    raise RuntimeError(_lib.strerror(st))
        for _ in range(max(1, args.warmup // 2)):
            e2e_step()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ksteps = max(1, min(args.steps, 5))
        _barrier(ws)
        e0.record(stream)
        for _ in range(ksteps):
            e2e_step()
        e1.record(stream)
        stream.synchronize()
        et = _reduce_max(e0.elapsed_time(e1) / 1e3, ws)
        _lib.check(_lib.lscan_stream_status(sp), "e2e")
        # sanity check against the device-resident run of the same input
        # (head and tail; float add within the FP64-carry bound's scale)
        ok = True
        for c, _, dt in CASES:
            for sl in (slice(0, 1 << 16), slice(N - (1 << 16), N)):
                a = hy[c][sl].numpy()
                b = ys[c][sl].cpu().numpy()
                if dt == "i32":
                    ok &= bool(np.array_equal(a, b))
                else:
                    ok &= bool(np.all(np.abs(a.astype(np.float64) - b) <=
                                      1e-5 * np.abs(b.astype(np.float64))))
        e2e = {"value": step_bytes * ksteps * ws / et / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": sum(x.nbytes for x in host.values()),
               "d2h_bytes_per_step": sum(x.nbytes for x in host.values()),
               "steps": ksteps, "result_check": bool(ok),
               "path": "lscan_scan_host from pinned host buffers: " +
                       (f"chunks of {args.e2e_chunk} elements"
                        if args.e2e_chunk else
                        "chunks of 2^20 doubling to 2^23 elements and halving "
                        "again at the end") +
                       ", copy-in, scan and copy-out overlapped on three "
                       "streams"}
        del hx, hy

    # the host link's own ceiling for the same traffic
    if e2e is not None and not args.no_link:
        link = host_link_ceiling(dev)
        e2e["host_link"] = link
        e2e["frac_of_duplex_copy"] = round(e2e["value"] / link["duplex_gbs"], 4)

    # ---- comparators: CUB's device scan on the same resident inputs, and a
    # multi-threaded scan on the host cores ----
    cub = None
    if not args.no_cub and ws == 1 and not args.sharded:
        cub = bench_cub(dev, stream, peak, xs, ys, launch, N)
    cpu_par = None
    if not args.no_cpu_parallel and ws == 1 and not args.sharded:
        cpu_par = bench_cpu_parallel(host, N)

    # ---- batched: one graph-replayed persistent launch vs 4096 launches ----
    batched = None
    if not args.no_batched:
        batched = bench_batched(args, dev, stream, peak)

    # ---- the paper's data types (Table 2) and the small-array latency ----
    dtypes = None if args.no_dtypes else bench_dtypes(args, dev, stream, peak)
    precision = None if args.no_precision else bench_precision(
        args, dev, stream, peak, min(26, args.log2n))
    bf16 = None if args.no_bf16 else bench_bf16(args, dev, stream, peak,
                                                args.log2n)
    small = None if args.no_small else bench_small(args, dev, stream)
    select = None if args.no_select else bench_select(args, dev, stream, peak,
                                                      args.log2n)
    radix = None if args.no_radix else bench_radix(args, dev, stream, peak,
                                                   args.log2n)

    # ---- serving: Poisson stream through the continuous-batching server ----
    serving = None
    if not args.no_serving:
        serving = bench_serving(args, dev, peak, args.serving_requests,
                                [float(f) for f in args.serving_loads.split(",")])

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * elapsed_max / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "i32/f32", "data": "synthetic",
        "config": {"workload": _workload(N), "n": N, "tile_config": args.config or tuned,
                   "carry": ["auto", "lookback", "chained"][args.carry],
                   "l2": "inputs 1 GiB per array > 129 MB L2; no flush",
                   "parallelism": (f"one array sharded over {ws} ranks "
                                   "(reduce, all-gather of totals, carry-in "
                                   "scan)" if args.sharded and ws > 1
                                   else f"replicas x{ws}")},
        "hbm_frac_measured": round(value / ws / peak, 4),
        "geps": round(N * len(CASES) * args.steps * ws / elapsed_max / 1e9, 2),
        "kernels": {c: {k: round(v, 2) for k, v in d.items()}
                    for c, d in per_kernel.items()},
        "roofline": roofline,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "batched": batched,
        "dtypes": dtypes,
        "precision": precision,
        "bf16": bf16,
        "small": small,
        "select": select,
        "radix": radix,
        "cub": cub,
        "cpu_parallel": cpu_par,
        "serving": serving,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(budget_s=args.cpu_budget, n=N)
    print(json.dumps(line), flush=True)
    return 0


def _time_launches(stream, fn, reps):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3


def bench_dtypes(args, dev, stream, peak, log2n=27):
    """Add scans of every element type at one size, GB/s and GEPS (giga
    elements per second, the paper's Table 2 unit); the default tile
    configuration of each kind.  Inputs (2^27 elements: 0.5-1 GiB) exceed
    L2."""
    import torch

    import paper_1604_04815_gb300 as lscan
    n = 1 << log2n
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    out = {"n": n, "op": "add", "inclusive": True}
    cases = (("i32", torch.int32), ("f32", torch.float32),
             ("i64", torch.int64), ("f64", torch.float64))
    with torch.cuda.stream(stream):
        for name, dt in cases:
            if dt.is_floating_point:
                x = torch.rand(n, device=dev, dtype=dt, generator=g)
            else:
                x = torch.randint(-1000, 1001, (n,), device=dev, dtype=dt,
                                  generator=g)
            y = torch.empty_like(x)
            def run():
                lscan.scan(x, "add", True, out=y, stream=stream)
            for _ in range(3):
                run()
            t = _time_launches(stream, run, 10)
            gbs = 2 * n * x.element_size() / t / 1e9
            out[name] = {"gbs": round(gbs, 1), "geps": round(n / t / 1e9, 2),
                         "frac_measured": round(gbs / peak, 4)}
            del x, y
    lscan.stream_status(stream)
    return out


PREC_PATHS = ("plain", "f64", "df", "comp")


def bench_precision(args, dev, stream, peak, log2n=26):
    """The precision workload: N = 2^26 values s * exp(2 Z) (log-normal with
    random signs, cancellation-heavy), fp32 and bf16 inputs, every carry
    path (plain fp32, FP64, double-float, compensated).  Per result: GB/s of
    the timed launches and max_j |err_j| / S_j and max_j |err_j| against an
    FP64 reference taken outside the timed region (numpy's sequential
    float64 cumsum of the exactly widened inputs; S_j = the float64 cumsum of
    |x_i|).  Gates: 1e-5 for plain/FP64/double-float, 2.5e-7 compensated."""
    import torch

    from paper_1604_04815_gb300 import _lib, workloads
    n = 1 << log2n
    x32, xb = workloads.precision(n)
    codes = {"plain": _lib.LSCAN_PREC_F32_CARRY,
             "f64": _lib.LSCAN_PREC_F64_CARRY,
             "df": _lib.LSCAN_PREC_DF_CARRY,
             "comp": _lib.LSCAN_PREC_COMPENSATED}
    gate = {"plain": 1e-5, "f64": 1e-5, "df": 1e-5, "comp": 2.5e-7}
    out = {"n": n, "input": "s*exp(2Z), Z~N(0,1), s=+-1, seed 4",
           "reference": "float64 cumsum of the widened inputs (numpy, "
                        "sequential)"}
    sp = stream.cuda_stream
    for name, host, dcode, in_b in (
            ("f32", x32, _lib.LSCAN_F32, 4),
            ("bf16", xb, _lib.LSCAN_BF16, 2)):
        x64 = (host.astype(np.float64) if name == "f32" else
               workloads.bf16_bits_to_f32(host).astype(np.float64))
        ref = np.cumsum(x64)
        S = np.cumsum(np.abs(x64))
        del x64
        if name == "f32":
            xd = torch.from_numpy(host).to(dev)
        else:
            xd = torch.from_numpy(host.view(np.int16)).to(dev)
        yd = torch.empty(n, dtype=torch.float32, device=dev)
        res = {}
        for path in PREC_PATHS:
            o = _lib.make_options(precision=codes[path])

            def run():
                st = _lib.lscan_scan(_lib.LSCAN_ADD, dcode, 1, xd.data_ptr(),
                                     yd.data_ptr(), n, o, sp)
                if st:
                    raise RuntimeError(_lib.strerror(st))
            with torch.cuda.stream(stream):
                for _ in range(3):
                    run()
                t = _time_launches(stream, run, 10)
            _lib.check(_lib.lscan_stream_status(sp), "precision")
            err = np.abs(yd.cpu().numpy().astype(np.float64) - ref)
            pos = S > 0
            ratio = float(np.max(err[pos] / S[pos]))
            gbs = (in_b + 4) * n / t / 1e9
            res[path] = {"gbs": round(gbs, 1),
                         "frac_measured": round(gbs / peak, 4),
                         "max_err_over_S": float(f"{ratio:.3e}"),
                         "max_abs_err": float(f"{float(np.max(err)):.3e}"),
                         "bound": gate[path], "within_bound": ratio <= gate[path]}
        out[name + "_to_f32"] = res
        del xd, yd, ref, S
    return out


def bench_bf16(args, dev, stream, peak, log2n=28):
    """bf16 scans at N = 2^28 (uniform [-1, 1) for max, [0, 1) for add):
    max (bf16 out), add with the default carry to fp32 and to bf16 output.
    Algorithmic bytes: input + output, once each."""
    import torch

    from paper_1604_04815_gb300 import _lib
    n = 1 << log2n
    g = torch.Generator(device=dev)
    g.manual_seed(11)
    sp = stream.cuda_stream
    out = {"n": n}
    xm = (torch.rand(n, device=dev, generator=g) * 2 - 1).to(torch.bfloat16)
    xa = torch.rand(n, device=dev, generator=g).to(torch.bfloat16)
    for name, x, op, odt in (("max", xm, _lib.LSCAN_MAX, torch.bfloat16),
                             ("add_to_f32", xa, _lib.LSCAN_ADD, torch.float32),
                             ("add_to_bf16", xa, _lib.LSCAN_ADD,
                              torch.bfloat16)):
        y = torch.empty(n, dtype=odt, device=dev)
        o = _lib.make_options(out_dtype=_lib.LSCAN_BF16
                              if (op == _lib.LSCAN_ADD and odt ==
                                  torch.bfloat16) else 0)

        def run():
            st = _lib.lscan_scan(op, _lib.LSCAN_BF16, 1, x.data_ptr(),
                                 y.data_ptr(), n, o, sp)
            if st:
                raise RuntimeError(_lib.strerror(st))
        with torch.cuda.stream(stream):
            for _ in range(3):
                run()
            t = _time_launches(stream, run, 10)
        gbs = (2 + y.element_size()) * n / t / 1e9
        out[name] = {"us": round(t * 1e6, 1), "gbs": round(gbs, 1),
                     "frac_measured": round(gbs / peak, 4)}
        del y
    _lib.check(_lib.lscan_stream_status(sp), "bf16")
    return out


def bench_cub(dev, stream, peak, xs, ys, launch, n, reps=10):
    """Comparator: CUB's single-pass device scan (cub::DeviceScan, built from
    the CUDA toolkit's headers into libcubcmp.so beside liblscan.so) on the
    headline's resident 2^28-element inputs, timed the same way and
    alternating with this library's scans on the same buffers.  For the
    int32 scans its output is compared with this library's bit for bit."""
    import ctypes

    import torch

    from paper_1604_04815_gb300 import build as _build
    path = _build.CMP_LIB
    if not os.path.exists(path):
        return {"unavailable": "libcubcmp.so was not built (CUB headers missing?)"}
    lib = ctypes.CDLL(path)
    lib.cubcmp_temp_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                      ctypes.POINTER(ctypes.c_size_t)]
    lib.cubcmp_inclusive.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_longlong,
                                     ctypes.c_void_p, ctypes.c_size_t,
                                     ctypes.c_void_p]
    sp = stream.cuda_stream
    y2 = torch.empty(n, dtype=torch.int32, device=dev)
    out = {"n": n, "source": "cub::DeviceScan::InclusiveSum / InclusiveScan "
           "(cuda::maximum) from the CUDA toolkit's CCCL headers"}
    for c, op, dt in CASES:
        opc, dtc = (0 if op == "add" else 1), (0 if dt == "i32" else 1)
        nb = ctypes.c_size_t(0)
        if lib.cubcmp_temp_bytes(opc, dtc, n, ctypes.byref(nb)) != 0:
            return {"unavailable": "cub temp-storage query failed"}
        tmp = torch.empty(max(1, nb.value), dtype=torch.uint8, device=dev)
        x = xs[c]

        def run_cub():
            if lib.cubcmp_inclusive(opc, dtc, x.data_ptr(), y2.data_ptr(), n,
                                    tmp.data_ptr(), nb.value, sp) != 0:
                raise RuntimeError("cub scan failed")
        with torch.cuda.stream(stream):
            t_cub, t_ls = [], []
            for _ in range(3):
                run_cub()
                launch(c, op, dt)
            for _ in range(3):  # alternate, best of three batches each
                t_cub.append(_time_launches(stream, run_cub, reps))
                t_ls.append(_time_launches(stream, lambda: launch(c, op, dt), reps))
        tc, tl = min(t_cub), min(t_ls)
        gb = 8 * n / 1e9
        r = {"cub_us": round(tc * 1e6, 1), "cub_gbs": round(gb / tc, 1),
             "cub_frac_measured": round(gb / tc / peak, 4),
             "lscan_us": round(tl * 1e6, 1), "lscan_gbs": round(gb / tl, 1),
             "lscan_over_cub": round(tc / tl, 3)}
        if dt == "i32":
            stream.synchronize()
            r["same_output"] = bool(torch.equal(y2, ys[c]))
        out[c] = r
        del tmp
    return out


def bench_cpu_parallel(host, n, reps=3):
    """Comparator: a multi-threaded inclusive scan on all host cores
    (reduce-then-scan over one chunk per thread, libcpuscan.so beside
    liblscan.so), the counterpart of the paper's parallel-CPU comparison,
    on the headline's arrays in host memory; best of `reps` per scan."""
    import ctypes

    import numpy as np

    from paper_1604_04815_gb300 import build as _build
    if not os.path.exists(_build.CPU_LIB):
        return {"unavailable": "libcpuscan.so was not built (no C compiler?)"}
    lib = ctypes.CDLL(_build.CPU_LIB)
    lib.cpuscan_inclusive.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
    threads = max(1, min(256, os.cpu_count() or 1))
    out = {"n": n, "threads": threads,
           "method": "reduce-then-scan, one contiguous chunk per thread (pthreads)"}
    tot_t = 0.0
    for c, op, dt in CASES:
        x = host[c]
        y = np.empty_like(x)
        best = None
        for _ in range(reps):
            t0 = time.perf_counter()
            if lib.cpuscan_inclusive(0 if op == "add" else 1, 0 if dt == "i32" else 1,
                                     x.ctypes.data, y.ctypes.data, n, threads) != 0:
                return {"unavailable": "host scan failed"}
            t = time.perf_counter() - t0
            best = t if best is None else min(best, t)
        tot_t += best
        out[c] = {"gbs": round(8 * n / best / 1e9, 2)}
        del y
    out["gbs"] = round(len(CASES) * 8 * n / tot_t / 1e9, 2)
    return out


def host_link_ceiling(dev, nbytes=1 << 30, reps=3):
    """Plain pinned copies on the same box: host->device alone, device->host
    alone, and both at once on two streams.  The duplex figure in the scan
    metric (bytes in + bytes out per second) is the ceiling of an end-to-end
    scan of host arrays."""
    import torch
    h_in = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d_a = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d_b = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn):
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        return best
    with torch.cuda.stream(s1):
        d_a.copy_(h_in, non_blocking=True)
    torch.cuda.synchronize()

    def h2d():
        with torch.cuda.stream(s1):
            d_a.copy_(h_in, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s2):
            h_out.copy_(d_b, non_blocking=True)

    def both():
        h2d()
        d2h()
    t_in, t_out, t_both = timed(h2d), timed(d2h), timed(both)
    res = {"h2d_gbs": round(nbytes / t_in / 1e9, 1),
           "d2h_gbs": round(nbytes / t_out / 1e9, 1),
           "duplex_gbs": round(2 * nbytes / t_both / 1e9, 1),
           "bytes_each_way": nbytes,
           "method": "torch copy_ of pinned uint8 buffers, best of "
                     f"{reps}, wall clock around a device synchronize"}
    del h_in, h_out, d_a, d_b
    return res


def bench_select(args, dev, stream, peak, log2n=28):
    """Stream compaction of int32 values by byte flags, half of them kept,
    in one pass.  Algorithmic bytes: n flags + 4n values read + 4k kept
    values written."""
    import torch

    import paper_1604_04815_gb300 as lscan
    n = 1 << log2n
    g = torch.Generator(device=dev)
    g.manual_seed(9)
    x = torch.randint(-1000, 1001, (n,), device=dev, dtype=torch.int32,
                      generator=g)
    flags = (torch.rand(n, device=dev, generator=g) < 0.5).to(torch.uint8)
    out = torch.empty_like(x)
    with torch.cuda.stream(stream):
        def run():
            lscan.select_flagged(x, flags, out=out, stream=stream)
        for _ in range(3):
            run()
        t = _time_launches(stream, run, 10)
        _, count = lscan.select_flagged(x, flags, out=out, stream=stream)
    lscan.stream_status(stream)
    k = int(count.item())
    ok = k == int(flags.sum().item()) and bool(
        torch.equal(out[:k], x[flags.bool()]))
    nbytes = n + 4 * n + 4 * k
    gbs = nbytes / t / 1e9
    return {"n": n, "dtype": "i32", "kept": k, "us": round(t * 1e6, 1),
            "gbs": round(gbs, 1), "frac_measured": round(gbs / peak, 4),
            "geps": round(n / t / 1e9, 2), "result_check": ok}


def bench_radix(args, dev, stream, peak, log2n=28):
    """Radix-sort digit offsets of 2^log2n uniform uint32 keys with 8-bit
    digits (4 positions x 256 buckets) in one pass.  Algorithmic bytes: the
    keys, 4 B each (the 8 KiB of counters and offsets are negligible)."""
    import torch

    import paper_1604_04815_gb300 as lscan
    n = 1 << log2n
    g = torch.Generator(device=dev)
    g.manual_seed(10)
    keys = torch.randint(0, 2 ** 32, (n,), device=dev, dtype=torch.int64,
                         generator=g).to(torch.int32)
    out = torch.empty((4, 256), dtype=torch.int64, device=dev)
    with torch.cuda.stream(stream):
        def run():
            lscan.radix_offsets(keys, 8, out=out, stream=stream)
        for _ in range(3):
            run()
        t = _time_launches(stream, run, 10)
        # sanity check on the device (not a parity claim): the offsets of
        # digit 0 against torch's own histogram of that digit
        h0 = torch.bincount((keys & 255).long(), minlength=256)
        ok = bool(torch.equal(out[0], torch.cumsum(h0, 0) - h0))
    gbs = 4 * n / t / 1e9
    return {"n": n, "key": "u32", "digit_bits": 8, "us": round(t * 1e6, 1),
            "gbs": round(gbs, 1), "frac_measured": round(gbs / peak, 4),
            "gkeys_per_s": round(n / t / 1e9, 2), "result_check": ok}


def bench_small(args, dev, stream):
    """The 2^20-element int32 add (4 MiB in + out): it fits in L2, so it is
    reported as latency per launch, warm (inputs L2-resident, launches back
    to back) and cold (a 256 MiB buffer written between launches evicts
    L2)."""
    import torch

    import paper_1604_04815_gb300 as lscan
    n = 1 << 20
    g = torch.Generator(device=dev)
    g.manual_seed(8)
    x = torch.randint(-1000, 1001, (n,), device=dev, dtype=torch.int32,
                      generator=g)
    y = torch.empty_like(x)
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)
    with torch.cuda.stream(stream):
        def run():
            lscan.scan(x, "add", True, out=y, stream=stream)
        for _ in range(5):
            run()
        warm = _time_launches(stream, run, 50)
        cold = []
        for i in range(20):
            flush.fill_(i)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            e1.synchronize()
            cold.append(e0.elapsed_time(e1) / 1e3)
        # a tiny array (the single-CTA kernel): per call through Python, and
        # on the device from a CUDA graph of 100 captured launches (the
        # tiny path allocates nothing, so it can be captured directly)
        xt, yt = x[:1000], y[:1000]
        def run_tiny():
            lscan.scan(xt, "add", True, out=yt, stream=stream)
        for _ in range(5):
            run_tiny()
        tiny = _time_launches(stream, run_tiny, 200)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            for _ in range(100):
                lscan.scan(xt, "add", True, out=yt,
                           stream=torch.cuda.current_stream())
        graph.replay()
        tiny_graph = _time_launches(stream, graph.replay, 10) / 100
    lscan.stream_status(stream)
    cold = float(np.median(cold))
    return {"n": n, "dtype": "i32", "op": "add",
            "warm_us_per_launch": round(warm * 1e6, 2),
            "warm_gbs": round(8 * n / warm / 1e9, 1),
            "cold_us_per_launch": round(cold * 1e6, 2),
            "cold_gbs": round(8 * n / cold / 1e9, 1),
            "n1000_us_per_call": round(tiny * 1e6, 2),
            "n1000_us_per_launch_in_graph": round(tiny_graph * 1e6, 2)}


def bench_batched(args, dev, stream, peak):
    import torch

    import paper_1604_04815_gb300 as lscan
    from paper_1604_04815_gb300 import _lib, workloads
    out = {}
    sp = stream.cuda_stream
    for dt in ("i32", "f32"):
        x, off = workloads.batched(dt)
        total = int(off[-1])
        xd = torch.from_numpy(x).to(dev)
        yd = torch.empty_like(xd)
        od = torch.from_numpy(off).to(dev)
        tuned_cfg = None
        if args.config == 0:
            st, res = _lib.lscan_autotune(
                _lib.LSCAN_ADD, _lib.LSCAN_I32 if dt == "i32" else _lib.LSCAN_F32,
                1, xd.data_ptr(), yd.data_ptr(), total, od.data_ptr(),
                len(off) - 1, reps=args.tune_reps, stream=sp)
            _lib.check(st, "lscan_autotune (batched)")
            tuned_cfg = res["config"]
        g = lscan.Graph.batched(xd, od, yd)
        reps = max(3, args.steps)
        for _ in range(3):
            g.launch(stream)
        stream.synchronize()
        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        e0.record(stream)
        for _ in range(reps):
            g.launch(stream)
        e1.record(stream)
        stream.synchronize()
        g.status()
        tg = e0.elapsed_time(e1) / 1e3 / reps
        # per-array: one plain launch per segment
        opcode = _lib.LSCAN_ADD
        dcode = _lib.LSCAN_I32 if dt == "i32" else _lib.LSCAN_F32
        es = 4
        starts = off[:-1].tolist()
        lens = np.diff(off).tolist()
        xp, yp = xd.data_ptr(), yd.data_ptr()

        def per_array():
            for a, ln in zip(starts, lens):
                st = _lib.lscan_inclusive(opcode, dcode, xp + a * es,
                                          yp + a * es, ln, sp)
                if st:
                    raise RuntimeError(_lib.strerror(st))
        per_array()
        stream.synchronize()
        e0.record(stream)
        per_array()
        e1.record(stream)
        stream.synchronize()
        tp = e0.elapsed_time(e1) / 1e3
        _lib.check(_lib.lscan_stream_status(sp), "batched")
        nbytes = 2 * total * es
        out[dt] = {"segments": len(lens), "elements": total,
                   "tuned_config": tuned_cfg,
                   "graph_gbs": round(nbytes / tg / 1e9, 1),
                   "graph_frac_measured": round(nbytes / tg / 1e9 / peak, 4),
                   "per_array_gbs": round(nbytes / tp / 1e9, 1),
                   "speedup_vs_per_array": round(tp / tg, 2)}
        g.close()
        del xd, yd, od
        torch.cuda.empty_cache()
    return out


SIZE_CLASSES = [(10, 14), (14, 18), (18, 22), (22, 25)]


def bench_serving(args, dev, peak, n_req, fracs, seed=6):
    """Poisson stream of scan requests through lscan_server_replay.

    Request mix: sizes round(2^(10 + 14 U)), dtype int32/fp32/bf16 at
    50/35/15 %, op add/max 50/50, inclusive; inputs are slices of a device
    resident synthetic array per dtype, outputs are allocated by the server
    from its 16 GiB budget.  First a closed-loop run (every request arrives at
    t = 0) gives the saturation rate; then open-loop Poisson runs at the given
    fractions of it.  Latency = completion - scheduled arrival."""
    import torch

    import paper_1604_04815_gb300 as lscan
    from paper_1604_04815_gb300 import workloads
    rng = np.random.default_rng(seed)
    lake_n = 1 << 27  # per dtype: larger than the 129 MB L2
    lakes = {
        torch.int32: torch.from_numpy(rng.integers(
            -(1 << 15), (1 << 15) + 1, size=lake_n, dtype=np.int32)).to(dev),
        torch.float32: torch.from_numpy(rng.random(
            size=lake_n, dtype=np.float32)).to(dev),
        torch.bfloat16: torch.from_numpy(workloads.f32_to_bf16_bits(
            rng.random(size=lake_n, dtype=np.float32)).view(np.int16)).to(
                dev).view(torch.bfloat16),
    }
    mix = workloads.serving_requests(n_req, seed=seed)
    tdt = {"i32": torch.int32, "f32": torch.float32, "bf16": torch.bfloat16}
    base = []
    nbytes = 0
    for r in mix:
        t = tdt[r["dtype"]]
        lk = lakes[t]
        es = lk.element_size()
        off = int(rng.integers(0, lake_n - r["n"])) // 8 * 8
        out_es = 4 if (r["op"] == "add" and r["dtype"] == "bf16") else es
        nbytes += r["n"] * (es + out_es)
        base.append([r["op"], t, True, lk.data_ptr() + off * es, r["n"]])
    n_streams = getattr(args, "serving_streams", 2)
    srv = lscan.Server(budget_bytes=16 << 30, n_streams=n_streams)
    small_max = getattr(args, "serving_small_max", 1 << 14)
    bulk_tiles = getattr(args, "serving_bulk_tiles", 16384)
    reserve = getattr(args, "serving_reserve_sms", 8)
    srv.set_lanes(small_max, bulk_tiles, reserve)
    out = {"requests": n_req, "budget_gib": 16, "n_streams": n_streams,
           "lanes": {"small_max_elems": small_max,
                     "bulk_batch_tiles": bulk_tiles, "reserve_sms": reserve},
           "mean_elems": float(np.mean([r["n"] for r in mix]))}
    try:
        # warm-up (kernels, scratch, pool) on a short closed-loop burst
        srv.replay([b + [0.0] for b in base[: min(200, n_req)]])
        stats, wall = srv.replay([b + [0.0] for b in base])
        sat_rps = n_req / (wall / 1e6)
        out["saturation"] = {"gbs": round(nbytes / (wall / 1e6) / 1e9, 1),
                             "frac_measured": round(
                                 nbytes / (wall / 1e6) / 1e9 / peak, 4),
                             "req_per_s": round(sat_rps, 1)}
        runs = []
        for f in fracs:
            rate = f * sat_rps
            gaps = workloads.poisson_gaps(n_req, rate, seed=seed + 10)
            arr = np.cumsum(gaps) * 1e6
            arr -= arr[0]
            stats, wall = srv.replay([b + [float(a)] for b, a in
                                      zip(base, arr)])
            lat = np.array([s["done_us"] - s["submit_us"] for s in stats])
            ns = np.array([s["n"] for s in stats])
            ok = all(s["status"] == 0 for s in stats)
            per = {}
            for lo, hi in SIZE_CLASSES:
                m = (ns >= (1 << lo)) & (ns < (1 << hi))
                if m.any():
                    per[f"2^{lo}-2^{hi}"] = {
                        "count": int(m.sum()),
                        "p50_us": round(float(np.percentile(lat[m], 50)), 1),
                        "p99_us": round(float(np.percentile(lat[m], 99)), 1)}
            small = per.get(f"2^{SIZE_CLASSES[0][0]}-2^{SIZE_CLASSES[0][1]}")
            large = per.get(f"2^{SIZE_CLASSES[-1][0]}-2^{SIZE_CLASSES[-1][1]}")
            runs.append({"load": f, "offered_req_per_s": round(rate, 1),
                         "gbs": round(nbytes / (wall / 1e6) / 1e9, 1),
                         "p50_us": round(float(np.percentile(lat, 50)), 1),
                         "p99_us": round(float(np.percentile(lat, 99)), 1),
                         "mean_batch": round(float(np.mean(
                             [s["batch_requests"] for s in stats])), 1),
                         "all_ok": ok, "size_classes": per,
                         "large_over_small_p50": round(
                             large["p50_us"] / small["p50_us"], 2)
                         if small and large else None})
        out["runs"] = runs
    finally:
        srv.close()
        del lakes
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lscan", choices=["lscan", "reference"])
    ap.add_argument("--config", type=int, default=0)
    ap.add_argument("--tune-reps", type=int, default=5,
                    help="timed launches per configuration in the autotuner "
                         "(median kept)")
    ap.add_argument("--carry", type=int, default=0)
    ap.add_argument("--sharded", action="store_true",
                    help="with N > 1 ranks: each rank's arrays are shards of "
                         "one N-times-longer array (a collective per scan) "
                         "instead of independent replicas")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-radix", action="store_true")
    ap.add_argument("--no-cub", action="store_true",
                    help="skip the CUB device-scan comparator")
    ap.add_argument("--no-cpu-parallel", action="store_true",
                    help="skip the multi-threaded host-scan comparator")
    ap.add_argument("--e2e-chunk", type=int, default=0,
                    help="elements per chunk of lscan_scan_host (0 = the "
                         "library's ramped schedule)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-dtypes", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-select", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-bf16", action="store_true")
    ap.add_argument("--no-link", action="store_true",
                    help="skip the plain pinned-copy ceiling of the e2e leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=20000)
    ap.add_argument("--serving-loads", default="0.5,0.8,0.95",
                    help="offered loads as fractions of the saturation rate")
    ap.add_argument("--serving-streams", type=int, default=2)
    ap.add_argument("--serving-small-max", type=int, default=1 << 14,
                    help="largest request (elements) of the resident lane; "
                         "0 = every request in the bulk lane")
    ap.add_argument("--serving-bulk-tiles", type=int, default=32768,
                    help="tiles per bulk-lane batch")
    ap.add_argument("--serving-reserve-sms", type=int, default=4,
                    help="SMs kept for the resident lane's kernel")
    ap.add_argument("--log2n", type=int, default=28,
                    help="array size 2^k (28 = the benchmarked workload; "
                         "smaller only for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    global N
    N = 1 << args.log2n
    ws, rank, local = _dist()
    if ws > 1 and args.impl != "reference":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    try:
        if args.impl == "reference":
            return run_reference(args, ws, rank)
        return run_gpu(args, ws, rank, local)
    finally:
        if ws > 1 and args.impl != "reference":
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
