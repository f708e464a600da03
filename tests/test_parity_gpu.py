"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element, over every kind, tile configuration, inclusive/exclusive,
ragged sizes, unaligned and in-place buffers, both carry protocols and the
batched (segmented) mode.  Integer and max scans must be bit-exact; float add
must stay within |err_j| <= c * S_j (c = 1e-5 for the fp32/FP64 carry paths,
2.5e-7 for the compensated path)."""
import numpy as np
import pytest
import torch

from gpu_util import (assert_matches, run_c_abi, to_device, to_host, LDT, LOP,
                      PREC_CODE, TEST_WAIT_NS, out_torch_dtype)
from paper_1604_04815_gb300 import _lib
from paper_1604_04815_gb300.workloads import (random_array, batched_lengths,
                                              offsets_from_lengths)

pytestmark = pytest.mark.gpu

# (op, dtype, precision, bf16 output)
KINDS = [
    ("add", "i32", None, False),
    ("max", "i32", None, False),
    ("max", "f32", None, False),
    ("max", "bf16", None, False),
    ("add", "f32", "plain", False),
    ("add", "f32", "f64", False),
    ("add", "f32", "comp", False),
    ("add", "bf16", "plain", False),
    ("add", "bf16", "f64", False),
    ("add", "bf16", "comp", False),
    ("add", "bf16", "plain", True),
    ("add", "bf16", "f64", True),
    ("add", "bf16", "comp", True),
    # the double-float carry (the default precision of float add)
    ("add", "f32", "df", False),
    ("add", "bf16", "df", False),
    ("add", "bf16", "df", True),
    # the paper's 64-bit types (Table 2)
    ("add", "i64", None, False),
    ("max", "i64", None, False),
    ("max", "f64", None, False),
    ("add", "f64", None, False),
]
KIND_IDS = [f"{o}-{d}-{p or 'exact'}{'-bf16out' if b else ''}"
            for o, d, p, b in KINDS]


def _pick(*ids):
    """(kinds, ids) of the named kinds, for parametrize."""
    idx = [KIND_IDS.index(i) for i in ids]
    return [KINDS[i] for i in idx], [KIND_IDS[i] for i in idx]


CHAINED_KINDS = _pick("add-i32-exact", "max-i32-exact", "add-f32-f64",
                      "add-f32-df", "add-bf16-comp", "add-i64-exact",
                      "add-f64-exact")
BATCHED_KINDS = _pick("add-i32-exact", "max-i32-exact", "max-f32-exact",
                      "max-bf16-exact", "add-f32-f64", "add-f32-comp",
                      "add-f32-df", "add-bf16-f64", "add-bf16-df",
                      "add-bf16-df-bf16out", "add-bf16-comp-bf16out",
                      "add-i64-exact", "max-i64-exact", "max-f64-exact",
                      "add-f64-exact")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_04815_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    _lib.load()
    _lib.lscan_set_wait_limit_ns(TEST_WAIT_NS)
    yield


def _input(op, dtype, n, seed):
    rng = np.random.default_rng(seed)
    if dtype in ("i32", "i64"):
        return random_array(dtype, n, rng, kind="full" if op == "max" or
                            seed % 2 else "uniform")
    return random_array(dtype, n, rng, kind="signed")


def _tile(config, dtype):
    return _lib.lscan_config_info(config, LDT[dtype])["tile"]


def _sizes(tile):
    return [1, 2, 31, 33, 1000, tile - 1, tile, tile + 1, 7 * tile + 123]


# every tile configuration the autotuner may choose for a single array
ALL_CONFIGS = list(range(1, 18))


@pytest.mark.parametrize("config", ALL_CONFIGS)
@pytest.mark.parametrize("inclusive", [True, False], ids=["incl", "excl"])
@pytest.mark.parametrize("kind", KINDS, ids=KIND_IDS)
def test_sizes_configs(kind, inclusive, config):
    op, dtype, prec, ob = kind
    for i, n in enumerate(_sizes(_tile(config, dtype))):
        x = _input(op, dtype, n, seed=1000 * config + i)
        y = run_c_abi(op, dtype, to_device(x, dtype), inclusive, prec=prec,
                      config=config, out_bf16=ob)
        assert_matches(op, dtype, x, to_host(y), inclusive, prec or "f64",
                       out_bf16=ob)


def test_empty_input_launches_nothing():
    before = _lib.lscan_launch_count()
    x = torch.empty(0, dtype=torch.int32, device="cuda")
    y = torch.empty(0, dtype=torch.int32, device="cuda")
    st = _lib.lscan_inclusive(_lib.LSCAN_ADD, _lib.LSCAN_I32, x.data_ptr(),
                              y.data_ptr(), 0,
                              torch.cuda.current_stream().cuda_stream)
    assert st == _lib.LSCAN_OK
    assert _lib.lscan_launch_count() == before


@pytest.mark.parametrize("inclusive", [True, False], ids=["incl", "excl"])
@pytest.mark.parametrize("kind", KINDS, ids=KIND_IDS)
def test_unaligned_pointers(kind, inclusive):
    """x and/or y not 16-byte aligned: the plain-load path."""
    op, dtype, prec, ob = kind
    for (px, py), n in (((1, 0), 5000), ((0, 1), 70001), ((3, 1), 1)):
        x = _input(op, dtype, n, seed=77 + n)
        xd = to_device(x, dtype, pad_front=px)
        odt = (torch.bfloat16 if ob else torch.float32) if (
            op == "add" and dtype == "bf16") else xd.dtype
        yb = torch.empty(n + py, dtype=odt, device="cuda")
        y = run_c_abi(op, dtype, xd, inclusive, prec=prec, out_bf16=ob,
                      y_dev=yb[py:])
        assert_matches(op, dtype, x, to_host(y), inclusive, prec or "f64",
                       out_bf16=ob)


@pytest.mark.parametrize("config", [1, 3])
@pytest.mark.parametrize("kind", [k for k in KINDS
                                  if not (k[0] == "add" and k[1] == "bf16")],
                         ids=[i for k, i in zip(KINDS, KIND_IDS)
                              if not (k[0] == "add" and k[1] == "bf16")])
def test_in_place(kind, config):
    """y == x (Section 4.5): every element is read before it is written."""
    op, dtype, prec, ob = kind
    n = 9 * _tile(config, dtype) + 5
    x = _input(op, dtype, n, seed=5)
    xd = to_device(x, dtype)
    y = run_c_abi(op, dtype, xd, True, prec=prec, config=config, y_dev=xd)
    assert y.data_ptr() == xd.data_ptr()
    assert_matches(op, dtype, x, to_host(y), True, prec or "f64")


@pytest.mark.parametrize("inclusive", [True, False], ids=["incl", "excl"])
@pytest.mark.parametrize("kind", CHAINED_KINDS[0], ids=CHAINED_KINDS[1])
def test_chained_carry(kind, inclusive):
    """The paper's neighbour-to-neighbour hand-off (Algorithm 4)."""
    op, dtype, prec, ob = kind
    for n in (1, 4096 * 3 + 1, (1 << 20) + 7):
        x = _input(op, dtype, n, seed=n)
        y = run_c_abi(op, dtype, to_device(x, dtype), inclusive, prec=prec,
                      carry=_lib.LSCAN_CARRY_CHAINED, out_bf16=ob)
        assert_matches(op, dtype, x, to_host(y), inclusive, prec or "f64",
                       out_bf16=ob)


@pytest.mark.parametrize("prec", ["plain", "f64", "comp"])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_float_integer_values_bit_exact(dtype, prec):
    """Integer-valued inputs keep every fp32 prefix exact (< 2^24), so every
    float path must reproduce the oracle bit for bit."""
    rng = np.random.default_rng(12)
    n = (1 << 20) + 3
    x = random_array(dtype, n, rng, kind="intval")
    y = run_c_abi("add", dtype, to_device(x, dtype), True, prec=prec)
    got = to_host(y).astype(np.float64)
    want = __import__("oracle").scan("add", dtype, x, True)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("kind", KINDS, ids=KIND_IDS)
def test_one_mebi(kind):
    op, dtype, prec, ob = kind
    n = (1 << 20) + 7
    x = _input(op, dtype, n, seed=3)
    for inclusive in (True, False):
        y = run_c_abi(op, dtype, to_device(x, dtype), inclusive, prec=prec,
                      out_bf16=ob)
        assert_matches(op, dtype, x, to_host(y), inclusive, prec or "f64",
                       out_bf16=ob)


def test_small_i32_workload_bit_exact():
    """The 2^20 int32 workload (uniform [-1000, 1000], seed 0)."""
    from paper_1604_04815_gb300.workloads import small_i32
    x = small_i32()
    y = run_c_abi("add", "i32", to_device(x, "i32"), True)
    assert_matches("add", "i32", x, to_host(y), True)


# ------------------------------------------------------------ batched mode
def _offsets(kind, rng):
    if kind == "mixed":
        lens = [0, 1, 0, 5, 2048, 0, 2, 4095, 4096, 4097, 1, 30000, 0, 3]
    elif kind == "tiny":
        lens = [1] * 4096
    elif kind == "huge_plus_tiny":
        lens = [300001] + [1, 2, 0, 3] * 500
    elif kind == "empty_tail":
        lens = [10, 0, 0, 0]
    elif kind == "tile_aligned":
        # heads only at tile starts for every config (tiles of 2^11..2^14
        # elements): tiles take the unsegmented code with an identity carry
        lens = [16384, 32768, 0, 49152, 16384, 5]
    else:  # log-uniform like the batched workload, smaller
        lens = batched_lengths(300, max_log2=14, seed=int(rng.integers(1e6)))
    return offsets_from_lengths(lens)


@pytest.mark.parametrize("pattern", ["mixed", "tiny", "huge_plus_tiny",
                                     "empty_tail", "loguniform",
                                     "tile_aligned"])
@pytest.mark.parametrize("inclusive", [True, False], ids=["incl", "excl"])
@pytest.mark.parametrize("kind", BATCHED_KINDS[0], ids=BATCHED_KINDS[1])
def test_batched(kind, inclusive, pattern):
    op, dtype, prec, ob = kind
    rng = np.random.default_rng(sum(map(ord, pattern)))
    off = _offsets(pattern, rng)
    n = int(off[-1])
    x = _input(op, dtype, n, seed=9)
    for config in range(1, 7):  # the configurations built for batched scans
        xd = to_device(x, dtype)
        od = torch.from_numpy(off).cuda()
        y = torch.empty(n, dtype=out_torch_dtype(op, dtype, ob), device="cuda")
        opts = _lib.make_options(precision=PREC_CODE[prec] if prec else 0,
                                 config=config,
                                 out_dtype=_lib.LSCAN_BF16 if ob else 0)
        s = torch.cuda.current_stream().cuda_stream
        st = _lib.lscan_batched(LOP[op], LDT[dtype], int(inclusive),
                                xd.data_ptr(), y.data_ptr(), od.data_ptr(),
                                len(off) - 1, n, opts, s)
        assert st == _lib.LSCAN_OK
        assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
        assert_matches(op, dtype, x, to_host(y), inclusive, prec or "f64",
                       out_bf16=ob, offsets=off)


def test_batched_unaligned_and_chained():
    off = _offsets("mixed", None)
    n = int(off[-1])
    x = _input("add", "i32", n, seed=4)
    xd = to_device(x, "i32", pad_front=1)
    od = torch.from_numpy(off).cuda()
    for carry in (_lib.LSCAN_CARRY_LOOKBACK, _lib.LSCAN_CARRY_CHAINED):
        y = torch.empty(n, dtype=torch.int32, device="cuda")
        opts = _lib.make_options(carry=carry)
        s = torch.cuda.current_stream().cuda_stream
        st = _lib.lscan_batched(LOP["add"], LDT["i32"], 1, xd.data_ptr(),
                                y.data_ptr(), od.data_ptr(), len(off) - 1, n,
                                opts, s)
        assert st == _lib.LSCAN_OK
        assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
        assert_matches("add", "i32", x, to_host(y), True, offsets=off)


# -------------------------------------------------- robustness of the carry
def test_many_launches_epoch_and_ticket_rearm():
    """Hundreds of back-to-back launches of varying size on one stream: the
    kernel re-arms the ticket and advances the epoch itself."""
    rng = np.random.default_rng(21)
    xs = [random_array("i32", int(n), rng, kind="full")
          for n in rng.integers(1, 200000, size=40)]
    devs = [to_device(x, "i32") for x in xs]
    outs = []
    for rep in range(5):
        for xd in devs:
            outs.append(run_c_abi("add", "i32", xd, True, config=1,
                                  check_status=False))
    assert _lib.lscan_stream_status(
        torch.cuda.current_stream().cuda_stream) == _lib.LSCAN_OK
    for rep in range(5):
        for i, x in enumerate(xs):
            assert_matches("add", "i32", x, to_host(outs[rep * len(xs) + i]))


def test_chained_scans_back_to_back_in_one_stream():
    """Each scan reads the previous one's output, queued without a host
    synchronisation: kernels launched with programmatic stream serialization
    may start while their predecessor finishes, and must still see all of
    its output (persistent -> persistent -> single-CTA -> persistent)."""
    import oracle
    rng = np.random.default_rng(29)
    n = 3_000_017
    x = random_array("i32", n, rng, kind="full")
    xd = to_device(x, "i32")
    y1 = run_c_abi("add", "i32", xd, True, check_status=False)
    y2 = run_c_abi("add", "i32", y1, True, check_status=False)
    y3 = run_c_abi("add", "i32", y2[:4000], False, check_status=False)
    y4 = run_c_abi("add", "i32", y2, False, check_status=False)
    s = torch.cuda.current_stream().cuda_stream
    assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
    w1 = oracle.scan("add", "i32", x, True)
    w2 = oracle.scan("add", "i32", w1, True)
    assert np.array_equal(to_host(y1), w1)
    assert np.array_equal(to_host(y2), w2)
    assert np.array_equal(to_host(y3), oracle.scan("add", "i32", w2[:4000], False))
    assert np.array_equal(to_host(y4), oracle.scan("add", "i32", w2, False))


def test_new_host_thread_on_a_used_stream():
    """A host thread whose first library call reuses a stream (and so its
    scratch) set up by another thread: it makes no CUDA call that binds a
    context before the launch builds the tile copies' tensor maps, which
    must still work.  Every kind's default configuration, full tiles and a
    ragged tail."""
    import threading
    s = torch.cuda.Stream()
    rng = np.random.default_rng(23)
    cases = [("add", "i32"), ("max", "f32"), ("add", "f32"), ("max", "bf16"),
             ("add", "f64")]
    xs = [random_array(dt, (1 << 21) + 13, rng, kind="full") for _, dt in cases]
    ds = [to_device(x, dt) for x, (_, dt) in zip(xs, cases)]
    ys = [torch.empty(d.shape[0], dtype=out_torch_dtype(op, dt, False), device="cuda")
          for d, (op, dt) in zip(ds, cases)]
    with torch.cuda.stream(s):
        run_c_abi("add", "i32", ds[0], True, y_dev=ys[0])  # scratch set up here
    s.synchronize()
    errs = []

    def worker():
        try:
            for d, y, (op, dt) in zip(ds, ys, cases):
                st = _lib.lscan_scan(LOP[op], LDT[dt], 1, d.data_ptr(),
                                     y.data_ptr(), d.shape[0], None, s.cuda_stream)
                assert st == _lib.LSCAN_OK, (op, dt, _lib.strerror(st))
        except Exception as e:  # reported on the main thread
            errs.append(e)

    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert not errs, errs
    s.synchronize()
    assert _lib.lscan_stream_status(s.cuda_stream) == _lib.LSCAN_OK
    for x, y, (op, dt) in zip(xs, ys, cases):
        assert_matches(op, dt, x, to_host(y))


def test_concurrent_streams_independent_scratch():
    streams = [torch.cuda.Stream() for _ in range(4)]
    rng = np.random.default_rng(5)
    xs = [random_array("i32", 3_000_000 + 17 * i, rng, kind="full")
          for i in range(4)]
    devs = [to_device(x, "i32") for x in xs]
    torch.cuda.synchronize()
    ys = []
    for s, xd in zip(streams, devs):
        with torch.cuda.stream(s):
            ys.append(run_c_abi("add", "i32", xd, True, check_status=False))
    for s in streams:
        assert _lib.lscan_stream_status(s.cuda_stream) == _lib.LSCAN_OK
    for x, y in zip(xs, ys):
        assert_matches("add", "i32", x, to_host(y))


def test_wait_timeout_reports_and_recovers():
    """A tile that never publishes (host-injected): its successors' bounded
    waits run out, the launch finishes, the host gets LSCAN_ERR_TIMEOUT, and
    the next launch on the same stream is correct."""
    s = torch.cuda.current_stream().cuda_stream
    x = random_array("i32", 64 * 4096, np.random.default_rng(1))
    xd = to_device(x, "i32")
    assert _lib.lscan_set_wait_limit_ns(20_000_000) == _lib.LSCAN_OK
    try:
        for carry in (_lib.LSCAN_CARRY_LOOKBACK, _lib.LSCAN_CARRY_CHAINED):
            _lib.lscan_debug_skip_publish(3)
            run_c_abi("add", "i32", xd, True, carry=carry, config=2,
                      check_status=False)
            assert _lib.lscan_stream_status(s) == _lib.LSCAN_ERR_TIMEOUT
            y = run_c_abi("add", "i32", xd, True, carry=carry, config=2)
            assert_matches("add", "i32", x, to_host(y))
    finally:
        _lib.lscan_set_wait_limit_ns(TEST_WAIT_NS)
        _lib.lscan_debug_skip_publish(-1)


def test_graph_replay_batched():
    import paper_1604_04815_gb300 as lscan
    off = _offsets("loguniform", np.random.default_rng(3))
    n = int(off[-1])
    rng = np.random.default_rng(8)
    x = random_array("i32", n, rng, kind="full")
    xd = to_device(x, "i32")
    od = torch.from_numpy(off).cuda()
    y = torch.empty_like(xd)
    g = lscan.Graph.batched(xd, od, y)
    try:
        for rep in range(3):
            x = random_array("i32", n, rng, kind="full")
            xd.copy_(torch.from_numpy(x))
            g.launch()
            g.status()
            assert_matches("add", "i32", x, to_host(y), offsets=off)
    finally:
        g.close()


def test_graph_replay_single():
    import paper_1604_04815_gb300 as lscan
    rng = np.random.default_rng(9)
    n = 5_000_001
    x = random_array("f32", n, rng, kind="signed")
    xd = to_device(x, "f32")
    y = torch.empty_like(xd)
    g = lscan.Graph.scan(xd, y)
    try:
        for _ in range(3):
            g.launch()
            g.status()
            assert_matches("add", "f32", x, to_host(y))
    finally:
        g.close()


def test_torch_front_matches_c_abi():
    import paper_1604_04815_gb300 as lscan
    x = random_array("bf16", 123457, np.random.default_rng(2), kind="signed")
    xd = to_device(x, "bf16")
    a = lscan.inclusive(xd)
    b = run_c_abi("add", "bf16", xd, True)
    lscan.stream_status()
    assert torch.equal(a, b)
    assert a.dtype == torch.float32


def test_autotune_picks_a_config_and_stays_correct(tmp_path):
    """The autotuner times every configuration, records the fastest for this
    size class, and the tuned launch (config 0) still matches the oracle."""
    for op, dtype in (("add", "i32"), ("add", "f32")):
        x = _input(op, dtype, (1 << 22) + 3, seed=2)
        xd = to_device(x, dtype)
        y = torch.empty_like(xd)
        s = torch.cuda.current_stream().cuda_stream
        st, res = _lib.lscan_autotune(LOP[op], LDT[dtype], 1, xd.data_ptr(),
                                      y.data_ptr(), xd.shape[0], reps=5,
                                      stream=s)
        assert st == _lib.LSCAN_OK
        assert 1 <= res["config"] <= _lib.lscan_num_configs()
        assert res["n_timed"] == _lib.lscan_num_configs()
        assert res["ms"] > 0 and res["ms"] == min(
            [res["ms"]] + list(res["ms_by_config"].values()))
        assert res["default_ms"] >= res["ms"]
        # 1025 tiles at most: the chained carry is timed too
        assert res["chained_ms"] > 0
        assert_matches(op, dtype, x, to_host(y))       # y holds a real scan
        y2 = run_c_abi(op, dtype, xd, True)             # tuned configuration
        assert_matches(op, dtype, x, to_host(y2))
    assert _lib.lscan_tune_save(tmp_path / "t.json") == _lib.LSCAN_OK
    assert _lib.lscan_tune_reset() == _lib.LSCAN_OK


# ------------------------------------------------------------- carry-in
def _carry_value(op, dtype, ob, x, rng):
    """A carry-in in the output representation (numpy scalar) that matters:
    for max, a value above part of the input."""
    if op == "add" and dtype == "i32":
        return np.int32(rng.integers(-2**31, 2**31))
    if op == "add" and dtype == "i64":
        return np.int64(rng.integers(-2**63, 2**63 - 1, endpoint=True))
    if op == "add" and dtype == "f64":
        return np.float64(rng.choice([-1.0, 1.0]) * rng.random() * 100.0)
    if op == "max":
        if dtype == "bf16":
            from paper_1604_04815_gb300.workloads import bf16_bits_to_f32
            v = np.sort(bf16_bits_to_f32(x))[len(x) * 3 // 5] if len(x) else 0.0
            return np.uint16(np.float32(v).view(np.uint32) >> 16)  # exact
        if dtype in ("i32", "i64", "f64"):
            return np.sort(x)[len(x) * 3 // 5]
        return np.float32(np.sort(x)[len(x) * 3 // 5])
    v = np.float32(rng.choice([-1.0, 1.0]) * rng.random() * 100.0)
    if ob:
        from paper_1604_04815_gb300.workloads import f32_to_bf16_bits
        return f32_to_bf16_bits(np.array([v], dtype=np.float32))[0]
    return v


def _expect_with_carry(op, dtype, ob, want, c):
    """c (+) oracle prefix: exact for int and max, FP64 for float add."""
    from paper_1604_04815_gb300.workloads import bf16_bits_to_f32
    if op == "add" and dtype == "i32":
        return ((want.astype(np.int64) + int(c)) & 0xFFFFFFFF).astype(
            np.uint32).view(np.int32)
    if op == "add" and dtype == "i64":  # mod 2^64
        return (want.view(np.uint64) + np.uint64(int(c) % 2**64)).view(np.int64)
    if op == "max":
        if dtype == "bf16":
            wv = bf16_bits_to_f32(want)
            cv = bf16_bits_to_f32(np.array([c], dtype=np.uint16))[0]
            return np.where(wv > cv, want, np.uint16(c)).astype(np.uint16)
        return np.where(want > c, want, c).astype(want.dtype)
    cv = float(bf16_bits_to_f32(np.array([c], dtype=np.uint16))[0]) if ob \
        else float(c)
    return want + cv, abs(cv)


@pytest.mark.parametrize("inclusive", [True, False], ids=["incl", "excl"])
@pytest.mark.parametrize("kind", KINDS, ids=KIND_IDS)
def test_carry_in(kind, inclusive):
    """y = carry_in (+) scan(x): a shard of a longer scan."""
    import oracle
    from gpu_util import BOUND, BOUND_F64_ADD, DTYPES
    from paper_1604_04815_gb300.workloads import bf16_bits_to_f32
    op, dtype, prec, ob = kind
    rng = np.random.default_rng(77)
    odt = torch.bfloat16 if ob else (
        torch.float32 if (op == "add" and dtype == "bf16") else DTYPES[dtype])
    tile = _tile(2, dtype)
    for config, carry in ((0, 0), (2, 0), (2, _lib.LSCAN_CARRY_CHAINED)):
        for i, n in enumerate([1, 33, tile + 1, 7 * tile + 123]):
            x = _input(op, dtype, n, seed=300 + i)
            c = _carry_value(op, dtype, ob, x, rng)
            ca = np.array([c])
            if odt == torch.bfloat16:
                ca = ca.astype(np.uint16).view(np.int16)
            cdev = torch.from_numpy(ca).cuda().view(odt)
            xd = to_device(x, dtype)
            y = torch.empty(n, dtype=odt, device="cuda")
            opts = _lib.make_options(
                out_dtype=_lib.LSCAN_BF16 if ob else 0,
                precision=PREC_CODE[prec] if prec else 0, carry=carry,
                config=config, carry_in=cdev.data_ptr())
            s = torch.cuda.current_stream().cuda_stream
            st = _lib.lscan_scan(LOP[op], LDT[dtype], int(inclusive),
                                 xd.data_ptr(), y.data_ptr(), n, opts, s)
            assert st == _lib.LSCAN_OK
            assert _lib.lscan_stream_status(s) == _lib.LSCAN_OK
            got = to_host(y)
            want = oracle.scan(op, dtype, x, inclusive)
            if op == "max" or dtype in ("i32", "i64"):
                exp = _expect_with_carry(op, dtype, ob, want, c)
                bits = {"f32": np.uint32, "f64": np.uint64}.get(dtype)
                gb = got.view(bits) if bits else got
                eb = exp.view(bits) if bits else exp
                assert np.array_equal(gb, eb), (config, carry, n)
            else:
                exp, ac = _expect_with_carry(op, dtype, ob, want, c)
                sj = oracle.abs_prefix(dtype, x, inclusive) + ac
                g = (bf16_bits_to_f32(got) if ob else got).astype(np.float64)
                c_rel = BOUND_F64_ADD if dtype == "f64" else BOUND[prec]
                lim = c_rel * sj + (2.0 ** -8 * np.abs(exp) if ob else 0)
                assert np.all(np.abs(g - exp) <= lim), (config, carry, n)


def test_carry_in_is_read_at_each_graph_replay():
    """The carry-in is a device value read in stream order: a graph replays
    with whatever it holds at that time."""
    import paper_1604_04815_gb300 as lscan
    rng = np.random.default_rng(12)
    n = 5 * 4096 + 17
    x = random_array("i32", n, rng, kind="uniform")
    xd = to_device(x, "i32")
    y = torch.empty_like(xd)
    c = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = lscan.Graph.scan(xd, y, carry_in=c)
    try:
        for v in (0, 12345, -7):
            c.fill_(v)
            g.launch()
            g.status()
            want = (np.cumsum(x.astype(np.int64)) + v).astype(np.int32)
            assert np.array_equal(to_host(y), want)
    finally:
        g.close()


# ------------------------------------------------ single-CTA tiny arrays
@pytest.mark.parametrize("inclusive", [True, False], ids=["incl", "excl"])
@pytest.mark.parametrize("kind", KINDS, ids=KIND_IDS)
def test_tiny_arrays(kind, inclusive):
    """n <= 4096 with config 0 takes the single-CTA kernel (one launch, no
    carry); 4097 goes back to the persistent kernel.  Also unaligned, in
    place and with a carry-in."""
    import oracle
    op, dtype, prec, ob = kind
    for i, n in enumerate([1, 2, 31, 257, 1000, 4095, 4096, 4097]):
        x = _input(op, dtype, n, seed=900 + i)
        before = _lib.lscan_launch_count()
        y = run_c_abi(op, dtype, to_device(x, dtype), inclusive, prec=prec,
                      config=0, out_bf16=ob)
        assert _lib.lscan_launch_count() == before + 1
        assert_matches(op, dtype, x, to_host(y), inclusive, prec or "f64",
                       out_bf16=ob)
    # unaligned input and output
    n = 3000
    x = _input(op, dtype, n, seed=950)
    xd = to_device(x, dtype, pad_front=1)
    odt = (torch.bfloat16 if ob else torch.float32) if (
        op == "add" and dtype == "bf16") else xd.dtype
    yb = torch.empty(n + 1, dtype=odt, device="cuda")
    y = run_c_abi(op, dtype, xd, inclusive, prec=prec, out_bf16=ob,
                  y_dev=yb[1:])
    assert_matches(op, dtype, x, to_host(y), inclusive, prec or "f64",
                   out_bf16=ob)
    # in place (same element size only)
    if not (op == "add" and dtype == "bf16"):
        xd = to_device(x, dtype)
        y = run_c_abi(op, dtype, xd, inclusive, prec=prec, y_dev=xd)
        assert_matches(op, dtype, x, to_host(y), inclusive, prec or "f64")
