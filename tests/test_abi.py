"""C-ABI library checks that need no GPU: it builds, loads, exports every
symbol include/lscan.h declares, and rejects bad arguments on the host before
any CUDA call."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_1604_04815_gb300 import build
    build.build()
    from paper_1604_04815_gb300 import _lib
    return _lib


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "lscan.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lscan_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_expected_symbols(lib):
    assert _declared_symbols() == sorted(lib.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in _declared_symbols():
        assert hasattr(so, name), name


# input tile bytes of configurations 1..17 (the autotuner's search space)
TILE_KIB = [8, 16, 32, 16, 32, 32, 16, 32, 8, 16, 32, 64, 16, 32, 32, 16, 48]


def test_version_and_configs(lib):
    assert "sm_103a" in lib.lscan_version()
    assert lib.lscan_num_configs() == len(TILE_KIB)
    for c in range(1, lib.lscan_num_configs() + 1):
        for dt in (lib.LSCAN_I32, lib.LSCAN_F32, lib.LSCAN_BF16,
                   lib.LSCAN_I64, lib.LSCAN_F64):
            info = lib.lscan_config_info(c, dt)
            assert info["tile"] == info["items"] * info["threads"]
            assert info["stages"] >= 2
    # a configuration number means the same input bytes per tile for every
    # element size (bf16 entry 12: 56 KiB, items per thread are capped at 32
    # and a CTA at 1024 threads)
    nc = len(TILE_KIB)
    assert [lib.lscan_config_info(c, lib.LSCAN_I32)["tile"] * 4 // 1024
            for c in range(1, nc + 1)] == TILE_KIB
    assert [lib.lscan_config_info(c, lib.LSCAN_I64)["tile"] * 8 // 1024
            for c in range(1, nc + 1)] == TILE_KIB
    assert [lib.lscan_config_info(c, lib.LSCAN_BF16)["tile"] * 2 // 1024
            for c in range(1, nc + 1)] == TILE_KIB[:11] + [56] + TILE_KIB[12:]


def test_host_argument_checks(lib):
    L = lib
    assert L.lscan_inclusive(L.LSCAN_ADD, L.LSCAN_I32, 16, 32, -1) == \
        L.LSCAN_ERR_INVALID
    assert L.lscan_inclusive(L.LSCAN_ADD, L.LSCAN_I32, None, None, 5) == \
        L.LSCAN_ERR_INVALID
    assert L.lscan_inclusive(L.LSCAN_ADD, 7, 16, 64, 5) == L.LSCAN_ERR_INVALID
    assert L.lscan_inclusive(9, L.LSCAN_I32, 16, 64, 5) == L.LSCAN_ERR_INVALID
    # misaligned element pointers
    assert L.lscan_inclusive(L.LSCAN_ADD, L.LSCAN_I32, 18, 4096, 5) == \
        L.LSCAN_ERR_INVALID
    # partial overlap is rejected; identical ranges are the in-place case
    base = 1 << 20
    assert L.lscan_inclusive(L.LSCAN_ADD, L.LSCAN_I32, base, base + 4, 100) == \
        L.LSCAN_ERR_INVALID
    # bf16 add writes fp32 by default: same start is an overlap, not in-place
    assert L.lscan_inclusive(L.LSCAN_ADD, L.LSCAN_BF16, base, base, 100) == \
        L.LSCAN_ERR_INVALID
    # unsupported output dtype / precision
    o = L.make_options(out_dtype=L.LSCAN_BF16)
    assert L.lscan_scan(L.LSCAN_ADD, L.LSCAN_I32, 1, base, base * 2, 10, o) == \
        L.LSCAN_ERR_UNSUPPORTED
    o = L.make_options(precision=9)
    assert L.lscan_scan(L.LSCAN_ADD, L.LSCAN_F32, 1, base, base * 2, 10, o) == \
        L.LSCAN_ERR_UNSUPPORTED
    o = L.make_options(config=L.lscan_num_configs() + 1)
    assert L.lscan_scan(L.LSCAN_ADD, L.LSCAN_F32, 1, base, base * 2, 10, o) == \
        L.LSCAN_ERR_INVALID
    # batched scans have the first six configurations only
    o = L.make_options(config=7)
    assert L.lscan_batched(L.LSCAN_ADD, L.LSCAN_I32, 1, base, base * 2,
                           base * 4, 3, 10, o) == L.LSCAN_ERR_UNSUPPORTED
    o = L.make_options(carry=5)
    assert L.lscan_scan(L.LSCAN_ADD, L.LSCAN_F32, 1, base, base * 2, 10, o) == \
        L.LSCAN_ERR_INVALID
    # carry-in: aligned to the output element, single-array calls only
    o = L.make_options(carry_in=base + 2)
    assert L.lscan_scan(L.LSCAN_ADD, L.LSCAN_I32, 1, base, base * 2, 10, o) == \
        L.LSCAN_ERR_INVALID
    o = L.make_options(carry_in=base * 8)
    assert L.lscan_batched(L.LSCAN_ADD, L.LSCAN_I32, 1, base, base * 2,
                           base * 4, 3, 10, o) == L.LSCAN_ERR_INVALID
    # stream compaction: bad counts, missing or misaligned count pointer,
    # unknown dtype (all refused before any device work)
    sel = L.lscan_select_flagged
    assert sel(L.LSCAN_I32, base, base * 2, base * 4, -1, base * 8) == \
        L.LSCAN_ERR_INVALID
    assert sel(L.LSCAN_I32, base, base * 2, base * 4, 10, None) == \
        L.LSCAN_ERR_INVALID
    assert sel(L.LSCAN_I32, base, base * 2, base * 4, 10, base * 8 + 4) == \
        L.LSCAN_ERR_INVALID
    assert sel(9, base, base * 2, base * 4, 10, base * 8) == L.LSCAN_ERR_INVALID
    assert sel(L.LSCAN_I32, base, base * 2, base, 10, base * 8) == \
        L.LSCAN_ERR_INVALID                        # y overlaps x
    # batched: negative counts, missing offsets
    assert L.lscan_batched(L.LSCAN_ADD, L.LSCAN_I32, 1, base, base * 2, None,
                           3, 10) == L.LSCAN_ERR_INVALID
    assert L.lscan_batched(L.LSCAN_ADD, L.LSCAN_I32, 1, base, base * 2, base * 4,
                           -1, 10) == L.LSCAN_ERR_INVALID
    assert L.lscan_set_wait_limit_ns(0) == L.LSCAN_ERR_INVALID
    assert L.strerror(L.LSCAN_ERR_TIMEOUT) == "device wait ran out of time"


def test_host_scan_argument_checks(lib):
    """lscan_scan_host refuses bad arguments before any CUDA call (the
    pointers here are never dereferenced)."""
    L = lib
    f = L.lscan_scan_host
    base = 1 << 20
    add, i32, bf16 = L.LSCAN_ADD, L.LSCAN_I32, L.LSCAN_BF16
    assert f(add, i32, 1, base, base * 2, -1) == L.LSCAN_ERR_INVALID
    assert f(add, i32, 1, base, base * 2, 10, None, -5) == L.LSCAN_ERR_INVALID
    assert f(add, i32, 1, None, base * 2, 10) == L.LSCAN_ERR_INVALID
    assert f(add, i32, 1, base, None, 10) == L.LSCAN_ERR_INVALID
    assert f(add, i32, 1, base + 2, base * 2, 10) == L.LSCAN_ERR_INVALID
    assert f(add, i32, 1, base, base + 4, 10) == L.LSCAN_ERR_INVALID
    # bf16 add writes fp32: the same start is an overlap, not in place
    assert f(add, bf16, 1, base, base, 10) == L.LSCAN_ERR_INVALID
    assert f(9, i32, 1, base, base * 2, 10) == L.LSCAN_ERR_INVALID
    assert f(add, 7, 1, base, base * 2, 10) == L.LSCAN_ERR_INVALID
    o = L.make_options(out_dtype=L.LSCAN_BF16)
    assert f(add, i32, 1, base, base * 2, 10, o) == L.LSCAN_ERR_UNSUPPORTED
    o = L.make_options(config=L.lscan_num_configs() + 1)
    assert f(add, i32, 1, base, base * 2, 10, o) == L.LSCAN_ERR_INVALID
    o = L.make_options(carry_in=base + 2)
    assert f(add, i32, 1, base, base * 2, 10, o) == L.LSCAN_ERR_INVALID
    # nothing to do
    assert f(add, i32, 1, None, None, 0) == L.LSCAN_OK


def test_options_struct_layout(lib):
    """lscan_options: six int32 settings (the sixth the carry-in's type),
    then the carry-in pointer at byte 24 (32 bytes in all)."""
    import ctypes
    from paper_1604_04815_gb300 import _lib
    assert ctypes.sizeof(_lib.lscan_options) == 32
    assert _lib.lscan_options.carry_in_type.offset == 20
    assert _lib.lscan_options.carry_in.offset == 24


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1604_04815_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no fallback"):
        _lib.load()


def test_server_entry_points_reject_null_handles(lib):
    import ctypes
    L = lib.load()
    tk = ctypes.c_uint64()
    assert L.lscan_server_submit(None, 0, 0, 1, 16, None, 4,
                                 ctypes.byref(tk)) == lib.LSCAN_ERR_INVALID
    assert L.lscan_server_wait(None, 1, None) == lib.LSCAN_ERR_INVALID
    assert L.lscan_server_release(None, 1) == lib.LSCAN_ERR_INVALID
    assert L.lscan_server_alloc(None, 16, None) == lib.LSCAN_ERR_INVALID
    assert L.lscan_server_hold(None, 1) == lib.LSCAN_ERR_INVALID
    assert not L.lscan_server_create(1 << 20, 0)   # bad stream count
    L.lscan_server_destroy(None)                   # no-op


def test_noalloc_size_limits(lib):
    """lscan_scan_noalloc's fixed array holds 262144 status words; launches
    use tile configuration 2 (2 words per tile for every kind), or the
    plain-load configuration (tiles half as long) for unaligned pointers.
    One element past each limit is refused on the host; no GPU is touched
    (without one, an accepted size would fail with a CUDA error instead)."""
    L = lib
    f = L.lscan_scan_noalloc
    base = 1 << 44   # never dereferenced
    cases = [(L.LSCAN_ADD, L.LSCAN_I32, 0, 1 << 29),   # 4096-element tiles
             (L.LSCAN_ADD, L.LSCAN_F32, 0, 1 << 29),
             (L.LSCAN_MAX, L.LSCAN_BF16, 0, 1 << 30),  # 8192
             (L.LSCAN_ADD, L.LSCAN_I64, 0, 1 << 28),   # 2048
             (L.LSCAN_MAX, L.LSCAN_F64, 0, 1 << 28),
             (L.LSCAN_ADD, L.LSCAN_I32, 4, 1 << 28)]   # unaligned x: 2048
    for op, dt, off, limit in cases:
        assert f(op, dt, 1, base + off, base * 2, limit + 1) == \
            L.LSCAN_ERR_INVALID, (op, dt, off)
        # at the limit the host checks pass; with no GPU the call then fails
        # on its first CUDA call
        assert f(op, dt, 1, base + off, base * 2, limit) == L.LSCAN_ERR_CUDA


def test_tune_table_json_roundtrip(lib, tmp_path):
    """The tuning table loads/saves without a GPU; malformed files are
    refused and leave the table unchanged."""
    import json
    p = tmp_path / "t.json"
    # [kind, mode, log2 size class, configuration(, carry)]: four-field
    # entries mean carry 0 (auto)
    p.write_text('{"lscan_tune": 1, "entries": [[0, 0, 28, 3], [4, 1, 20, 1],'
                 ' [1, 0, 12, 2, 2]]}')
    assert lib.lscan_tune_load(p) == lib.LSCAN_OK
    out = tmp_path / "o.json"
    assert lib.lscan_tune_save(out) == lib.LSCAN_OK
    d = json.loads(out.read_text())
    assert d["lscan_tune"] == 1
    assert sorted(map(tuple, d["entries"])) == [(0, 0, 28, 3, 0),
                                                (1, 0, 12, 2, 2),
                                                (4, 1, 20, 1, 0)]
    bad = tmp_path / "bad.json"
    for entries in ("[[0, 0, 28, 99]]",        # no such configuration
                    "[[0, 1, 28, 9]]",         # not built for batched scans
                    "[[0, 0, 28, 2, 7]]",      # no such carry protocol
                    "[[99, 0, 28, 2]]"):       # no such kind
        bad.write_text('{"lscan_tune": 1, "entries": %s}' % entries)
        assert lib.lscan_tune_load(bad) == lib.LSCAN_ERR_INVALID, entries
    assert lib.lscan_tune_load(tmp_path / "missing.json") == lib.LSCAN_ERR_INVALID
    assert lib.lscan_tune_reset() == lib.LSCAN_OK
    assert lib.lscan_tune_save(out) == lib.LSCAN_OK
    assert json.loads(out.read_text())["entries"] == []
    # defaults are per kind, mode and size (kind 0, int32 add, defaults to
    # configuration 8): only entries that differ from them are saved
    p.write_text('{"lscan_tune": 1, "entries": [[0, 0, 28, 8], [0, 0, 27, 2]]}')
    assert lib.lscan_tune_load(p) == lib.LSCAN_OK
    assert lib.lscan_tune_save(out) == lib.LSCAN_OK
    assert json.loads(out.read_text())["entries"] == [[0, 0, 27, 2, 0]]
    assert lib.lscan_tune_reset() == lib.LSCAN_OK
    assert lib.lscan_autotune(0, 0, 1, 16, 32, 0)[0] == lib.LSCAN_ERR_INVALID


def test_radix_offsets_argument_checks(lib):
    """lscan_radix_offsets refuses bad arguments before any CUDA call."""
    L = lib
    f = L.lscan_radix_offsets
    base = 1 << 20
    out = base * 64
    assert f(base, 2, 10, 8, out) == L.LSCAN_ERR_INVALID     # key size
    assert f(base, 4, 10, 0, out) == L.LSCAN_ERR_INVALID     # digit bits
    assert f(base, 4, 10, 9, out) == L.LSCAN_ERR_INVALID
    assert f(base, 4, -1, 8, out) == L.LSCAN_ERR_INVALID
    assert f(base, 4, 1 << 32, 8, out) == L.LSCAN_ERR_INVALID
    assert f(base, 4, 10, 8, None) == L.LSCAN_ERR_INVALID
    assert f(base, 4, 10, 8, out + 4) == L.LSCAN_ERR_INVALID  # misaligned
    assert f(None, 4, 10, 8, out) == L.LSCAN_ERR_INVALID
    assert f(base + 2, 4, 10, 8, out) == L.LSCAN_ERR_INVALID
    assert f(base + 4, 8, 10, 8, out) == L.LSCAN_ERR_INVALID
    assert f(base, 4, 1000, 8, base + 64) == L.LSCAN_ERR_INVALID  # overlap
