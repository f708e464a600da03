"""ctypes binding of liblscan.so (argument marshalling only).

Every function of include/lscan.h is exposed under the same name.  The library
is built in-tree by ``paper_1604_04815_gb300.build``; if it is missing this
module raises -- there is no CPU or eager fallback.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblscan.so")

LSCAN_ADD, LSCAN_MAX = 0, 1
LSCAN_I32, LSCAN_F32, LSCAN_BF16, LSCAN_I64, LSCAN_F64 = 0, 1, 2, 3, 4
LSCAN_OK = 0
LSCAN_ERR_INVALID = 1
LSCAN_ERR_UNSUPPORTED = 2
LSCAN_ERR_CUDA = 3
LSCAN_ERR_TIMEOUT = 4
LSCAN_ERR_NOMEM = 5
LSCAN_ERR_BUSY = 6
LSCAN_ERR_DEVICE = 7
LSCAN_PREC_DEFAULT, LSCAN_PREC_F32_CARRY, LSCAN_PREC_F64_CARRY, \
    LSCAN_PREC_COMPENSATED, LSCAN_PREC_DF_CARRY = 0, 1, 2, 3, 4
LSCAN_CARRY_AUTO, LSCAN_CARRY_LOOKBACK, LSCAN_CARRY_CHAINED = 0, 1, 2

# every symbol include/lscan.h declares (checked by the ABI test)
EXPORTED = [
    "lscan_inclusive", "lscan_exclusive", "lscan_scan", "lscan_batched",
    "lscan_scan_host",
    "lscan_graph_create_scan", "lscan_graph_create_batched",
    "lscan_graph_launch", "lscan_graph_status", "lscan_graph_destroy",
    "lscan_stream_status", "lscan_reserve", "lscan_shutdown",
    "lscan_strerror", "lscan_version", "lscan_launch_count",
    "lscan_set_wait_limit_ns", "lscan_debug_skip_publish",
    "lscan_config_info", "lscan_num_configs", "lscan_scan_noalloc",
    "lscan_noalloc_status",
    "lscan_server_create", "lscan_server_destroy", "lscan_server_alloc",
    "lscan_server_free", "lscan_server_submit", "lscan_server_wait",
    "lscan_server_poll", "lscan_server_release", "lscan_server_replay",
    "lscan_server_hold", "lscan_server_set_lanes",
    "lscan_autotune", "lscan_tune_save", "lscan_tune_load",
    "lscan_tune_reset", "lscan_select_flagged", "lscan_radix_offsets",
    "lscan_carry_bytes", "lscan_reduce", "lscan_carry_combine",
]


class lscan_options(ctypes.Structure):
    _fields_ = [("out_dtype", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("carry", ctypes.c_int32), ("config", ctypes.c_int32),
                ("max_ctas", ctypes.c_int32), ("carry_in_type", ctypes.c_int32),
                ("carry_in", ctypes.c_void_p)]


class lscan_req_stats(ctypes.Structure):
    _fields_ = [("submit_us", ctypes.c_double), ("admit_us", ctypes.c_double),
                ("launch_us", ctypes.c_double), ("done_us", ctypes.c_double),
                ("y", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("status", ctypes.c_int32), ("batch_requests", ctypes.c_int32)]


class lscan_trace_req(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("inclusive", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("x", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("arrival_us", ctypes.c_double)]


LSCAN_TUNE_MAX_CONFIGS = 32


class lscan_tune_result(ctypes.Structure):
    _fields_ = [("config", ctypes.c_int32), ("carry", ctypes.c_int32),
                ("ms", ctypes.c_float), ("default_config", ctypes.c_int32),
                ("default_ms", ctypes.c_float), ("n_timed", ctypes.c_int32),
                ("chained_ms", ctypes.c_float),
                ("ms_by_config", ctypes.c_float * LSCAN_TUNE_MAX_CONFIGS)]


class LscanError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


_lib = None


def load():
    """Load liblscan.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"liblscan.so not found at {LIB_PATH}; build it with "
            "`python -m paper_1604_04815_gb300.build` (needs nvcc); "
            "there is no fallback path")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    optp = ctypes.POINTER(lscan_options)
    sig = {
        "lscan_inclusive": [i32, i32, vp, vp, i64, vp],
        "lscan_exclusive": [i32, i32, vp, vp, i64, vp],
        "lscan_scan": [i32, i32, i32, vp, vp, i64, optp, vp],
        "lscan_scan_host": [i32, i32, i32, vp, vp, i64, optp, i64, vp],
        "lscan_batched": [i32, i32, i32, vp, vp, vp, i64, i64, optp, vp],
        "lscan_graph_create_scan": [i32, i32, i32, vp, vp, i64, optp,
                                    ctypes.POINTER(vp)],
        "lscan_graph_create_batched": [i32, i32, i32, vp, vp, vp, i64, i64,
                                       optp, ctypes.POINTER(vp)],
        "lscan_scan_noalloc": [i32, i32, i32, vp, vp, i64, vp],
        "lscan_select_flagged": [i32, vp, vp, vp, i64, vp, vp],
        "lscan_radix_offsets": [vp, ctypes.c_int32, i64, ctypes.c_int32, vp,
                                vp],
        "lscan_graph_launch": [vp, vp],
        "lscan_graph_status": [vp],
        "lscan_stream_status": [vp],
        "lscan_reserve": [vp, i64],
        "lscan_set_wait_limit_ns": [ctypes.c_uint64],
        "lscan_debug_skip_publish": [i64],
        "lscan_config_info": [ctypes.c_int32, i32] +
                             [ctypes.POINTER(ctypes.c_int32)] * 4,
        "lscan_autotune": [i32, i32, i32, vp, vp, i64, vp, i64, optp, i32, vp,
                           ctypes.POINTER(lscan_tune_result)],
        "lscan_noalloc_status": [vp],
        "lscan_reduce": [i32, i32, vp, i64, optp, vp, vp],
        "lscan_carry_combine": [i32, i32, optp, vp, ctypes.c_int32, vp],
        "lscan_tune_save": [ctypes.c_char_p],
        "lscan_tune_load": [ctypes.c_char_p],
        "lscan_tune_reset": [],
        "lscan_server_alloc": [vp, ctypes.c_size_t, ctypes.POINTER(vp)],
        "lscan_server_free": [vp, vp],
        "lscan_server_submit": [vp, i32, i32, i32, vp, vp, i64,
                                ctypes.POINTER(ctypes.c_uint64)],
        "lscan_server_wait": [vp, ctypes.c_uint64,
                              ctypes.POINTER(lscan_req_stats)],
        "lscan_server_poll": [vp, ctypes.c_uint64,
                              ctypes.POINTER(lscan_req_stats)],
        "lscan_server_release": [vp, ctypes.c_uint64],
        "lscan_server_hold": [vp, ctypes.c_int],
        "lscan_server_set_lanes": [vp, i64, i64, ctypes.c_int32],
        "lscan_server_replay": [vp, ctypes.POINTER(lscan_trace_req), i64,
                                ctypes.POINTER(lscan_req_stats),
                                ctypes.POINTER(ctypes.c_double)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.lscan_server_create.argtypes = [ctypes.c_size_t, i32]
    lib.lscan_server_create.restype = vp
    lib.lscan_server_destroy.argtypes = [vp]
    lib.lscan_server_destroy.restype = None
    lib.lscan_graph_destroy.argtypes = [vp]
    lib.lscan_graph_destroy.restype = None
    lib.lscan_shutdown.argtypes = []
    lib.lscan_shutdown.restype = None
    lib.lscan_strerror.argtypes = [ctypes.c_int]
    lib.lscan_strerror.restype = ctypes.c_char_p
    lib.lscan_version.argtypes = []
    lib.lscan_version.restype = ctypes.c_char_p
    lib.lscan_launch_count.argtypes = []
    lib.lscan_launch_count.restype = ctypes.c_uint64
    lib.lscan_num_configs.argtypes = []
    lib.lscan_num_configs.restype = ctypes.c_int32
    lib.lscan_carry_bytes.argtypes = [i32, i32, optp]
    lib.lscan_carry_bytes.restype = ctypes.c_int32
    _lib = lib
    return lib


def strerror(status):
    return load().lscan_strerror(int(status)).decode()


def check(status, where):
    if status != LSCAN_OK:
        raise LscanError(status, where)


def make_options(out_dtype=0, precision=0, carry=0, config=0, max_ctas=0,
                 carry_in=None, carry_in_type=0):
    o = lscan_options()
    o.out_dtype = out_dtype
    o.precision = precision
    o.carry = carry
    o.config = config
    o.max_ctas = max_ctas
    o.carry_in = carry_in
    o.carry_in_type = carry_in_type
    return o


# Thin same-name wrappers: plain integers/pointers in, status out.
def lscan_inclusive(op, dtype, x, y, n, stream=None):
    return load().lscan_inclusive(op, dtype, x, y, n, stream)


def lscan_exclusive(op, dtype, x, y, n, stream=None):
    return load().lscan_exclusive(op, dtype, x, y, n, stream)


def lscan_scan(op, dtype, inclusive, x, y, n, opts=None, stream=None):
    return load().lscan_scan(op, dtype, inclusive, x, y, n,
                             ctypes.byref(opts) if opts is not None else None,
                             stream)


def lscan_scan_host(op, dtype, inclusive, hx, hy, n, opts=None, chunk=0,
                    stream=None):
    return load().lscan_scan_host(op, dtype, inclusive, hx, hy, n,
                                  ctypes.byref(opts) if opts is not None
                                  else None, chunk, stream)


def lscan_scan_noalloc(op, dtype, inclusive, x, y, n, stream=None):
    return load().lscan_scan_noalloc(op, dtype, inclusive, x, y, n, stream)


def lscan_select_flagged(dtype, x, flags, y, n, d_count, stream=None):
    return load().lscan_select_flagged(dtype, x, flags, y, n, d_count, stream)


def lscan_radix_offsets(keys, key_bytes, n, digit_bits, d_offsets,
                        stream=None):
    return load().lscan_radix_offsets(keys, key_bytes, n, digit_bits,
                                      d_offsets, stream)


def lscan_batched(op, dtype, inclusive, x, y, d_offsets, n_seg, n_total,
                  opts=None, stream=None):
    return load().lscan_batched(op, dtype, inclusive, x, y, d_offsets, n_seg,
                                n_total,
                                ctypes.byref(opts) if opts is not None
                                else None, stream)


def lscan_stream_status(stream=None):
    return load().lscan_stream_status(stream)


def lscan_reserve(stream, max_elems):
    return load().lscan_reserve(stream, max_elems)


def lscan_launch_count():
    return int(load().lscan_launch_count())


def lscan_set_wait_limit_ns(ns):
    return load().lscan_set_wait_limit_ns(ns)


def lscan_debug_skip_publish(tile):
    return load().lscan_debug_skip_publish(tile)


def lscan_shutdown():
    load().lscan_shutdown()


def lscan_config_info(config, dtype):
    vals = [ctypes.c_int32() for _ in range(4)]
    st = load().lscan_config_info(config, dtype, *[ctypes.byref(v)
                                                   for v in vals])
    check(st, "lscan_config_info")
    return dict(items=vals[0].value, threads=vals[1].value,
                stages=vals[2].value, tile=vals[3].value)


def lscan_num_configs():
    return int(load().lscan_num_configs())


def lscan_autotune(op, dtype, inclusive, x, y, n, d_offsets=None, n_seg=0,
                   opts=None, reps=5, stream=None):
    """Returns (status, result dict): the fastest configuration and carry,
    its median ms, the default configuration's median ms and every timed
    configuration's median ms (keyed by configuration number)."""
    r = lscan_tune_result()
    st = load().lscan_autotune(op, dtype, inclusive, x, y, n, d_offsets, n_seg,
                               ctypes.byref(opts) if opts is not None
                               else None, reps, stream, ctypes.byref(r))
    res = dict(config=r.config, carry=r.carry, ms=r.ms,
               default_config=r.default_config, default_ms=r.default_ms,
               n_timed=r.n_timed, chained_ms=r.chained_ms,
               ms_by_config={i + 1: r.ms_by_config[i]
                             for i in range(LSCAN_TUNE_MAX_CONFIGS)
                             if r.ms_by_config[i] > 0})
    return st, res


def lscan_noalloc_status(stream=None):
    return load().lscan_noalloc_status(stream)


def _optref(opts):
    return ctypes.byref(opts) if opts is not None else None


def lscan_carry_bytes(op, dtype, opts=None):
    return int(load().lscan_carry_bytes(op, dtype, _optref(opts)))


def lscan_reduce(op, dtype, x, n, opts=None, d_total=None, stream=None):
    return load().lscan_reduce(op, dtype, x, n, _optref(opts), d_total, stream)


def lscan_carry_combine(op, dtype, totals, count, opts=None):
    """Host fold of `count` carry-type totals (bytes, concatenated); returns
    (status, bytes of the result)."""
    nb = lscan_carry_bytes(op, dtype, opts)
    out = ctypes.create_string_buffer(max(nb, 1))
    buf = ctypes.create_string_buffer(bytes(totals), max(len(totals), 1))
    st = load().lscan_carry_combine(op, dtype, _optref(opts), buf, count, out)
    return st, out.raw[:nb]


def lscan_tune_save(path):
    return load().lscan_tune_save(str(path).encode())


def lscan_tune_load(path):
    return load().lscan_tune_load(str(path).encode())


def lscan_tune_reset():
    return load().lscan_tune_reset()


def lscan_version():
    return load().lscan_version().decode()


class _CudaArray:
    """Zero-copy view of device memory for torch.as_tensor."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {
            "shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
            "version": 3, "strides": None}


def device_view(ptr, n, torch_dtype):
    """torch tensor aliasing n elements at a device pointer (no copy)."""
    import torch
    typestr = {torch.int32: "<i4", torch.float32: "<f4",
               torch.bfloat16: "<i2"}[torch_dtype]
    t = torch.as_tensor(_CudaArray(ptr, n, typestr), device="cuda")
    return t.view(torch.bfloat16) if torch_dtype == torch.bfloat16 else t
