"""GB300-native single-pass scan (LightScan, arXiv 1604.04815), torch front.

Everything below marshals torch tensors into the C ABI of liblscan.so
(include/lscan.h); every step of the scan runs in the library's CUDA kernels.
torch is used for device memory and streams only.

    import paper_1604_04815_gb300 as lscan
    y = lscan.inclusive(x)                 # add, x: int32/float32/bfloat16
    y = lscan.exclusive(x, op="max")
    y = lscan.batched(x, offsets)          # offsets: int64 cuda tensor [S+1]
    y = lscan.scan_host(x_cpu)             # x_cpu in (pinned) host memory
    y = lscan.shard.sharded_scan(x_shard)  # one rank's shard of a global scan
"""
import torch

from . import _lib
from ._lib import LscanError, load  # noqa: F401

_DT = {torch.int32: _lib.LSCAN_I32, torch.float32: _lib.LSCAN_F32,
       torch.bfloat16: _lib.LSCAN_BF16, torch.int64: _lib.LSCAN_I64,
       torch.float64: _lib.LSCAN_F64}
_TORCH_DT = {v: k for k, v in _DT.items()}
_OPS = {"add": _lib.LSCAN_ADD, "max": _lib.LSCAN_MAX}
_PREC = {None: 0, "default": 0, "f32": 1, "plain": 1, "f64": 2,
         "compensated": 3, "comp": 3, "df": 4, "double-float": 4}
_CARRY = {None: 0, "auto": 0, "lookback": 1, "chained": 2}


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def out_dtype_for(op, dtype, out_dtype=None):
    """Output torch dtype of a scan (bf16 add writes fp32 by default)."""
    if out_dtype is not None:
        return out_dtype
    if op == "add" and dtype == torch.bfloat16:
        return torch.float32
    return dtype


def _options(op, x_dtype, out_dtype, precision, carry, config, max_ctas,
             carry_in=None):
    od = 0
    if out_dtype is not None and out_dtype != out_dtype_for(op, x_dtype):
        od = _DT[out_dtype]
    cin = None
    if carry_in is not None:
        if (not isinstance(carry_in, torch.Tensor) or not carry_in.is_cuda
                or carry_in.numel() < 1
                or carry_in.dtype != out_dtype_for(op, x_dtype, out_dtype)):
            raise TypeError("carry_in must be a CUDA tensor holding one "
                            "element of the output dtype")
        cin = carry_in.data_ptr()
    return _lib.make_options(out_dtype=od, precision=_PREC[precision],
                             carry=_CARRY[carry], config=int(config),
                             max_ctas=int(max_ctas), carry_in=cin)


def _check_input(x):
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError("x must be a CUDA tensor")
    if x.dtype not in _DT:
        raise TypeError(f"unsupported dtype {x.dtype}")
    if x.dim() != 1 or not x.is_contiguous():
        raise ValueError("x must be a contiguous 1-D tensor")


def scan(x, op="add", inclusive=True, out=None, *, precision=None,
         carry=None, config=0, max_ctas=0, out_dtype=None, carry_in=None,
         stream=None):
    """Inclusive or exclusive scan of a 1-D CUDA tensor (one kernel launch).
    carry_in: optional one-element CUDA tensor of the output dtype that is
    combined in front of x[0] (the offset of a shard of a longer scan)."""
    _check_input(x)
    odt = out_dtype_for(op, x.dtype, out_dtype)
    if out is None:
        out = torch.empty(x.shape[0], dtype=odt, device=x.device)
    elif out.dtype != odt or out.shape != x.shape or not out.is_contiguous():
        raise ValueError("out has the wrong dtype, shape or layout")
    opts = _options(op, x.dtype, out_dtype, precision, carry, config, max_ctas,
                    carry_in)
    st = _lib.lscan_scan(_OPS[op], _DT[x.dtype], int(bool(inclusive)),
                         x.data_ptr(), out.data_ptr(), x.shape[0], opts,
                         _stream_ptr(stream))
    _lib.check(st, "lscan_scan")
    return out


def scan_host(x, op="add", inclusive=True, out=None, *, chunk=0,
              precision=None, carry=None, config=0, max_ctas=0, out_dtype=None,
              stream=None, synchronize=True):
    """Scan of a 1-D CPU tensor through the library's host-buffer entry point
    (chunked copy-in, scan and copy-out, overlapped on the device).  Pinned
    tensors (Tensor.pin_memory()) get full copy bandwidth.  out: optional
    CPU tensor of the output dtype (may be x itself when the element sizes
    match).  With synchronize=False the call returns once the work is queued
    on stream; x and out must then stay alive until the stream reaches it."""
    if not isinstance(x, torch.Tensor) or x.is_cuda:
        raise TypeError("x must be a CPU tensor")
    if x.dtype not in _DT:
        raise TypeError(f"unsupported dtype {x.dtype}")
    if x.dim() != 1 or not x.is_contiguous():
        raise ValueError("x must be a contiguous 1-D tensor")
    odt = out_dtype_for(op, x.dtype, out_dtype)
    if out is None:
        out = torch.empty(x.shape[0], dtype=odt, pin_memory=x.is_pinned())
    elif (out.is_cuda or out.dtype != odt or out.shape != x.shape
          or not out.is_contiguous()):
        raise ValueError("out has the wrong device, dtype, shape or layout")
    opts = _options(op, x.dtype, out_dtype, precision, carry, config, max_ctas)
    if stream is None:
        stream = torch.cuda.current_stream()
    st = _lib.lscan_scan_host(_OPS[op], _DT[x.dtype], int(bool(inclusive)),
                              x.data_ptr(), out.data_ptr(), x.shape[0], opts,
                              int(chunk), stream.cuda_stream)
    _lib.check(st, "lscan_scan_host")
    if synchronize:
        stream.synchronize()
    return out


def inclusive(x, op="add", out=None, **kw):
    return scan(x, op, True, out, **kw)


def exclusive(x, op="add", out=None, **kw):
    return scan(x, op, False, out, **kw)


def batched(x, offsets, op="add", inclusive=True, out=None, *, n_total=None,
            precision=None, carry=None, config=0, max_ctas=0, out_dtype=None,
            stream=None):
    """Scan every segment [offsets[s], offsets[s+1]) of x independently."""
    _check_input(x)
    if offsets.dtype != torch.int64 or not offsets.is_cuda:
        raise TypeError("offsets must be an int64 CUDA tensor")
    n_total = x.shape[0] if n_total is None else int(n_total)
    odt = out_dtype_for(op, x.dtype, out_dtype)
    if out is None:
        out = torch.empty(x.shape[0], dtype=odt, device=x.device)
    opts = _options(op, x.dtype, out_dtype, precision, carry, config, max_ctas)
    st = _lib.lscan_batched(_OPS[op], _DT[x.dtype], int(bool(inclusive)),
                            x.data_ptr(), out.data_ptr(), offsets.data_ptr(),
                            offsets.shape[0] - 1, n_total, opts,
                            _stream_ptr(stream))
    _lib.check(st, "lscan_batched")
    return out


def radix_offsets(keys, digit_bits=8, out=None, *, stream=None):
    """Radix-sort digit offsets of a 1-D CUDA tensor of keys (int32/uint32
    or int64/uint64, read as unsigned), in one pass: out[p, v] = number of
    keys whose digit p (digit_bits wide, lowest first) is below v, i.e. where
    bucket v starts in a counting-sort pass on digit p.  Returns an int64
    CUDA tensor of shape (ceil(key_bits / digit_bits), 2^digit_bits)."""
    if (not isinstance(keys, torch.Tensor) or not keys.is_cuda
            or keys.dim() != 1 or not keys.is_contiguous()):
        raise TypeError("keys must be a contiguous 1-D CUDA tensor")
    kb = keys.element_size()
    if kb not in (4, 8) or keys.is_floating_point():
        raise TypeError("keys must be 32- or 64-bit integers")
    if not 1 <= int(digit_bits) <= 8:
        raise ValueError("digit_bits must be 1..8")
    shape = (-(-8 * kb // int(digit_bits)), 1 << int(digit_bits))
    if out is None:
        out = torch.empty(shape, dtype=torch.int64, device=keys.device)
    elif (out.dtype != torch.int64 or tuple(out.shape) != shape
          or not out.is_contiguous() or not out.is_cuda):
        raise ValueError("out has the wrong dtype, shape or layout")
    st = _lib.lscan_radix_offsets(keys.data_ptr(), kb, keys.shape[0],
                                  int(digit_bits), out.data_ptr(),
                                  _stream_ptr(stream))
    _lib.check(st, "lscan_radix_offsets")
    return out


def select_flagged(x, flags, out=None, *, stream=None):
    """Stream compaction: the elements of x whose flag (uint8/bool) is
    nonzero, in order, in one pass.  Returns (out, count): out has len(x)
    elements, the first count[0] of them selected; count is a one-element
    int64 CUDA tensor (read it after the stream has reached it)."""
    _check_input(x)
    if (not isinstance(flags, torch.Tensor) or not flags.is_cuda
            or flags.dtype not in (torch.uint8, torch.bool)
            or flags.shape != x.shape or not flags.is_contiguous()):
        raise TypeError("flags must be a contiguous uint8/bool CUDA tensor "
                        "shaped like x")
    if out is None:
        out = torch.empty_like(x)
    elif out.dtype != x.dtype or out.shape != x.shape or not out.is_contiguous():
        raise ValueError("out has the wrong dtype, shape or layout")
    count = torch.empty(1, dtype=torch.int64, device=x.device)
    st = _lib.lscan_select_flagged(_DT[x.dtype], x.data_ptr(), flags.data_ptr(),
                                   out.data_ptr(), x.shape[0],
                                   count.data_ptr(), _stream_ptr(stream))
    _lib.check(st, "lscan_select_flagged")
    return out, count


def stream_status(stream=None):
    """Synchronise the stream and raise if the device latched an error."""
    _lib.check(_lib.lscan_stream_status(_stream_ptr(stream)),
               "lscan_stream_status")


class Graph:
    """A scan captured into a CUDA graph once and replayed (one kernel)."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep  # tensors the graph's baked pointers refer to

    @classmethod
    def scan(cls, x, out, op="add", inclusive=True, **kw):
        import ctypes
        _check_input(x)
        cin = kw.get("carry_in")
        opts = _options(op, x.dtype, kw.get("out_dtype"), kw.get("precision"),
                        kw.get("carry"), kw.get("config", 0),
                        kw.get("max_ctas", 0), cin)
        h = ctypes.c_void_p()
        st = _lib.load().lscan_graph_create_scan(
            _OPS[op], _DT[x.dtype], int(bool(inclusive)), x.data_ptr(),
            out.data_ptr(), x.shape[0], ctypes.byref(opts), ctypes.byref(h))
        _lib.check(st, "lscan_graph_create_scan")
        return cls(h, (x, out, cin))

    @classmethod
    def batched(cls, x, offsets, out, op="add", inclusive=True, **kw):
        import ctypes
        _check_input(x)
        opts = _options(op, x.dtype, kw.get("out_dtype"), kw.get("precision"),
                        kw.get("carry"), kw.get("config", 0),
                        kw.get("max_ctas", 0))
        h = ctypes.c_void_p()
        st = _lib.load().lscan_graph_create_batched(
            _OPS[op], _DT[x.dtype], int(bool(inclusive)), x.data_ptr(),
            out.data_ptr(), offsets.data_ptr(), offsets.shape[0] - 1,
            x.shape[0], ctypes.byref(opts), ctypes.byref(h))
        _lib.check(st, "lscan_graph_create_batched")
        return cls(h, (x, offsets, out))

    def launch(self, stream=None):
        _lib.check(_lib.load().lscan_graph_launch(self._h, _stream_ptr(stream)),
                   "lscan_graph_launch")

    def status(self):
        _lib.check(_lib.load().lscan_graph_status(self._h), "lscan_graph_status")

    def close(self):
        if self._h is not None and self._h.value:
            _lib.load().lscan_graph_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching scan service (lscan_server_* of include/lscan.h).

    submit() returns a ticket at once; wait() blocks until the request's batch
    finished and returns its stats; output() views a server-allocated output;
    release() frees it.  Requests with out=None get their output from the
    server's HBM pool and wait in the admission queue until it fits.
    """

    def __init__(self, budget_bytes=16 << 30, n_streams=4):
        lib = _lib.load()
        self._h = lib.lscan_server_create(int(budget_bytes), int(n_streams))
        if not self._h:
            raise LscanError(_lib.LSCAN_ERR_NOMEM, "lscan_server_create")

    def submit(self, x, op="add", inclusive=True, out=None):
        import ctypes
        _check_input(x)
        tk = ctypes.c_uint64()
        st = _lib.load().lscan_server_submit(
            self._h, _OPS[op], _DT[x.dtype], int(bool(inclusive)),
            x.data_ptr(), out.data_ptr() if out is not None else None,
            x.shape[0], ctypes.byref(tk))
        _lib.check(st, "lscan_server_submit")
        return tk.value

    def wait(self, ticket):
        import ctypes
        s = _lib.lscan_req_stats()
        st = _lib.load().lscan_server_wait(self._h, ticket, ctypes.byref(s))
        _lib.check(st, "lscan_server_wait")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def output(self, stats, op, dtype):
        """View of a server-allocated output (valid until release)."""
        return _lib.device_view(stats["y"], stats["n"],
                                out_dtype_for(op, dtype))

    def set_lanes(self, small_max_elems=1 << 14, bulk_batch_tiles=32768,
                  reserve_sms=4):
        """Size-class lanes (the library's defaults): requests of at most
        small_max_elems elements go to the resident kernel on reserve_sms
        SMs; bulk batches hold at most bulk_batch_tiles tiles and run on the
        other SMs (lscan_server_set_lanes)."""
        _lib.check(_lib.load().lscan_server_set_lanes(
            self._h, int(small_max_elems), int(bulk_batch_tiles),
            int(reserve_sms)), "lscan_server_set_lanes")

    def hold(self, on=True):
        """Queue requests without launching (on) / launch what queued (off)."""
        _lib.check(_lib.load().lscan_server_hold(self._h, int(bool(on))),
                   "lscan_server_hold")

    def release(self, ticket):
        _lib.check(_lib.load().lscan_server_release(self._h, ticket),
                   "lscan_server_release")

    def replay(self, trace):
        """trace: list of (op, dtype(torch), inclusive, x_ptr, n, arrival_us).
        Returns (list of stats dicts, wall_us)."""
        import ctypes
        n = len(trace)
        arr = (_lib.lscan_trace_req * max(n, 1))()
        for i, (op, dt, incl, xp, nn, at) in enumerate(trace):
            arr[i].op = _OPS[op]
            arr[i].dtype = _DT[dt]
            arr[i].inclusive = int(bool(incl))
            arr[i].x = xp
            arr[i].n = nn
            arr[i].arrival_us = at
        out = (_lib.lscan_req_stats * max(n, 1))()
        wall = ctypes.c_double()
        st = _lib.load().lscan_server_replay(self._h, arr, n, out,
                                             ctypes.byref(wall))
        _lib.check(st, "lscan_server_replay")
        stats = [{k: getattr(out[i], k) for k, _ in out[i]._fields_}
                 for i in range(n)]
        return stats, wall.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().lscan_server_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


from . import shard  # noqa: E402,F401  (sharded scans over ranks)
