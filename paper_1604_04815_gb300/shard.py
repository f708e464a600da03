"""A scan of one array sharded over devices (one rank per GPU).

Reduce-then-scan over the C ABI (include/lscan.h, "sharded scans"):
  1. lscan_reduce: this rank's shard total in the kind's carry type;
  2. all-gather of the totals over the process group (NCCL between GPUs,
     gloo on CPU: the totals are 4 or 8 bytes each);
  3. lscan_carry_combine on the host folds the totals of the lower ranks
     into this rank's offset, which lscan_scan takes as its carry-in
     (carry_in_type 1).
This module only moves arguments and bytes; every step of the arithmetic
runs in liblscan.so.
"""
from . import _lib


def exchange_offset(total, op, dtype, opts=None, group=None):
    """total: this rank's shard total (bytes of the carry type).  All-gathers
    the totals and returns (offset bytes for this rank, list of all totals).
    The offset is the fold of the totals of ranks 0 .. rank-1 (the identity
    on rank 0)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    nb = _lib.lscan_carry_bytes(op, dtype, opts)
    if len(total) != nb:
        raise ValueError(f"a total of this kind is {nb} bytes, got {len(total)}")
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.frombuffer(bytearray(total), dtype=torch.uint8).to(dev)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    totals = [bytes(p.cpu().numpy().tobytes()) for p in parts]
    st, off = _lib.lscan_carry_combine(op, dtype, b"".join(totals[:rank]),
                                       rank, opts)
    _lib.check(st, "lscan_carry_combine")
    return off, totals


def sharded_scan(x, op="add", inclusive=True, out=None, *, precision=0,
                 group=None, stream=None):
    """Scan this rank's shard x (a CUDA tensor) as part of the array formed by
    the shards of ranks 0 .. world-1 in order.  Returns y (this rank's part
    of the global scan)."""
    import torch

    from . import _DT, _OPS, _check_input, out_dtype_for
    _check_input(x)
    o = _OPS[op]
    d = _DT[x.dtype]
    opts = _lib.make_options(precision=precision)
    nb = _lib.lscan_carry_bytes(o, d, opts)
    s = stream or torch.cuda.current_stream()
    sp = s.cuda_stream
    total = torch.empty(nb, dtype=torch.uint8, device=x.device)
    _lib.check(_lib.lscan_reduce(o, d, x.data_ptr(), x.shape[0], opts,
                                 total.data_ptr(), sp), "lscan_reduce")
    s.synchronize()
    off, _ = exchange_offset(total.cpu().numpy().tobytes(), o, d, opts, group)
    cin = torch.frombuffer(bytearray(off), dtype=torch.uint8).to(x.device)
    if out is None:
        out = torch.empty(x.shape[0], dtype=out_dtype_for(op, x.dtype),
                          device=x.device)
    so = _lib.make_options(precision=precision, carry_in=cin.data_ptr(),
                           carry_in_type=1)
    _lib.check(_lib.lscan_scan(o, d, int(bool(inclusive)), x.data_ptr(),
                               out.data_ptr(), x.shape[0], so, sp),
               "lscan_scan")
    # the carry-in is read in stream order; keep it alive until then
    s.synchronize()
    return out

