"""Precision of the float-add carry chain, N = 2^26, cancellation-heavy
inputs x = s * exp(2 Z) (Z ~ N(0,1), s = +-1), fp32 and bf16.

For every result the error against the FP64 oracle is reported as
max_j |y_j - ref_j| / S_j (S_j = sum_{i<=j} |x_i|).  Gates: the FP64-carry
path <= 1e-5 and the compensated path <= 2.5e-7; the plain fp32 carry is the
control (its worst case grows with the number of carry hops) and is held to
1e-5 only because it meets it on this input.  Throughput of each path is
printed beside its error."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import BOUND, run_c_abi, to_device, to_host
from paper_1604_04815_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu

N = 1 << 26


@pytest.fixture(scope="module")
def data():
    from paper_1604_04815_gb300 import build
    build.build()
    _lib.load()
    x32, xb = workloads.precision(N)
    refs = {}
    for dt, x in (("f32", x32), ("bf16", xb)):
        refs[dt] = (oracle.scan("add", dt, x, True),
                    oracle.abs_prefix(dt, x, True))
    return {"f32": x32, "bf16": xb}, refs


def _time_path(xd, prec, reps=5):
    y = None
    for _ in range(2):
        y = run_c_abi("add", "f32" if xd.dtype == torch.float32 else "bf16",
                      xd, True, prec=prec, y_dev=y, check_status=False)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(
        enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        run_c_abi("add", "f32" if xd.dtype == torch.float32 else "bf16", xd,
                  True, prec=prec, y_dev=y, check_status=False)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("prec", ["plain", "f64", "comp"])
def test_precision_paths(data, dtype, prec):
    xs, refs = data
    x = xs[dtype]
    ref, s = refs[dtype]
    xd = to_device(x, dtype)
    y = run_c_abi("add", dtype, xd, True, prec=prec)
    got = to_host(y).astype(np.float64)
    err = np.abs(got - ref)
    pos = s > 0
    ratio = float(np.max(err[pos] / s[pos]))
    t = _time_path(xd, prec)
    gbs = N * (x.itemsize + 4) / t / 1e9
    print(f"\nprecision {dtype:4s} {prec:5s}: max|err|/S = {ratio:.3e}  "
          f"max|err| = {float(err.max()):.3e}  {gbs:.0f} GB/s")
    assert ratio <= BOUND[prec], (dtype, prec, ratio)
