"""etd_fft_forward_noalloc: the forward FFT for callers that may not allocate device memory.

Such callers -- a host application that owns all device memory through its own pool or a
fixed footprint, or code on a latency-critical path where cudaMalloc/cudaFree could
synchronise the device -- cannot create a plan, because etd_plan allocates its workspace.
This entry point keeps its scratch in a static device array of 8 MiB instead.  The GPU
test checks its output against etd_fft_forward (the plan's entry point) on two calls in a
row that share that array; this file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes as ct

import numpy as np
import pytest

from paper_2606_04347_gb300 import abi
from paper_2606_04347_gb300 import workloads as wl


def _call(lib, dim, n, prec, field_ptr, out_ptr, stream=None):
    arr = (ct.c_int * 3)(*n)
    return lib.etd_fft_forward_noalloc(dim, arr, prec, field_ptr, out_ptr, stream)


def test_oversize_grid_is_rejected_before_any_gpu_work():
    lib = abi.load_library()
    code = _call(lib, 3, (128, 128, 128), 1, 16, 16)       # 8.5 MB of scratch needed
    assert code == 1
    msg = lib.etd_last_error().decode()
    assert "bytes of scratch" in msg and str(8 << 20) in msg
    assert _call(lib, 3, (96, 64, 64), 0, 16, 16) == 1     # not a power of two
    assert _call(lib, 3, (64, 64, 64), 0, None, 16) == 1   # NULL field


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol,dim,n", [
    (0, 1e-13, 3, (64, 64, 64)),
    (1, 2e-6, 3, (64, 64, 64)),
    (1, 2e-6, 3, (128, 128, 64)),
    (0, 1e-13, 2, (128, 128, 1)),
    (1, 2e-6, 3, (32, 256, 16)),
])
def test_noalloc_fft_matches_plan_fft_on_two_calls(prec, tol, dim, n):
    torch = pytest.importorskip("torch")
    from paper_2606_04347_gb300 import Plan
    lib = abi.load_library()
    p = wl.workload("c3", n=8)[0].replace(dim=dim, n=n, model=0, precision=prec)
    rdt = torch.float64 if prec == 0 else torch.float32
    cdt = torch.complex128 if prec == 0 else torch.complex64
    fields = [torch.tensor(wl.random_fields(p.shape, s, -1.0, 1.0), dtype=rdt, device="cuda:0") for s in (5, 6)]
    spec_shape = p.shape[:-1] + (n[0] // 2 + 1,)
    plan = Plan(p)
    want = []
    for f in fields:
        o = torch.zeros(spec_shape, dtype=cdt, device="cuda:0")
        plan.fft_forward(f, o)
        want.append(o.cpu().numpy())
    plan.close()
    stream = torch.cuda.current_stream()
    got = [torch.full(spec_shape, float("nan"), dtype=cdt, device="cuda:0") for _ in fields]
    for f, o in zip(fields, got):                          # two calls in a row, shared scratch
        code = _call(lib, dim, n, prec, f.data_ptr(), o.data_ptr(), stream.cuda_stream)
        assert code == 0, lib.etd_last_error().decode()
    torch.cuda.synchronize()
    for g, w in zip(got, want):
        g = g.cpu().numpy()
        err = np.linalg.norm(g - w) / np.linalg.norm(w)
        assert err < tol, err
