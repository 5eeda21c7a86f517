"""Bounded device waits: a wait that runs out returns ETD_ETIMEOUT and leaves the context usable.

The plan reads two limits at creation: ETD_WAIT_BUDGET (clock cycles a grid barrier of the
band solve may spin) and ETD_WAIT_TRIES (mbarrier polls for a pass-A tensor copy).  Setting
them to -1 and 0 makes the first wait give up at once: the waiting blocks record the status
and return (a block whose tensor copy is still in flight waits for its own copy once more
before it leaves), the call reports ETD_ETIMEOUT, and a plan created afterwards with the
default limits computes the same operation correctly in the same process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import band as obm  # noqa: E402
from oracle import fft as offt  # noqa: E402
from oracle import model as omodel  # noqa: E402
from paper_2606_04347_gb300 import Plan  # noqa: E402
from paper_2606_04347_gb300 import workloads as wl  # noqa: E402
from paper_2606_04347_gb300.abi import EtdError  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _plan_with_env(monkeypatch, p, **env):
    for k, v in env.items():
        monkeypatch.setenv(k, str(v))
    plan = Plan(p)
    for k in env:
        monkeypatch.delenv(k)
    return plan


def test_grid_barrier_timeout_is_reported_and_recoverable(monkeypatch):
    p, phi, _, _ = wl.workload("c3", n=32)
    p = p.replace(cg_rtol=1e-13)
    g = omodel.g_loc(phi)
    band = obm.band_mask(phi, p.band_mask_hi)
    f = np.where(band, wl.random_fields(p.shape, 4, -1.0, 1.0), 0.0)
    phid = torch.tensor(phi, dtype=torch.float64, device=DEV)
    fd = torch.tensor(f, dtype=torch.float64, device=DEV)
    w = torch.zeros(p.shape, dtype=torch.float64, device=DEV)
    plan = _plan_with_env(monkeypatch, p, ETD_WAIT_BUDGET=-1)
    with pytest.raises(EtdError) as ei:
        plan.nonlocal_solve(phid, fd, w)
    assert ei.value.code == 6
    plan.close()
    torch.cuda.synchronize()
    plan = Plan(p)
    w.zero_()
    plan.nonlocal_solve(phid, fd, w)
    want, _, _ = obm.solve_neg_lap(f, g, band, p.h, rtol=1e-14)
    assert _rel(w.cpu().numpy(), want) < 1e-10


def test_tensor_copy_timeout_is_reported_and_recoverable(monkeypatch):
    p = wl.workload("c3", n=8)[0].replace(n=(64, 64, 64), model=0, precision=1)
    f = wl.random_fields(p.shape, 6, -1.0, 1.0)
    fd = torch.tensor(f, dtype=torch.float32, device=DEV)
    spec = torch.zeros((64, 64, 33), dtype=torch.complex64, device=DEV)
    back = torch.zeros(p.shape, dtype=torch.float32, device=DEV)
    ok = Plan(p)
    ok.fft_forward(fd, spec)
    plan = _plan_with_env(monkeypatch, p, ETD_WAIT_TRIES=0)
    with pytest.raises(EtdError) as ei:
        plan.fft_inverse(spec, back)     # the inverse pass A stages its input by a tensor copy
    assert ei.value.code == 6
    plan.close()
    torch.cuda.synchronize()
    ok.fft_inverse(spec, back)
    assert _rel(back.cpu().numpy().astype(np.float64), f) < 2e-6
    want = offt.half_spectrum(offt.fftn(f))
    assert _rel(spec.cpu().numpy(), want) < 2e-6
