"""Pass A with its intermediate staged by tensor copies (TMA) against pass A with direct
loads and stores: the same arithmetic in the same order, so the transforms agree bit for bit.

The forward transform writes the four-step intermediate from pass A (staged store) and the
inverse reads it back (staged load); ETD_PASSA_DIRECT=1 selects the direct form for plans
created while it is set.  256^3 FP32 exercises the leftover columns (4 (Nx/2+1) = 516 columns
on 512 threads); 64^3 and the FP64 form do not have any.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_04347_gb300 import Plan  # noqa: E402
from paper_2606_04347_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def transforms(p, f, direct, monkeypatch):
    if direct:
        monkeypatch.setenv("ETD_PASSA_DIRECT", "1")
    else:
        monkeypatch.delenv("ETD_PASSA_DIRECT", raising=False)
    plan = Plan(p)
    fd = torch.tensor(f, dtype=torch.float64 if p.precision == 0 else torch.float32, device=DEV)
    spec = torch.zeros((p.n[2], p.n[1], p.n[0] // 2 + 1), dtype=plan.cdtype, device=DEV)
    plan.fft_forward(fd, spec)
    back = torch.zeros_like(fd)
    plan.fft_inverse(spec, back)
    out = spec.cpu().numpy(), back.cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("n,prec", [(64, 1), (64, 0), (256, 1)])
def test_staged_pass_a_matches_direct_bit_for_bit(n, prec, monkeypatch):
    p, phi, u, _ = wl.workload("c3", n=n, precision=prec)
    f = phi - 0.5 + 0.3 * u
    s_staged, b_staged = transforms(p, f, False, monkeypatch)
    s_direct, b_direct = transforms(p, f, True, monkeypatch)
    assert np.array_equal(s_staged.view(np.uint8), s_direct.view(np.uint8))
    assert np.array_equal(b_staged.view(np.uint8), b_direct.view(np.uint8))
