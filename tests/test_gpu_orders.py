"""Temporal orders of the GPU path (FP64): ETD1 first and ETDRK2 second order in tau.

The same fixed-membrane case as the oracle's order test (tests/test_oracle_etd.py, the
Sec. 2 model on the spectral split of Sec. 3, 32^2), run through the CUDA path against
its own fine-step solution, with the oracle test's bounds on the last observed rate.
On finer grids both the oracle and the GPU path see the ETDRK2 rate fall toward 1 over
the same step range (identical rates at 64^2: 1.46, 1.24), the order reduction of a stiff
problem, which is not asserted here.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import model as omodel  # noqa: E402
from paper_2606_04347_gb300 import Plan  # noqa: E402
from paper_2606_04347_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _rates(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def test_fixed_scheme_orders_on_gpu():
    p = wl.workload("c1", n=32)[0].replace(eps_u=0.4, gamma=20.0, M=20.0, B2=400.0, cg_rtol=1e-13)
    phi = wl.sphere_phi(p, 1.8, 0.3)
    u0 = wl.random_fields(p.shape, 9, 0.4, 0.6)
    T = 0.016

    def run(tau, scheme):
        plan = Plan(p.replace(tau=tau, scheme=scheme))
        u = torch.tensor(u0, dtype=torch.float64, device=DEV)
        plan.step(torch.tensor(phi, dtype=torch.float64, device=DEV), u, int(round(T / tau)))
        return u.cpu().numpy()

    sel = omodel.g_loc(phi) > p.recover_delta
    rates = {}
    for s in (1, 2):
        ref = run(T / 256, s)
        errs = [np.max(np.abs(run(T / m, s) - ref)[sel]) for m in (4, 8, 16)]
        rates[s] = _rates(errs)
    print("fixed 32^2 rates on the GPU: ETD1", rates[1], "ETDRK2", rates[2])
    assert 0.85 <= rates[1][-1] <= 1.15
    assert 1.75 <= rates[2][-1] <= 2.25
