"""Temporal rates of the Sec. 2.2 scheme on the GPU in the paper's rate-study setting
(Sec. 4.1, Tables 1-2): 256^2 on [-1,1]^2, circle membrane, eps_phi = 10 h, eps_u = 10 h,
gamma = 100, B = 2000, M = 600 (ETD1) or 200 (ETDRK2), ubar = 0.3, U0 = 1 on a protein patch
holding 35% of the membrane's g-mass (a seeded connected stand-in for the paper's random
patch), T = 0.02.

The paper measures errors against a run at tau = 1e-6; here the rates come from successive
differences |U_tau - U_{tau/2}|_inf of runs at tau = 1e-4 / 2^k, k = 1..4, which converge at the
same order without a 20000-step reference.  The last rate is compared with the paper's printed
final rate for eps_u = 10 h (tests/golden/paper_table_rates.txt: ETD1 1.060, ETDRK2 1.882).
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_04347_gb300 import Plan  # noqa: E402
from paper_2606_04347_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_table_rates.txt")


def _paper_rates():
    rows = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, *vals = line.split()
            rows[name] = [float(v) for v in vals]
    return rows


def _run(scheme, tau, T=0.02):
    p, phi, u0 = wl.paper2d("circle", 10.0, scheme, 0, tau=tau)
    p = p.replace(model=2, cg_rtol=1e-11)
    plan = Plan(p)
    u = torch.tensor(u0, device="cuda:0")
    plan.step(torch.tensor(phi, device="cuda:0"), u, int(round(T / tau)), diag=True)
    plan.close()
    return u.cpu().numpy()


def test_sec2_rates_match_paper_tables():
    paper = _paper_rates()
    for scheme, name in ((1, "ETD1"), (2, "ETDRK2")):
        sols = [_run(scheme, 1e-4 / 2 ** k) for k in range(1, 5)]
        diffs = [float(np.max(np.abs(sols[i] - sols[i + 1]))) for i in range(3)]
        rates = [math.log2(diffs[i] / diffs[i + 1]) for i in range(2)]
        want = paper[name][1]
        print(name, "successive differences", diffs, "rates", rates, "paper (10h)", want)
        assert abs(rates[-1] - want) < 0.25, (name, rates, want)
