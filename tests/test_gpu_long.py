"""Long runs of the FP64 GPU form against the FP64 oracle.

* 100 coupled ETDRK2 steps of c3 at 32^3, fields compared in relative L2 (the 1e-11 bar for
  FP64 after 100 steps); the oracle runs here, about half a minute.
* The full 500 steps of c3 at 64^3 against the oracle's run of the same steps
  (tests/golden/c3_64_long.txt, written by tests/golden/make_c3_64_long.py from the oracle
  alone): max|2U - 1| over the recovery set and the volume <phi, 1>_h after every 25th step
  (the file's mass column, <G (U - ubar), 1>_h, is not what etd_energy reports: its mass is
  the energy's <g (f(U) - ubar), 1>_h).  The run is the workload's full length; the GPU
  form has to follow the oracle through all of it.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import etd as oetd  # noqa: E402
from paper_2606_04347_gb300 import Plan  # noqa: E402
from paper_2606_04347_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c3_64_long.txt")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_c3_32_fp64_100_steps_matches_the_oracle():
    p, phi, u, _ = wl.workload("c3", n=32)
    want_phi, want_u = oetd.CoupledStepper(p).run(phi.copy(), u.copy(), 100)
    plan = Plan(p)
    f = torch.tensor(phi, dtype=torch.float64, device=DEV)
    ud = torch.tensor(u, dtype=torch.float64, device=DEV)
    plan.step(f, ud, 100)
    e_phi, e_u = rel_l2(f.cpu().numpy(), want_phi), rel_l2(ud.cpu().numpy(), want_u)
    print("100 steps at 32^3: rel L2 phi", e_phi, "u", e_u)
    assert e_phi < 1e-11
    assert e_u < 1e-11


def test_c3_64_fp64_500_steps_tracks_the_oracle():
    rows = np.loadtxt(GOLDEN, comments="#")
    p, phi, u, _ = wl.workload("c3", n=64)
    plan = Plan(p.replace(precision=0, cg_rtol=1e-12, cg_rtol_pred=0.0))
    f = torch.tensor(phi, dtype=torch.float64, device=DEV)
    ud = torch.tensor(u, dtype=torch.float64, device=DEV)
    done = 0
    worst = [0.0, 0.0]
    for step, mb, vol, _ in rows:
        plan.step(f, ud, int(step) - done)
        done = int(step)
        d = plan.energy(f, ud)
        e = [abs(d["max_bound"] - mb) / mb, abs(d["volume"] - vol) / abs(vol)]
        worst = [max(a, b) for a, b in zip(worst, e)]
    print("500 steps at 64^3, worst relative differences (bound, volume):", worst)
    assert worst[0] < 1e-9
    assert worst[1] < 1e-12
