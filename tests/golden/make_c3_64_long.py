"""Writes c3_64_long.txt: the FP64 oracle's coupled ETDRK2 run of the c3 workload at 64^3
(ellipsoid membrane, random U on the band, tau = 1e-4; Algorithm 1 of Sec. 3.3) over 500
steps, with max|2U - 1| over the recovery set (G > 1e-3), the volume <phi, 1>_h and the mass
<G (U - ubar), 1>_h after every 25th step.  Calls the oracle only; takes about 40 minutes.

    python tests/golden/make_c3_64_long.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import etd as oetd  # noqa: E402
from oracle import model as omodel  # noqa: E402
from paper_2606_04347_gb300 import workloads as wl  # noqa: E402


def main():
    p, phi, u, _ = wl.workload("c3", n=64)
    cs = oetd.CoupledStepper(p)
    lines = ["# c3 at 64^3, FP64 oracle, coupled ETDRK2 (Algorithm 1), tau = 1e-4; written by make_c3_64_long.py",
             "# step max|2U-1| over G > 1e-3, <phi,1>_h, <G (U - ubar),1>_h"]
    for k in range(20):
        phi, u = cs.run(phi, u, 25)
        G = omodel.g_loc(phi)
        mb = omodel.bound_stats(u, G, p.recover_delta)[0]
        lines.append(f"{25 * (k + 1)} {mb!r} {omodel.volume(phi, p)!r} {omodel.mass_coupled(u, G, p)!r}")
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "c3_64_long.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
