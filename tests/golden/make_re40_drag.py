"""Writes re40_drag_330.txt: the oracle's drag history of the impulsively
started cylinder at Re 40 on the 330 x 330 grid of Table 3 (minimum width
0.02, uniform on [-0.54, 0.54]^2, stretched by about 1.02 to [-15, 15]^2),
158 boundary points (Table 1, system 1), freestream 1 on the left, top and
bottom, convective outflow on the right, uniform start (section 5.2).

The time step is not printed for this case; 0.01 is used (CFL 0.5 on the
freestream at the minimum width).  Run from the repository root:

    python tests/golden/make_re40_drag.py

It calls only the oracle and the input generators (about 15 minutes on one
core).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import Oracle  # noqa: E402

DT, T_END = 0.01, 60.0


def main():
    c = W.cylinder_impulsive_re40_330(DT, int(round(T_END / DT)))
    o = Oracle(c)
    rows = []
    t0 = time.time()
    every = int(round(0.5 / DT))
    for k in range(1, c.nsteps + 1):
        s = o.step()
        if k % every == 0:
            rows.append((s.t, s.cd, s.cl))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "re40_drag_330.txt")
    with open(out, "w") as f:
        f.write("# Drag and lift of the impulsively started cylinder, Re 40, 330 x 330 grid of Table 3,\n")
        f.write(f"# {c.n_b} points, dt {DT}; written by make_re40_drag.py from the oracle "
                f"({time.time() - t0:.0f} s).  Section 5.2 prints the steady drag 1.57.\n")
        f.write("# t cd cl\n")
        for t, cd, cl in rows:
            f.write(f"{t:.4f} {cd:.10f} {cl:.3e}\n")


if __name__ == "__main__":
    main()
