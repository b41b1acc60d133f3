"""Writes wake_re<Re>.txt: the oracle's drag and lift history of the
cylinder wake of section 5.3 (Table 4) at one Reynolds number.

Grid and body as in ``workloads.cylinder_wake``: 30 x 30 domain, width 0.02
from x = -0.6 through the whole wake and for |y| <= 0.6, stretched by about
1.02 to the left, top and bottom (917 x 334 cells), 158 points, uniform
start.  The cylinder starts 0.05 above the centre and is brought to it at
constant speed over the first 0.5 time units (the start-up nudge of section
5.3; its size and duration are not printed); from then on it is fixed, and
the oracle keeps the factorisation of the last nudge step, whose body
positions are the final ones.  The time step is not printed: dt = 0.01 to
t = 150 at Re 100 and 150; at Re 200 that step diverges within the first
half time unit (the start-up flow reaches twice the freestream speed, a CFL
number of 1 for Adams-Bashforth 2 with less viscous damping), so Re 200 uses
dt = 0.005 to t = 100.  Run from the repository root, one process per
Reynolds number:

    python tests/golden/make_wake_forces.py 100
    python tests/golden/make_wake_forces.py 150
    python tests/golden/make_wake_forces.py 200 0.005 100

It calls only the oracle and the input generators (45 to 80 minutes on one
core per Reynolds number).
"""
import dataclasses
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import Oracle  # noqa: E402

def main(re: float, dt: float = 0.01, t_end: float = 150.0):
    every = int(round(0.1 / dt))
    c = W.cylinder_wake(re, dt, int(round(t_end / dt)))
    body = c.bodies[0]
    fixed = dataclasses.replace(c, bodies=[dataclasses.replace(body, nudge_y0=0.0, nudge_time=0.0)])
    o = Oracle(c)
    rows = []
    t0 = time.time()
    for k in range(1, c.nsteps + 1):
        s = o.step()
        if o.case is c and o.t >= body.nudge_time - 0.5 * dt:
            o.case = fixed
        if k % every == 0:
            rows.append((s.t, s.cd, s.cl))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"wake_re{int(re)}.txt")
    with open(out, "w") as f:
        f.write(f"# Drag and lift of the cylinder wake (section 5.3, Table 4) at Re {re:g}, {c.nx} x {c.ny} grid,\n")
        f.write(f"# {c.n_b} points, dt {dt:g}, nudge 0.05 over 0.5; written by make_wake_forces.py from the oracle "
                f"({time.time() - t0:.0f} s).\n")
        f.write("# t cd cl\n")
        for t, cd, cl in rows:
            f.write(f"{t:.4f} {cd:.10f} {cl:.10f}\n")


if __name__ == "__main__":
    main(*[float(a) for a in sys.argv[1:4]])
