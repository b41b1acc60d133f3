"""Seeded synthetic inputs for the immersed-boundary projection method.

This module is shared by the CPU oracle (``oracle/``) and by the CUDA path
(``paper_1109_3524_gb300``).  It holds only input generation: grid face
coordinates, Lagrangian body points, prescribed body kinematics, the initial
velocity field with its seeded perturbation, and the named workload
configurations.  None of the method's arithmetic (operators, convection,
solves, projection) lives here.

Workloads follow the cases of the paper:
  * flow past a circular cylinder (D = 1) on a uniform or stretched staggered
    grid, uniform inflow, convective outflow (section "Flow over an
    impulsively started cylinder", Table 3; "External flow over a circular
    cylinder", Table 4);
  * a transversely oscillating cylinder and a 2x2 array of cylinders, two of
    them heaving (moving-body cases, section "Simulations of wake flows and
    moving boundaries");
  * Couette flow between concentric cylinders (section "Couette flow between
    concentric cylinders").
The paper's grids are exponentially stretched away from a uniform core around
the body (Table 3, ratio 1.01-1.02); the rule used here is stated in
``stretched_faces``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Tuple

import numpy as np

MASK64 = (1 << 64) - 1


# ----------------------------------------------------------------------------
# Counter-based random numbers: splitmix64 (Steele, Lea & Flood 2014).
# ----------------------------------------------------------------------------
def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied elementwise to uint64 counters."""
    z = (x + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(MASK64)
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & np.uint64(MASK64)
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & np.uint64(MASK64)
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from splitmix64(seed ^ (stream << 40) ^ index)."""
    idx = np.arange(n, dtype=np.uint64)
    key = np.uint64((seed ^ (stream << 40)) & MASK64)
    with np.errstate(over="ignore"):
        z = splitmix64(idx ^ key)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ----------------------------------------------------------------------------
# Grids
# ----------------------------------------------------------------------------
def uniform_faces(n: int, lo: float, hi: float) -> np.ndarray:
    """n+1 equally spaced face coordinates on [lo, hi]."""
    return np.linspace(lo, hi, n + 1)


def _geometric_extent(h: float, r: float, s: int) -> float:
    # width of the k-th stretched cell (k = 1..s) is h r^k
    return h * r * (r ** s - 1.0) / (r - 1.0)


def stretched_faces(n: int, half_core: float, half_domain: float,
                    ratio: float = 1.02) -> Tuple[np.ndarray, dict]:
    """Face coordinates of a symmetric stretched grid of n cells.

    A uniform core [-half_core, half_core] of n - 2s cells of width h is
    flanked on each side by s cells of widths h r, h r^2, ..., h r^s.  The
    side count s is the one for which ratio ``ratio`` gives the side extent
    closest to half_domain - half_core; r is then adjusted by bisection so
    that the extent is exact.  (The paper states only the stretching ratio and
    the core extent, Table 3; this rule is a reading of it.)
    """
    a, L = half_core, half_domain
    best = None
    for s in range(1, n // 2):
        h = 2.0 * a / (n - 2 * s)
        e = _geometric_extent(h, ratio, s)
        d = abs(e - (L - a))
        if best is None or d < best[0]:
            best = (d, s, h)
    _, s, h = best
    lo, hi = 1.0 + 1e-12, 1.5
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _geometric_extent(h, mid, s) < L - a:
            lo = mid
        else:
            hi = mid
    r = 0.5 * (lo + hi)
    ncore = n - 2 * s
    core = -a + h * np.arange(ncore + 1)
    core[-1] = a
    widths = h * r ** np.arange(1, s + 1)
    right = a + np.cumsum(widths)
    right[-1] = L
    faces = np.concatenate([-right[::-1], core, right])
    info = {"n_core": ncore, "n_side": s, "h": h, "ratio": r}
    assert faces.shape == (n + 1,)
    assert np.all(np.diff(faces) > 0)
    return faces, info


# ----------------------------------------------------------------------------
# Bodies
# ----------------------------------------------------------------------------
def cylinder_points(n_b: int, xc: float = 0.0, yc: float = 0.0,
                    diameter: float = 1.0) -> Tuple[np.ndarray, np.ndarray]:
    """n_b points equally spaced in angle on a circle, the first at angle 0."""
    th = 2.0 * np.pi * np.arange(n_b) / n_b
    rad = 0.5 * diameter
    return xc + rad * np.cos(th), yc + rad * np.sin(th)


@dataclasses.dataclass
class Body:
    """A rigid cylinder with an optional prescribed transverse heave
    y_c(t) = y0 + amp sin(2 pi freq t), and an optional start-up nudge: an
    offset nudge_y0 removed at constant speed over 0 <= t < nudge_time."""
    n_b: int
    xc: float
    yc: float
    diameter: float = 1.0
    heave_amp: float = 0.0
    heave_freq: float = 0.0
    omega: float = 0.0          # rigid rotation rate (Couette inner cylinder)
    nudge_y0: float = 0.0
    nudge_time: float = 0.0

    def _yoff(self, t: float) -> float:
        y = self.heave_amp * math.sin(2.0 * math.pi * self.heave_freq * t)
        if self.nudge_y0 != 0.0 and t < self.nudge_time:
            y += self.nudge_y0 * (1.0 - t / self.nudge_time)
        return y

    def positions(self, t: float) -> Tuple[np.ndarray, np.ndarray]:
        return cylinder_points(self.n_b, self.xc, self.yc + self._yoff(t), self.diameter)

    def velocities(self, t: float) -> Tuple[np.ndarray, np.ndarray]:
        vy = self.heave_amp * 2.0 * math.pi * self.heave_freq * math.cos(
            2.0 * math.pi * self.heave_freq * t)
        if self.nudge_y0 != 0.0 and t < self.nudge_time:
            vy -= self.nudge_y0 / self.nudge_time
        x, y = self.positions(t)
        ub = -self.omega * (y - (self.yc + self._yoff(t)))
        vb = self.omega * (x - self.xc) + vy
        return ub, vb

    @property
    def moving(self) -> bool:
        return self.heave_amp != 0.0 or self.nudge_y0 != 0.0

    @property
    def perimeter(self) -> float:
        return math.pi * self.diameter


def ellipse_points(n_b: int, chord: float = 1.0, thickness: float = 0.12) -> Tuple[np.ndarray, np.ndarray]:
    """n_b points equally spaced in arc length on an ellipse with semi-axes
    chord / 2 (along x) and thickness * chord / 2, in the body frame; the first
    point is the tip at (chord / 2, 0), then counter-clockwise."""
    a, b = 0.5 * chord, 0.5 * thickness * chord
    m = 200000
    s = np.linspace(0.0, 2.0 * np.pi, m + 1)
    x, y = a * np.cos(s), b * np.sin(s)
    arc = np.concatenate([[0.0], np.cumsum(np.hypot(np.diff(x), np.diff(y)))])
    target = arc[-1] * np.arange(n_b) / n_b
    st = np.interp(target, arc, s)
    return a * np.cos(st), b * np.sin(st)


def ellipse_perimeter(chord: float = 1.0, thickness: float = 0.12) -> float:
    x, y = ellipse_points(1, chord, thickness)  # noqa: F841 (same sampling as the points)
    a, b = 0.5 * chord, 0.5 * thickness * chord
    s = np.linspace(0.0, 2.0 * np.pi, 200001)
    return float(np.sum(np.hypot(np.diff(a * np.cos(s)), np.diff(b * np.sin(s)))))


@dataclasses.dataclass
class FlappingEllipse:
    """Rigid elliptic airfoil (thickness-to-chord ratio ``thickness``) whose
    centre moves along the x axis and which rotates about its centre
    (section 6.2): x_c(t) = x0 + (A0 / 2) cos(2 pi f t), y_c = y0,
    alpha(t) = alpha0 + beta sin(2 pi f t + phi), alpha measured from the line
    of oscillation (the x axis) to the chord, counter-clockwise."""
    n_b: int
    A0: float = 2.8
    freq: float = 0.25
    alpha0: float = 0.5 * math.pi
    beta: float = 0.25 * math.pi
    phi: float = 0.0
    x0: float = 0.0
    y0: float = 0.0
    chord: float = 1.0
    thickness: float = 0.12

    def __post_init__(self):
        self._local = ellipse_points(self.n_b, self.chord, self.thickness)

    @property
    def diameter(self) -> float:       # reference length of the force coefficients
        return self.chord

    @property
    def perimeter(self) -> float:
        return ellipse_perimeter(self.chord, self.thickness)

    @property
    def moving(self) -> bool:
        return True

    def state(self, t: float):
        w = 2.0 * math.pi * self.freq
        xc = self.x0 + 0.5 * self.A0 * math.cos(w * t)
        uc = -0.5 * self.A0 * w * math.sin(w * t)
        al = self.alpha0 + self.beta * math.sin(w * t + self.phi)
        om = self.beta * w * math.cos(w * t + self.phi)
        return xc, uc, al, om

    def positions(self, t: float) -> Tuple[np.ndarray, np.ndarray]:
        xc, _, al, _ = self.state(t)
        lx, ly = self._local
        c, s = math.cos(al), math.sin(al)
        return xc + c * lx - s * ly, self.y0 + s * lx + c * ly

    def velocities(self, t: float) -> Tuple[np.ndarray, np.ndarray]:
        xc, uc, _, om = self.state(t)
        x, y = self.positions(t)
        return uc - om * (y - self.y0), om * (x - xc)

    @property
    def max_speed(self) -> float:
        """Maximum translational speed pi f A0 (the velocity scale of Re)."""
        return math.pi * self.freq * self.A0


# ----------------------------------------------------------------------------
# Cases
# ----------------------------------------------------------------------------
BC_FREESTREAM = "freestream"   # Dirichlet U,V on left/bottom/top, convective outflow right
BC_WALLS = "walls"             # Dirichlet U,V on all four sides (box)


@dataclasses.dataclass
class Case:
    name: str
    xf: np.ndarray
    yf: np.ndarray
    bodies: List[Body]
    nu: float
    dt: float
    nsteps: int
    uinf: float = 1.0
    vinf: float = 0.0
    bc: str = BC_FREESTREAM
    noise_amp: float = 0.0
    seed: int = 0
    h: float = 0.0                 # uniform cell width around the bodies
    grid_info: Optional[dict] = None

    @property
    def nx(self) -> int:
        return len(self.xf) - 1

    @property
    def ny(self) -> int:
        return len(self.yf) - 1

    @property
    def n_b(self) -> int:
        return sum(b.n_b for b in self.bodies)

    @property
    def moving(self) -> bool:
        return any(b.moving for b in self.bodies)

    def body_state(self, t: float):
        """Concatenated (xb, yb, ub, vb) of all bodies at time t."""
        if not self.bodies:
            z = np.zeros(0)
            return z, z, z, z
        xs, ys, us, vs = [], [], [], []
        for b in self.bodies:
            x, y = b.positions(t)
            u, v = b.velocities(t)
            xs.append(x), ys.append(y), us.append(u), vs.append(v)
        return (np.concatenate(xs), np.concatenate(ys),
                np.concatenate(us), np.concatenate(vs))

    def spacing_over_h(self) -> List[float]:
        """Arc spacing of each body's points (perimeter / n_b) divided by the delta
        width h.  Section 2 asks for a spacing close to the cell width; well
        above 1 the body leaks (fluid passes between the points' supports)."""
        return [b.perimeter / b.n_b / self.h for b in self.bodies]

    def initial_velocity(self) -> Tuple[np.ndarray, np.ndarray]:
        """Face velocities at t = 0 (boundary faces included).

        u has shape (ny, nx+1) (x-faces i = 0..nx at cell-centre rows j),
        v has shape (ny+1, nx).  For the freestream case the field is the
        uniform (U, V) with U(-a, a) noise of amplitude ``noise_amp`` added to
        every interior face, drawn from splitmix64 with stream 1 for u and
        stream 2 for v, in row-major order of the interior faces.
        """
        nx, ny = self.nx, self.ny
        if self.bc == BC_FREESTREAM:
            u = np.full((ny, nx + 1), self.uinf)
            v = np.full((ny + 1, nx), self.vinf)
        else:
            u = np.zeros((ny, nx + 1))
            v = np.zeros((ny + 1, nx))
        if self.noise_amp != 0.0:
            nu_int = ny * (nx - 1)
            nv_int = (ny - 1) * nx
            a = self.noise_amp
            u[:, 1:nx] += (a * (2.0 * uniform01(self.seed, nu_int, 1) - 1.0)).reshape(ny, nx - 1)
            v[1:ny, :] += (a * (2.0 * uniform01(self.seed, nv_int, 2) - 1.0)).reshape(ny - 1, nx)
        return u, v


def _check_bodies_in_core(case: Case, margin_cells: float = 2.0, times=None) -> None:
    """Every body point, with the delta support plus a margin, must lie in
    the uniform part of the grid (the discrete delta needs uniform cells
    near the body)."""
    h = case.h
    if times is None:
        times = (0.0, 0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 1.75, 2.0, 2.25, 2.5)
    for axis_faces, coord in ((case.xf, 0), (case.yf, 1)):
        w = np.diff(axis_faces)
        uni = np.abs(w - h) <= 1e-9 * h
        for t in times:
            pts = case.body_state(t)[coord]
            for p in (pts.min() - margin_cells * h, pts.max() + margin_cells * h):
                k = np.searchsorted(axis_faces, p) - 1
                assert 0 <= k < len(w) and uni[k], "body outside the uniform core"


def cylinder_re40_128(seed: int = 0) -> Case:
    """Fixed cylinder, 128x128 uniform grid on [-2,2]^2, 100 points, Re 40,
    dt 0.005, 50 steps, 1e-3 uniform noise on interior velocities."""
    xf = uniform_faces(128, -2.0, 2.0)
    c = Case("cylinder_re40_128", xf, xf.copy(), [Body(100, 0.0, 0.0)],
             nu=1.0 / 40.0, dt=0.005, nsteps=50, noise_amp=1e-3, seed=seed,
             h=4.0 / 128)
    _check_bodies_in_core(c)
    return c


def cylinder_stretched(n: int, re: float, dt: float, nsteps: int, n_b: int = 630,
                       seed: int = 0, name: Optional[str] = None) -> Case:
    """Fixed cylinder at the origin on an n x n grid over [-15,15]^2,
    uniform in [-2,2]^2 and stretched by ratio 1.02 outside."""
    xf, info = stretched_faces(n, 2.0, 15.0, 1.02)
    c = Case(name or f"cylinder_re{int(re)}_{n}", xf, xf.copy(), [Body(n_b, 0.0, 0.0)],
             nu=1.0 / re, dt=dt, nsteps=nsteps, seed=seed, h=info["h"], grid_info=info)
    _check_bodies_in_core(c)
    return c


def wake_faces(h: float, half_core: float, half_domain: float,
               ratio: float = 1.02) -> Tuple[np.ndarray, dict]:
    """Faces over [-half_domain, half_domain] with width h from -half_core to
    +half_domain (the whole wake) and geometric widths h r, h r^2, ... to the
    left; the left cell count is the one for which ``ratio`` gives the extent
    closest to half_domain - half_core, and r is then set by bisection so that
    the extent is exact (section 5.3 gives only the minimum width, the
    uniform wake and the ratio)."""
    a, L = half_core, half_domain
    nu = int(round((L + a) / h))
    assert abs(nu * h - (L + a)) < 1e-9 * L
    s = min(range(1, 2000), key=lambda k: abs(_geometric_extent(h, ratio, k) - (L - a)))
    lo, hi = 1.0 + 1e-12, 1.5
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _geometric_extent(h, mid, s) < L - a:
            lo = mid
        else:
            hi = mid
    r = 0.5 * (lo + hi)
    left = -a - np.cumsum(h * r ** np.arange(1, s + 1))
    left[-1] = -L
    uni = -a + h * np.arange(nu + 1)
    uni[-1] = L
    faces = np.concatenate([left[::-1], uni])
    assert np.all(np.diff(faces) > 0)
    return faces, {"n_uniform": nu, "n_left": s, "h": h, "ratio": r}


def cylinder_wake(re: float, dt: float = 0.01, nsteps: int = 10000, nudge_y0: float = 0.05,
                  nudge_time: float = 0.5) -> Case:
    """Cylinder wake of section 5.3: 30 x 30 domain, width 0.02 from x = -0.6
    through the whole wake, stretched by about 1.02 to the left, top and
    bottom (uniform for |y| <= 0.6), 158 points, uniform start.  The cylinder
    starts offset by nudge_y0 and is brought to the centre at constant speed
    over nudge_time (the start-up nudge of section 5.3; its size and duration
    are not printed)."""
    h = 0.02
    xf, xinfo = wake_faces(h, 0.6, 15.0, 1.02)
    yf, yinfo = stretched_faces(60 + 2 * 137, 0.6, 15.0, 1.02)
    assert abs(yinfo["h"] - h) < 1e-12
    c = Case(f"cylinder_wake_re{int(re)}", xf, yf,
             [Body(158, 0.0, 0.0, nudge_y0=nudge_y0, nudge_time=nudge_time)], nu=1.0 / re, dt=dt,
             nsteps=nsteps, h=h, grid_info={"x": xinfo, "y": yinfo})
    _check_bodies_in_core(c)
    return c


def cylinder_impulsive_re40_330(dt: float = 0.01, nsteps: int = 6000) -> Case:
    """Impulsively started cylinder at Re 40 on the 330 x 330 grid of Table 3:
    minimum width 0.02, uniform on [-0.54, 0.54]^2, stretched by about 1.02
    to [-15, 15]^2; 158 points (Table 1, system 1); uniform start, no noise.
    The time step is not printed for this case (0.01 gives CFL 0.5 on the
    freestream at the minimum width)."""
    xf, info = stretched_faces(330, 0.54, 15.0, 1.02)
    return Case("cylinder_impulsive_re40_330", xf, xf.copy(), [Body(158, 0.0, 0.0)], nu=1.0 / 40.0, dt=dt,
                nsteps=nsteps, h=info["h"], grid_info=info)


def flapping_ellipse(nx: int = 930, ny: int = 654, ratio: float = 1.01, re: float = 75.0,
                     dt: float = 0.001, nsteps: int = 4000, n_b: int = 101) -> Case:
    """Flapping airfoil of section 6.2 in fluid at rest: elliptic airfoil of
    chord 1 and thickness-to-chord ratio 0.12, A0 / c = 2.8, alpha0 = pi / 2,
    beta = pi / 4, f = 0.25, phi = 0, Re = 75 on the maximum translational
    speed pi f A0 and the chord; 30 x 30 domain, uniform cells on
    [-2, 2] x [-0.52, 0.52], stretched by about ``ratio`` outside (the grid
    rule of ``stretched_faces``: 930 x 654 cells give width 0.01 and ratio
    1.00996 in both directions, Table 1's system 3 with its 101 points); one
    flapping period is 4000 steps of 0.001.  The walls are at rest (Dirichlet zero on
    the left, bottom and top; the convective outflow on the right carries
    nothing with U = 0)."""
    xf, xinfo = stretched_faces(nx, 2.0, 15.0, ratio)
    yf, yinfo = stretched_faces(ny, 0.52, 15.0, ratio)
    h = xinfo["h"]
    if abs(yinfo["h"] - h) > 1e-12 * h:
        raise ValueError(f"core widths differ: {h} (x) and {yinfo['h']} (y)")
    body = FlappingEllipse(n_b)
    c = Case(f"flapping_ellipse_re{int(re)}_{nx}x{ny}", xf, yf, [body],
             nu=body.max_speed * body.chord / re, dt=dt, nsteps=nsteps, uinf=0.0, vinf=0.0, h=h,
             grid_info={"x": xinfo, "y": yinfo})
    # the chord reaches y = +-0.5 at alpha = pi / 2, one delta support (1.5 h)
    # from the end of the uniform band at width 0.01
    _check_bodies_in_core(c, margin_cells=1.5, times=np.linspace(0.0, 1.0 / body.freq, 65))
    return c


def oscillating_cylinder(n: int = 1024, re: float = 100.0, dt: float = 0.002,
                         nsteps: int = 2000, n_b: int = 630) -> Case:
    """Cylinder heaving transversely with amplitude 0.2 D at frequency 0.2."""
    xf, info = stretched_faces(n, 2.0, 15.0, 1.02)
    c = Case(f"oscillating_cylinder_re{int(re)}_{n}", xf, xf.copy(),
             [Body(n_b, 0.0, 0.0, heave_amp=0.2, heave_freq=0.2)],
             nu=1.0 / re, dt=dt, nsteps=nsteps, h=info["h"], grid_info=info)
    _check_bodies_in_core(c)
    return c


def four_cylinders(n: int = 4096, re: float = 150.0, dt: float = 0.0005,
                   nsteps: int = 500, n_b_each: int = 630) -> Case:
    """2x2 cylinders at (+-1.5, +-1.5); the downstream pair heaves in phase
    with amplitude 0.25 D at frequency 0.2.  Core enlarged to [-3,3]^2."""
    xf, info = stretched_faces(n, 3.0, 15.0, 1.02)
    bodies = [Body(n_b_each, -1.5, -1.5), Body(n_b_each, -1.5, 1.5),
              Body(n_b_each, 1.5, -1.5, heave_amp=0.25, heave_freq=0.2),
              Body(n_b_each, 1.5, 1.5, heave_amp=0.25, heave_freq=0.2)]
    c = Case(f"four_cylinders_re{int(re)}_{n}", xf, xf.copy(), bodies,
             nu=1.0 / re, dt=dt, nsteps=nsteps, h=info["h"], grid_info=info)
    _check_bodies_in_core(c)
    return c


def couette(n: int, dt: float, nsteps: int, n_inner: Optional[int] = None,
            n_outer: Optional[int] = None) -> Case:
    """Couette flow between concentric cylinders r_i = 0.5 (rotating at
    Omega = 0.5) and r_o = 1 (fixed), nu = 0.03, in a closed box
    [-1.5,1.5]^2 with walls at rest, uniform n x n grid."""
    xf = uniform_faces(n, -1.5, 1.5)
    h = 3.0 / n
    if n_inner is None:
        n_inner = int(round(np.pi * 1.0 / h))
    if n_outer is None:
        n_outer = int(round(np.pi * 2.0 / h))
    bodies = [Body(n_inner, 0.0, 0.0, 1.0, omega=0.5), Body(n_outer, 0.0, 0.0, 2.0)]
    c = Case(f"couette_{n}", xf, xf.copy(), bodies, nu=0.03, dt=dt, nsteps=nsteps,
             uinf=0.0, vinf=0.0, bc=BC_WALLS, h=h)
    return c


def body_free(n: int, lo: float = -1.0, hi: float = 1.0, nu: float = 0.01,
              dt: float = 0.01) -> Case:
    """Uniform grid with no immersed body (plain 5-point Poisson system)."""
    xf = uniform_faces(n, lo, hi)
    return Case(f"body_free_{n}", xf, xf.copy(), [], nu=nu, dt=dt, nsteps=1,
                h=(hi - lo) / n)


def table1_system(k: int) -> Case:
    """The four coupled systems of Table 1 rebuilt with cylinders of D = 1
    (section 3 names only their sizes and point counts).
      1: 330 x 330, 158 points: the Re 40 grid of Table 3;
      2: 986 x 986, 786 points: the Re 3000 grid of Table 3 (minimum width
         0.004, uniform on [-0.52, 0.52]^2, ratio about 1.01);
      3: 930 x 654, 101 points (a flapping wing in the paper): uniform cells
         of width pi / 101 with a cylinder at the centre;
      4: 690 x 690, 474 points (three moving cylinders in the paper): uniform
         cells of width 0.02, three cylinders of 158 points."""
    if k == 1:
        return cylinder_impulsive_re40_330(nsteps=1)
    if k == 2:
        xf, info = stretched_faces(986, 0.52, 15.0, 1.01)
        return Case("table1_system2", xf, xf.copy(), [Body(786, 0.0, 0.0)], nu=1.0 / 3000.0, dt=0.002,
                    nsteps=1, h=info["h"], grid_info=info)
    if k == 3:
        h = math.pi / 101
        xf = h * (np.arange(931) - 465.0)
        yf = h * (np.arange(655) - 327.0)
        return Case("table1_system3", xf, yf, [Body(101, 0.0, 0.0)], nu=1.0 / 75.0, dt=0.005, nsteps=1, h=h)
    if k == 4:
        h = 0.02
        xf = h * (np.arange(691) - 345.0)
        bodies = [Body(158, -2.0, 0.0), Body(158, 1.0, 1.5), Body(158, 1.0, -1.5)]
        return Case("table1_system4", xf, xf.copy(), bodies, nu=0.01, dt=0.005, nsteps=1, h=h)
    raise ValueError(k)


def resolved_points(n: int, half_core: float, half_domain: float = 15.0, diameter: float = 1.0) -> int:
    """Points of a cylinder whose arc spacing equals the uniform width h of
    ``stretched_faces(n, half_core, half_domain)``: round(pi D / h)."""
    _, info = stretched_faces(n, half_core, half_domain, 1.02)
    return int(round(math.pi * diameter / info["h"]))


def named(name: str) -> Case:
    """Workloads by name (sizes in the name)."""
    table = {
        "cylinder_re40_128": lambda: cylinder_re40_128(),
        "cylinder_re100_1024": lambda: cylinder_stretched(1024, 100.0, 0.002, 2000),
        "cylinder_re200_2048": lambda: cylinder_stretched(2048, 200.0, 0.001, 1000),
        "oscillating_cylinder_re100_1024": lambda: oscillating_cylinder(),
        "four_cylinders_re150_4096": lambda: four_cylinders(),
        "flapping_ellipse_re75_930x654": lambda: flapping_ellipse(),
        # the same grids with point spacing equal to h (n_b = round(pi D / h))
        "cylinder_re200_2048_resolved": lambda: cylinder_stretched(2048, 200.0, 0.001, 1000,
                                                                   n_b=resolved_points(2048, 2.0)),
        "four_cylinders_re150_4096_resolved": lambda: four_cylinders(n_b_each=resolved_points(4096, 3.0)),
    }
    return table[name]()


def he_normal(shapes, seed: int = 0) -> np.ndarray:
    """Initial parameters of a convolution network: for each (k, cin, cout)
    in `shapes`, He-normal weights W[ky, kx, cin, cout] with standard deviation
    sqrt(2 / (k k cin)) from splitmix64 counters (Box-Muller, stream 100 + i),
    then zero biases.  Returned as one flat float64 vector."""
    parts = []
    for i, (k, ci, co) in enumerate(shapes):
        nw = k * k * ci * co
        u = uniform01(seed, 2 * nw, stream=100 + i)
        u1 = np.maximum(u[:nw], 1e-300)
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u[nw:])
        parts.append(z * np.sqrt(2.0 / (k * k * ci)))
        parts.append(np.zeros(co))
    return np.concatenate(parts)
