"""FP64 CPU oracle of the immersed-boundary projection method (test infrastructure).

This module is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import or run it; the product
path (the CUDA library and its Python binding) never does.  It shares no code
with the CUDA path; only the seeded input generators of ``workloads`` serve
both.

What it computes (paper section "Immersed Boundary Projection Method"):
  * staggered Cartesian grid, possibly stretched (Eq. 2 context);
  * the Roma et al. 3-point discrete delta (Eq. 5) and the interpolation
    matrix E with E_{k,i} = dx dy d(x_i - xi_k) d(y_i - eta_k) (Eq. 4, Eq. 6),
    written on momentum fluxes q (u dy on x-faces, v dx on y-faces);
  * Adams-Bashforth 2 convection and Crank-Nicolson diffusion with central
    differences;
  * the transformed symmetric system in q, phi, f~ (Eq. 7, Eq. 8) with
    Q = [G E^T], and its approximate factorisation (Eq. 9a-c) with
    B^N = sum_{k<N} ((dt/2) M^-1 L)^k dt M^-1 (N = 1 by default: B^1 = dt M^-1);
  * one pressure value pinned (the sentence after Eq. 9);
  * both linear systems solved by a direct sparse LU (SuperLU), FP64, no
    iteration.

Readings of points the paper leaves open (it defers the transformed operators
to an appendix of another paper):
  R1  q_u = u dy_j, q_v = v dx_i; the x-momentum finite-volume balance is
      divided by dy_j and the y-balance by dx_i.  Then M_u = dxf_i / dy_j,
      M_v = dyf_j / dx_i, G is the +-1 cell-to-interior-face incidence
      (G^T = -divergence) and L is symmetric; A = M/dt - L/2.
  R2  B^1 = dt M^-1 (N = 1) for the paper's runs; B^N is the N-term
      expansion of A^-1 about dt M^-1 (pinned for N = 3 by Table 2's temporal
      order on the Couette flow).
  R3  Pinned cell p0 = (0, 0): its row and column are removed except the
      diagonal, and its right-hand side is set to zero.
  R4  Tangential Dirichlet values sit on the boundary, half a cell from the
      nearest unknown (one-sided difference).
  R5  Convection in conservative form on each staggered control volume, with
      linear interpolation to the control-volume faces.
  R6  AB2 start: N^{n-1} := N^n on the first step.
  R7  Convective outflow on the right edge, explicit first-order upwind with
      the freestream speed, for the normal (u) and tangential (v) values;
      then a uniform shift of the outflow u so that the net boundary flux is
      zero.
  R8  The delta uses h = the uniform cell width around the bodies; the force
      enters the momentum rows as +E^T f~ on the left, so f~ is the force
      exerted by the fluid on each body point; C_d = 2 sum f~_x / (U^2 D).
  R9  E is evaluated at the body positions of t^{n+1}; u_B at t^{n+1}.

Pinned (tests/test_oracle_pins.py) by the delta's moment identities, E exact
on linear fields, operator symmetry and null space, the dense saddle-point
solve of Eq. 8, the constraints after Eq. 9c, closed-form truncation orders,
the Taylor-Green decay and a manufactured solution with a momentum source,
Table 1's system sizes, the Couette closed form of section 5.1 (first order in
space), Table 2's temporal orders (N = 1 and N = 3), the
steady drag 1.57 of the Re 40 cylinder of section 5.2 (1.568 here), and
Table 4's Strouhal numbers and force coefficients of the cylinder wake.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Dict, Optional, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ----------------------------------------------------------------------------
# Discrete delta (Eq. 5)
# ----------------------------------------------------------------------------
def roma_delta(r, h: float):
    """d_h(r) of Roma, Peskin & Berger: support |r| <= 1.5 h (Eq. 5).

    The paper's case split has 0 < |r|/h <= 0.5 for the inner branch; r = 0
    belongs to that branch (the formula is continuous there)."""
    a = np.abs(np.asarray(r, dtype=np.float64)) / h
    out = np.zeros_like(a)
    inner = a <= 0.5
    outer = (a > 0.5) & (a <= 1.5)
    out[inner] = (1.0 + np.sqrt(1.0 - 3.0 * a[inner] ** 2)) / (3.0 * h)
    ao = a[outer]
    out[outer] = (5.0 - 3.0 * ao - np.sqrt(np.maximum(0.0, 1.0 - 3.0 * (1.0 - ao) ** 2))) / (6.0 * h)
    return out


# ----------------------------------------------------------------------------
# Grid and unknown numbering
# ----------------------------------------------------------------------------
class Grid:
    """Staggered grid from face coordinates xf (nx+1) and yf (ny+1): the
    staggered Cartesian grid of section 2, non-uniform where it is stretched
    away from the body (section 2; Table 3's grids).

    Unknown numbering (oracle's own):
      u unknown (i = 1..nx-1, j = 0..ny-1) -> j*(nx-1) + (i-1)
      v unknown (i = 0..nx-1, j = 1..ny-1) -> nu + (j-1)*nx + i
      cell (i, j) -> j*nx + i
    """

    def __init__(self, xf: np.ndarray, yf: np.ndarray):
        self.xf = np.asarray(xf, dtype=np.float64)
        self.yf = np.asarray(yf, dtype=np.float64)
        self.nx = len(xf) - 1
        self.ny = len(yf) - 1
        self.dx = np.diff(self.xf)
        self.dy = np.diff(self.yf)
        self.xc = 0.5 * (self.xf[:-1] + self.xf[1:])
        self.yc = 0.5 * (self.yf[:-1] + self.yf[1:])
        # dxf[i] = xc[i] - xc[i-1] for i = 1..nx-1 (index 0 and nx unused -> nan)
        self.dxf = np.full(self.nx + 1, np.nan)
        self.dxf[1:self.nx] = self.xc[1:] - self.xc[:-1]
        self.dyf = np.full(self.ny + 1, np.nan)
        self.dyf[1:self.ny] = self.yc[1:] - self.yc[:-1]
        self.nu = (self.nx - 1) * self.ny
        self.nv = self.nx * (self.ny - 1)
        self.nq = self.nu + self.nv
        self.nc = self.nx * self.ny

    # index helpers (vectorised)
    def iu(self, i, j):
        return j * (self.nx - 1) + (i - 1)

    def iv(self, i, j):
        return self.nu + (j - 1) * self.nx + i

    def ic(self, i, j):
        return j * self.nx + i

    def u_ij(self):
        """(I, J) of all u unknowns in numbering order."""
        J, I = np.meshgrid(np.arange(self.ny), np.arange(1, self.nx), indexing="ij")
        return I.ravel(), J.ravel()

    def v_ij(self):
        J, I = np.meshgrid(np.arange(1, self.ny), np.arange(self.nx), indexing="ij")
        return I.ravel(), J.ravel()

    # conversions between face arrays and q
    def q_from_uv(self, U: np.ndarray, V: np.ndarray) -> np.ndarray:
        """U (ny, nx+1), V (ny+1, nx) velocities -> fluxes q on interior faces."""
        qu = U[:, 1:self.nx] * self.dy[:, None]
        qv = V[1:self.ny, :] * self.dx[None, :]
        return np.concatenate([qu.ravel(), qv.ravel()])

    def uv_interior_from_q(self, q: np.ndarray):
        qu = q[:self.nu].reshape(self.ny, self.nx - 1)
        qv = q[self.nu:].reshape(self.ny - 1, self.nx)
        return qu / self.dy[:, None], qv / self.dx[None, :]


@dataclasses.dataclass
class Boundary:
    """Boundary velocities.

    u_left, u_right: normal u on x = xf[0], xf[nx] at rows j (ny each);
    v_bottom, v_top: normal v on y = yf[0], yf[ny] at columns i (nx each);
    u_bottom, u_top: tangential u on the bottom/top edge at x = xf[i] (nx+1);
    v_left, v_right: tangential v on the left/right edge at y = yf[j] (ny+1).
    """
    u_left: np.ndarray
    u_right: np.ndarray
    v_bottom: np.ndarray
    v_top: np.ndarray
    u_bottom: np.ndarray
    u_top: np.ndarray
    v_left: np.ndarray
    v_right: np.ndarray

    def copy(self) -> "Boundary":
        return Boundary(*[np.array(getattr(self, f.name)) for f in dataclasses.fields(self)])


# ----------------------------------------------------------------------------
# Operators
# ----------------------------------------------------------------------------
def mass_diag(g: Grid) -> np.ndarray:
    """M: dxf_i/dy_j on u unknowns, dyf_j/dx_i on v unknowns (reading R1)."""
    Iu, Ju = g.u_ij()
    Iv, Jv = g.v_ij()
    return np.concatenate([g.dxf[Iu] / g.dy[Ju], g.dyf[Jv] / g.dx[Iv]])


def laplacian(g: Grid, nu: float) -> sp.csr_matrix:
    """L acting on q (interior faces only; boundary values enter through
    ``laplacian_bc``): the viscous term of the momentum rows (section 2,
    central differences, Crank-Nicolson in A = M/dt - L/2 of Eq. 7).
    Finite-volume viscous flux balance of each staggered control volume,
    divided by dy_j (u) or dx_i (v) (reading R1; wall rows by reading R4)."""
    nx, ny = g.nx, g.ny
    rows, cols, vals = [], [], []

    def add(r, c, v):
        rows.append(r), cols.append(c), vals.append(v)

    # ---- u unknowns: control volume [xc_{i-1}, xc_i] x [yf_j, yf_{j+1}]
    I, J = g.u_ij()
    r = g.iu(I, J)
    dyj = g.dy[J]
    # x-direction: nu/dy_j * [(u_{i+1}-u_i)/dx_i - (u_i-u_{i-1})/dx_{i-1}] * dy_j / dy_j
    # with u = q/dy_j (same row j): coefficient nu/(dy_j dx)
    ce = nu / (dyj * g.dx[I])
    cw = nu / (dyj * g.dx[I - 1])
    add(r, r, -(ce + cw))
    m = I + 1 <= nx - 1
    add(r[m], g.iu(I[m] + 1, J[m]), ce[m])
    m = I - 1 >= 1
    add(r[m], g.iu(I[m] - 1, J[m]), cw[m])
    # y-direction: nu dxf_i/dy_j * [(u_{j+1}-u_j)/dyf_{j+1} - (u_j-u_{j-1})/dyf_j]
    dxfi = g.dxf[I]
    m = J + 1 <= ny - 1
    cn = np.zeros_like(dyj)
    cn[m] = nu * dxfi[m] / (dyj[m] * g.dyf[J[m] + 1])
    add(r[m], g.iu(I[m], J[m] + 1), cn[m] / g.dy[J[m] + 1])
    add(r[m], r[m], -cn[m] / dyj[m])
    m = ~m  # top wall: derivative (u_top - u_j)/(dy_j/2)
    add(r[m], r[m], -nu * dxfi[m] / dyj[m] * 2.0 / dyj[m] / dyj[m])
    m = J - 1 >= 0
    cs = np.zeros_like(dyj)
    cs[m] = nu * dxfi[m] / (dyj[m] * g.dyf[J[m]])
    add(r[m], g.iu(I[m], J[m] - 1), cs[m] / g.dy[J[m] - 1])
    add(r[m], r[m], -cs[m] / dyj[m])
    m = ~m  # bottom wall
    add(r[m], r[m], -nu * dxfi[m] / dyj[m] * 2.0 / dyj[m] / dyj[m])

    # ---- v unknowns: control volume [xf_i, xf_{i+1}] x [yc_{j-1}, yc_j]
    I, J = g.v_ij()
    r = g.iv(I, J)
    dxi = g.dx[I]
    # y-direction (normal): nu/dx_i * [(q_{j+1}-q_j)/dy_j - (q_j-q_{j-1})/dy_{j-1}]
    cn = nu / (dxi * g.dy[J])
    cs = nu / (dxi * g.dy[J - 1])
    add(r, r, -(cn + cs))
    m = J + 1 <= ny - 1
    add(r[m], g.iv(I[m], J[m] + 1), cn[m])
    m = J - 1 >= 1
    add(r[m], g.iv(I[m], J[m] - 1), cs[m])
    # x-direction (tangential): nu dyf_j/dx_i * [(v_{i+1}-v_i)/dxf_{i+1} - (v_i-v_{i-1})/dxf_i]
    dyfj = g.dyf[J]
    m = I + 1 <= nx - 1
    ce = np.zeros_like(dxi)
    ce[m] = nu * dyfj[m] / (dxi[m] * g.dxf[I[m] + 1])
    add(r[m], g.iv(I[m] + 1, J[m]), ce[m] / g.dx[I[m] + 1])
    add(r[m], r[m], -ce[m] / dxi[m])
    m = ~m  # right edge: (v_right - v_i)/(dx_i/2)
    add(r[m], r[m], -nu * dyfj[m] / dxi[m] * 2.0 / dxi[m] / dxi[m])
    m = I - 1 >= 0
    cw = np.zeros_like(dxi)
    cw[m] = nu * dyfj[m] / (dxi[m] * g.dxf[I[m]])
    add(r[m], g.iv(I[m] - 1, J[m]), cw[m] / g.dx[I[m] - 1])
    add(r[m], r[m], -cw[m] / dxi[m])
    m = ~m  # left edge
    add(r[m], r[m], -nu * dyfj[m] / dxi[m] * 2.0 / dxi[m] / dxi[m])

    R = np.concatenate(rows)
    C = np.concatenate(cols)
    Vv = np.concatenate(vals)
    return sp.csr_matrix((Vv, (R, C)), shape=(g.nq, g.nq))


def laplacian_bc(g: Grid, nu: float, b: Boundary) -> np.ndarray:
    """Boundary-value part of the viscous term, L_full(u) = L q + bc: the
    viscous share of bc_1 in Eq. 7 (section 2; tangential walls by reading R4)."""
    nx, ny = g.nx, g.ny
    out = np.zeros(g.nq)
    I, J = g.u_ij()
    r = g.iu(I, J)
    dyj = g.dy[J]
    # x neighbours that are boundary faces (i+1 = nx or i-1 = 0): nu/dy_j * u_b/dx * dy_j
    m = I + 1 == nx
    out[r[m]] += nu * b.u_right[J[m]] / g.dx[I[m]]
    m = I - 1 == 0
    out[r[m]] += nu * b.u_left[J[m]] / g.dx[I[m] - 1]
    dxfi = g.dxf[I]
    m = J == ny - 1
    out[r[m]] += nu * dxfi[m] / dyj[m] * 2.0 * b.u_top[I[m]] / dyj[m]
    m = J == 0
    out[r[m]] += nu * dxfi[m] / dyj[m] * 2.0 * b.u_bottom[I[m]] / dyj[m]

    I, J = g.v_ij()
    r = g.iv(I, J)
    dxi = g.dx[I]
    m = J + 1 == ny
    out[r[m]] += nu * b.v_top[I[m]] / g.dy[J[m]]
    m = J - 1 == 0
    out[r[m]] += nu * b.v_bottom[I[m]] / g.dy[J[m] - 1]
    dyfj = g.dyf[J]
    m = I == nx - 1
    out[r[m]] += nu * dyfj[m] / dxi[m] * 2.0 * b.v_right[J[m]] / dxi[m]
    m = I == 0
    out[r[m]] += nu * dyfj[m] / dxi[m] * 2.0 * b.v_left[J[m]] / dxi[m]
    return out


def gradient(g: Grid) -> sp.csr_matrix:
    """G of Eq. 7 (Q = [G E^T], section 2): cells -> interior faces,
    (G phi)_face = phi(right/upper cell) - phi(left/lower cell).
    G^T = -(divergence of q over interior faces), the continuity row of Eq. 2
    in q (reading R1)."""
    Iu, Ju = g.u_ij()
    Iv, Jv = g.v_ij()
    ru = g.iu(Iu, Ju)
    rv = g.iv(Iv, Jv)
    rows = np.concatenate([ru, ru, rv, rv])
    cols = np.concatenate([g.ic(Iu, Ju), g.ic(Iu - 1, Ju), g.ic(Iv, Jv), g.ic(Iv, Jv - 1)])
    vals = np.concatenate([np.ones(len(ru)), -np.ones(len(ru)), np.ones(len(rv)), -np.ones(len(rv))])
    return sp.csr_matrix((vals, (rows, cols)), shape=(g.nq, g.nc))


def divergence_full(g: Grid, q: np.ndarray, b: Boundary) -> np.ndarray:
    """Net outflow of each cell: (u_{i+1}-u_i) dy_j + (v_{j+1}-v_j) dx_i,
    with boundary faces from ``b``: the continuity row of Eq. 2 with its
    boundary part bc_2, so that -divergence_full(q*) = G^T q* + bc_2 is the
    pressure part of the right-hand side of Eq. 9b."""
    nx, ny = g.nx, g.ny
    QU = np.zeros((ny, nx + 1))
    QV = np.zeros((ny + 1, nx))
    QU[:, 1:nx] = q[:g.nu].reshape(ny, nx - 1)
    QV[1:ny, :] = q[g.nu:].reshape(ny - 1, nx)
    QU[:, 0] = b.u_left * g.dy
    QU[:, nx] = b.u_right * g.dy
    QV[0, :] = b.v_bottom * g.dx
    QV[ny, :] = b.v_top * g.dx
    div = (QU[:, 1:] - QU[:, :-1]) + (QV[1:, :] - QV[:-1, :])
    return div.ravel()


def interpolation_E(g: Grid, xb: np.ndarray, yb: np.ndarray, h: float) -> sp.csr_matrix:
    """E (2 n_b x n_q): rows 0..n_b-1 interpolate u, rows n_b.. interpolate v.

    Eq. 6 on velocities, E_{k,i} = dx dy d(x_i - xi_k) d(y_i - eta_k); on the
    flux q_u = u dy_j the entry becomes dxf_i d d (and dyf_j d d on q_v = v dx_i)
    so that E q is the interpolated velocity."""
    n_b = len(xb)
    rows, cols, vals = [], [], []
    for k in range(n_b):
        xi, eta = xb[k], yb[k]
        # u faces: x = xf[i] (i = 1..nx-1), y = yc[j]
        i_lo = np.searchsorted(g.xf, xi - 1.5 * h) - 1
        j_lo = np.searchsorted(g.yc, eta - 1.5 * h) - 1
        for i in range(max(i_lo, 1), min(i_lo + 5, g.nx)):
            dxw = roma_delta(g.xf[i] - xi, h)
            if dxw == 0.0:
                continue
            for j in range(max(j_lo, 0), min(j_lo + 5, g.ny)):
                dyw = roma_delta(g.yc[j] - eta, h)
                if dyw == 0.0:
                    continue
                rows.append(k), cols.append(g.iu(i, j)), vals.append(g.dxf[i] * dxw * dyw)
        # v faces: x = xc[i], y = yf[j] (j = 1..ny-1)
        i_lo = np.searchsorted(g.xc, xi - 1.5 * h) - 1
        j_lo = np.searchsorted(g.yf, eta - 1.5 * h) - 1
        for i in range(max(i_lo, 0), min(i_lo + 5, g.nx)):
            dxw = roma_delta(g.xc[i] - xi, h)
            if dxw == 0.0:
                continue
            for j in range(max(j_lo, 1), min(j_lo + 5, g.ny)):
                dyw = roma_delta(g.yf[j] - eta, h)
                if dyw == 0.0:
                    continue
                rows.append(n_b + k), cols.append(g.iv(i, j)), vals.append(g.dyf[j] * dxw * dyw)
    return sp.csr_matrix((np.array(vals, dtype=np.float64), (rows, cols)), shape=(2 * n_b, g.nq))


def convection(g: Grid, U: np.ndarray, V: np.ndarray, b: Boundary) -> np.ndarray:
    """N(q), the convective term of r^n (section 2: explicit Adams-Bashforth
    2, central differences): conservative convective flux balance of each
    staggered control volume divided by dy_j (u) or dx_i (v), central (linear)
    interpolation (reading R5).  U (ny, nx+1) and V (ny+1, nx) include the normal boundary
    values; tangential boundary values come from ``b``."""
    nx, ny = g.nx, g.ny
    dx, dy, dxf, dyf = g.dx, g.dy, g.dxf, g.dyf
    # ---------------- u control volumes, i = 1..nx-1, j = 0..ny-1
    i = np.arange(1, nx)[None, :]
    j = np.arange(ny)[:, None]
    Uc = U[:, 1:nx]
    uE = 0.5 * (Uc + U[:, 2:nx + 1])
    uW = 0.5 * (U[:, 0:nx - 1] + Uc)
    # value of u at the top corner (xf_i, yf_{j+1})
    uN = np.empty_like(Uc)
    wN = (0.5 * dy[:ny - 1] / dyf[1:ny])[:, None]
    uN[:ny - 1] = Uc[:ny - 1] + (Uc[1:] - Uc[:ny - 1]) * wN
    uN[ny - 1] = b.u_top[1:nx]
    uS = np.empty_like(Uc)
    wS = (0.5 * dy[:ny - 1] / dyf[1:ny])[:, None]
    uS[1:] = Uc[:ny - 1] + (Uc[1:] - Uc[:ny - 1]) * wS
    uS[0] = b.u_bottom[1:nx]
    # v at the corners (xf_i, yf_{j+1}) and (xf_i, yf_j): interpolate in x
    wx = (0.5 * dx[0:nx - 1] / dxf[1:nx])[None, :]
    vN = V[1:ny + 1, 0:nx - 1] + (V[1:ny + 1, 1:nx] - V[1:ny + 1, 0:nx - 1]) * wx
    vS = V[0:ny, 0:nx - 1] + (V[0:ny, 1:nx] - V[0:ny, 0:nx - 1]) * wx
    Nu = (uE ** 2 - uW ** 2) + (uN * vN - uS * vS) * (dxf[1:nx][None, :] / dy[:, None])

    # ---------------- v control volumes, i = 0..nx-1, j = 1..ny-1
    Vc = V[1:ny, :]
    vN2 = 0.5 * (Vc + V[2:ny + 1, :])
    vS2 = 0.5 * (V[0:ny - 1, :] + Vc)
    # u at (xf_{i+1}, yf_j) and (xf_i, yf_j): interpolate in y between rows j-1, j
    wy = (0.5 * dy[0:ny - 1] / dyf[1:ny])[:, None]
    uE2 = U[0:ny - 1, 1:nx + 1] + (U[1:ny, 1:nx + 1] - U[0:ny - 1, 1:nx + 1]) * wy
    uW2 = U[0:ny - 1, 0:nx] + (U[1:ny, 0:nx] - U[0:ny - 1, 0:nx]) * wy
    vE2 = np.empty_like(Vc)
    wE = (0.5 * dx[0:nx - 1] / dxf[1:nx])[None, :]
    vE2[:, :nx - 1] = Vc[:, :nx - 1] + (Vc[:, 1:] - Vc[:, :nx - 1]) * wE
    vE2[:, nx - 1] = b.v_right[1:ny]
    vW2 = np.empty_like(Vc)
    vW2[:, 1:] = Vc[:, :nx - 1] + (Vc[:, 1:] - Vc[:, :nx - 1]) * wE
    vW2[:, 0] = b.v_left[1:ny]
    Nv = (uE2 * vE2 - uW2 * vW2) * (dyf[1:ny][:, None] / dx[None, :]) + (vN2 ** 2 - vS2 ** 2)
    return np.concatenate([Nu.ravel(), Nv.ravel()])


# ----------------------------------------------------------------------------
# Boundary conditions
# ----------------------------------------------------------------------------
def freestream_boundary(g: Grid, U: np.ndarray, V: np.ndarray, uinf: float, vinf: float) -> Boundary:
    """External-flow boundary values of sections 5.2 and 5.3: Dirichlet
    (U, V) on left, bottom, top; right-edge values taken from the given face
    arrays (u) and set to V (tangential v) initially."""
    nx, ny = g.nx, g.ny
    return Boundary(u_left=np.full(ny, uinf), u_right=np.array(U[:, nx]),
                    v_bottom=np.full(nx, vinf), v_top=np.full(nx, vinf),
                    u_bottom=np.full(nx + 1, uinf), u_top=np.full(nx + 1, uinf),
                    v_left=np.full(ny + 1, vinf), v_right=np.full(ny + 1, vinf))


def wall_boundary(g: Grid) -> Boundary:
    """Walls at rest on all four sides (the closed box of section 5.1)."""
    nx, ny = g.nx, g.ny
    z = np.zeros
    return Boundary(z(ny), z(ny), z(nx), z(nx), z(nx + 1), z(nx + 1), z(ny + 1), z(ny + 1))


def convective_outflow(g: Grid, b: Boundary, U: np.ndarray, V: np.ndarray,
                       uinf: float, dt: float) -> Boundary:
    """Convective outflow of section 5.2: right-edge values at t^{n+1} from
    du/dt + U du/dx = 0, explicit
    first-order upwind from time-n values, then a uniform shift of the
    outflow u that makes the net boundary flux zero (reading R7)."""
    nx, ny = g.nx, g.ny
    nb = b.copy()
    cu = uinf * dt / g.dx[nx - 1]
    nb.u_right = b.u_right - cu * (b.u_right - U[:, nx - 1])
    cv = uinf * dt / (0.5 * g.dx[nx - 1])
    nb.v_right = b.v_right.copy()
    nb.v_right[1:ny] = b.v_right[1:ny] - cv * (b.v_right[1:ny] - V[1:ny, nx - 1])
    inflow = np.sum(nb.u_left * g.dy) + np.sum(nb.v_bottom * g.dx) - np.sum(nb.v_top * g.dx)
    outflow = np.sum(nb.u_right * g.dy)
    nb.u_right = nb.u_right + (inflow - outflow) / np.sum(g.dy)
    return nb


# ----------------------------------------------------------------------------
# The time step (Eq. 9a-c)
# ----------------------------------------------------------------------------
def pin_matrix(S: sp.spmatrix, p0: int) -> sp.csr_matrix:
    """Remove the off-diagonal entries of row and column p0: one pressure
    value pinned (the sentence after Eq. 9; reading R3)."""
    S = sp.csr_matrix(S)
    n = S.shape[0]
    d = S[p0, p0]
    keep = np.ones(n)
    keep[p0] = 0.0
    K = sp.diags(keep)
    e = sp.csr_matrix(([d], ([p0], [p0])), shape=(n, n))
    return (K @ S @ K + e).tocsr()


@dataclasses.dataclass
class StepStats:
    t: float
    cd: float
    cl: float
    fx: float
    fy: float
    max_div: float
    slip: float


class Oracle:
    """Direct-solve FP64 implementation of the factorised step (Eq. 9a-c).

    ``bc_fn(t) -> Boundary`` overrides the freestream/walls boundary values
    (time-dependent Dirichlet data for closed-form tests); ``source_fn(t) ->
    array(n_q)`` adds a momentum source to r1 (manufactured solutions).
    ``bn_exact=True`` replaces B^1 by A^-1 (dense, small grids only) so that
    the factorisation is exact.  ``bn_order=N`` uses the N-term expansion of
    A^-1 = (M/dt - L/2)^-1 about dt M^-1 (Eq. 9 with B^N):
    B^N = sum_{k<N} ((dt/2) M^-1 L)^k dt M^-1, which is symmetric because L is
    and M is diagonal.
    """

    def __init__(self, case, pin_cell: Tuple[int, int] = (0, 0),
                 bc_fn: Optional[Callable[[float], Boundary]] = None,
                 source_fn: Optional[Callable[[float], np.ndarray]] = None,
                 bn_exact: bool = False, U0=None, V0=None, factorize: bool = True, bn_order: int = 1):
        self.case = case
        g = self.g = Grid(case.xf, case.yf)
        self.nu_visc = case.nu
        self.dt = case.dt
        self.h = case.h
        self.bc_fn = bc_fn
        self.source_fn = source_fn
        self.bn_exact = bn_exact
        self.bn_order = int(bn_order)
        if self.bn_order < 1:
            raise ValueError("bn_order must be >= 1")
        self.p0 = g.ic(*pin_cell)
        self.M = mass_diag(g)
        self.L = laplacian(g, case.nu)
        self.A = (sp.diags(self.M / case.dt) - 0.5 * self.L).tocsc()
        self.G = gradient(g)
        self.Bdiag = case.dt / self.M
        # factorize=False builds the operators only (residual checks at sizes
        # where a direct factorisation is too slow)
        self._A_lu = spla.splu(self.A, permc_spec="MMD_AT_PLUS_A") if factorize else None
        self._Ainv = None
        if bn_exact:
            self._Ainv = np.linalg.inv(self.A.toarray())
        if U0 is None:
            U0, V0 = case.initial_velocity()
        self.t = 0.0
        self.step_count = 0
        if bc_fn is not None:
            self.bnd = bc_fn(0.0)
        elif case.bc == "freestream":
            self.bnd = freestream_boundary(g, U0, V0, case.uinf, case.vinf)
        else:
            self.bnd = wall_boundary(g)
        self.q = g.q_from_uv(U0, V0)
        self.N_prev = None
        self.n_b = case.n_b
        self.lam = np.zeros(g.nc + 2 * self.n_b)
        self._S_lu = None
        self._E_t = None
        self.E = None
        self.S = None
        self.last_solve = {}

    # ---- full face arrays of the current state
    def face_arrays(self, q=None, b: Optional[Boundary] = None):
        g = self.g
        q = self.q if q is None else q
        b = self.bnd if b is None else b
        U = np.zeros((g.ny, g.nx + 1))
        V = np.zeros((g.ny + 1, g.nx))
        ui, vi = g.uv_interior_from_q(q)
        U[:, 1:g.nx] = ui
        V[1:g.ny, :] = vi
        U[:, 0], U[:, g.nx] = b.u_left, b.u_right
        V[0, :], V[g.ny, :] = b.v_bottom, b.v_top
        return U, V

    def set_state(self, U, V, N_prev=None, lam=None, t=None, step=None, v_right=None):
        g = self.g
        self.q = g.q_from_uv(U, V)
        self.bnd.u_right = np.array(U[:, g.nx])
        self.bnd.u_left = np.array(U[:, 0])
        self.bnd.v_bottom = np.array(V[0, :])
        self.bnd.v_top = np.array(V[g.ny, :])
        if v_right is not None:
            self.bnd.v_right = np.array(v_right)
        self.N_prev = None if N_prev is None else np.array(N_prev)
        if lam is not None:
            self.lam = np.array(lam)
        if t is not None:
            self.t = t
        if step is not None:
            self.step_count = step

    # ---- operators at given body positions
    def build_poisson(self, xb, yb, factorize: bool = True):
        g = self.g
        self.E = interpolation_E(g, xb, yb, self.h) if self.n_b else sp.csr_matrix((0, g.nq))
        Q = sp.hstack([self.G, self.E.T]).tocsr()
        if self.bn_exact:
            S = Q.T @ (self._Ainv @ Q.toarray())
            S = sp.csr_matrix(S)
        else:
            S = (Q.T @ self.B_matrix() @ Q).tocsr()
        self.Q = Q
        self.S_unpinned = S
        self.S = pin_matrix(S, self.p0)
        self._S_lu = spla.splu(self.S.tocsc(), permc_spec="MMD_AT_PLUS_A") if factorize else None

    def B_matrix(self):
        """B^N as a sparse matrix (B^1 = dt M^-1 is diagonal)."""
        Minv = sp.diags(1.0 / self.M)
        term = sp.diags(self.Bdiag).tocsr()
        B = term
        K = (0.5 * self.dt) * (Minv @ self.L)
        for _ in range(1, self.bn_order):
            term = (K @ term).tocsr()
            B = B + term
        return B.tocsr()

    def apply_B(self, x):
        if self.bn_exact:
            return self._Ainv @ x
        y = self.Bdiag * x
        out = y
        for _ in range(1, self.bn_order):
            y = (0.5 * self.dt) * (self.L @ y) / self.M
            out = out + y
        return out

    def explicit_terms(self):
        """(r1, boundary at t^{n+1}, body state at t^{n+1}) for the current
        state, without solving (used for residual checks of a computed step)."""
        g, dt, case = self.g, self.dt, self.case
        tn, tn1 = self.t, self.t + dt
        b_n = self.bnd
        U, V = self.face_arrays()
        if self.bc_fn is not None:
            b_n1 = self.bc_fn(tn1)
        elif case.bc == "freestream":
            b_n1 = convective_outflow(g, b_n, U, V, case.uinf, dt)
        else:
            b_n1 = b_n.copy()
        N = convection(g, U, V, b_n)
        N_prev = N if self.N_prev is None else self.N_prev
        r1 = (self.M / dt) * self.q + 0.5 * (self.L @ self.q + laplacian_bc(g, self.nu_visc, b_n)) \
            + 0.5 * laplacian_bc(g, self.nu_visc, b_n1) - (1.5 * N - 0.5 * N_prev)
        return r1, b_n1, case.body_state(tn1), N

    def step(self) -> StepStats:
        g, dt, case = self.g, self.dt, self.case
        tn, tn1 = self.t, self.t + dt
        b_n = self.bnd
        U, V = self.face_arrays()
        # boundary values at t^{n+1}
        if self.bc_fn is not None:
            b_n1 = self.bc_fn(tn1)
        elif case.bc == "freestream":
            b_n1 = convective_outflow(g, b_n, U, V, case.uinf, dt)
        else:
            b_n1 = b_n.copy()
        # body positions at t^{n+1} (reading R9)
        xb, yb, ub, vb = case.body_state(tn1)
        if self._S_lu is None or case.moving:
            self.build_poisson(xb, yb)
        # explicit terms: AB2 convection, CN diffusion (Eq. 7 right-hand side)
        N = convection(g, U, V, b_n)
        N_prev = N if self.N_prev is None else self.N_prev
        r1 = (self.M / dt) * self.q + 0.5 * (self.L @ self.q + laplacian_bc(g, self.nu_visc, b_n)) \
            + 0.5 * laplacian_bc(g, self.nu_visc, b_n1) - (1.5 * N - 0.5 * N_prev)
        if self.source_fn is not None:
            r1 = r1 + self.source_fn(tn + 0.5 * dt)
        # Eq. 9a
        if self.bn_exact:
            qs = self._Ainv @ r1
        else:
            qs = self._A_lu.solve(r1)
        # Eq. 9b right-hand side: [G^T q* + bc2 ; E q* - u_B]
        rhs_phi = -divergence_full(g, qs, b_n1)
        rhs_f = self.E @ qs - np.concatenate([ub, vb]) if self.n_b else np.zeros(0)
        rhs = np.concatenate([rhs_phi, rhs_f])
        rhs[self.p0] = 0.0
        lam = self._S_lu.solve(rhs)
        # Eq. 9c
        qn1 = qs - self.apply_B(self.Q @ lam)
        self.last_solve = {"r1": r1, "qstar": qs, "rhs2": rhs, "lam": lam}
        self.q = qn1
        self.N_prev = N
        self.lam = lam
        self.bnd = b_n1
        self.t = tn1
        self.step_count += 1
        return self.stats(ub, vb)

    def forces(self):
        nb = self.n_b
        f = self.lam[self.g.nc:]
        return f[:nb], f[nb:]

    def stats(self, ub=None, vb=None) -> StepStats:
        g = self.g
        fx, fy = self.forces()
        Fx, Fy = float(np.sum(fx)), float(np.sum(fy))
        uref = self.case.uinf if self.case.uinf != 0 else 1.0
        D = self.case.bodies[0].diameter if self.case.bodies else 1.0
        div = divergence_full(g, self.q, self.bnd)
        slip = 0.0
        if self.n_b and ub is not None:
            slip = float(np.max(np.abs(self.E @ self.q - np.concatenate([ub, vb]))))
        return StepStats(t=self.t, cd=2.0 * Fx / (uref ** 2 * D), cl=2.0 * Fy / (uref ** 2 * D),
                         fx=Fx, fy=Fy, max_div=float(np.max(np.abs(div))), slip=slip)

    def run(self, nsteps: int):
        return [self.step() for _ in range(nsteps)]
