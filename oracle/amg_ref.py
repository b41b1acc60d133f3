"""Plain NumPy/SciPy application of a smoothed-aggregation hierarchy and of
CG / flexible CG (test infrastructure).

Only ``tests/`` may import this module.  Given the level operators A_l, the
prolongators P_l (restriction R_l = P_l^T) and the damped-Jacobi weights of a
hierarchy, it applies one V-cycle exactly as defined for the preconditioner of
Eq. 9b (section 3 of the paper uses a smoothed-aggregation V-cycle inside
preconditioned CG): on each level, `pre` damped-Jacobi sweeps starting from
zero, residual, restriction by P^T, recursion, prolongation and correction,
`post` damped-Jacobi sweeps; the coarsest level is solved directly in FP64.
"""
import numpy as np
import scipy.sparse as sp


def vcycle(As, Ps, omegas, b, pre=2, post=2, level=0, coarse_inv=None, pre0=None, post0=None):
    """pre0 / post0 (default: pre / post) are the sweep counts of the finest
    level alone, which the library can set apart from the coarser levels."""
    A = As[level]
    if level == len(As) - 1:
        if coarse_inv is None:
            coarse_inv = np.linalg.inv(A.toarray())
        return coarse_inv @ b
    npre = pre0 if (level == 0 and pre0 is not None) else pre
    npost = post0 if (level == 0 and post0 is not None) else post
    d = A.diagonal()
    w = omegas[level]
    x = w * b / d
    for _ in range(npre - 1):
        x = x + w * (b - A @ x) / d
    r = b - A @ x
    xc = vcycle(As, Ps, omegas, Ps[level].T @ r, pre, post, level + 1, coarse_inv)
    x = x + Ps[level] @ xc
    for _ in range(npost):
        x = x + w * (b - A @ x) / d
    return x


def pcg(A, b, M, x0=None, tol=1e-10, maxit=1000):
    """Preconditioned CG with the stopping rule ||b - A x|| <= tol ||b||."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    bb = np.linalg.norm(b)
    if bb == 0:
        return np.zeros_like(b), 0
    if np.linalg.norm(r) <= tol * bb:
        return x, 0
    z = M(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        if np.linalg.norm(r) <= tol * bb:
            return x, it
        z = M(r)
        rzn = r @ z
        p = z + (rzn / rz) * p
        rz = rzn
    return x, maxit


def csr(n, m, rowptr, col, val):
    return sp.csr_matrix((val, col, rowptr), shape=(n, m))
