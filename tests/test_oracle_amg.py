"""Pins of the reference V-cycle and PCG (oracle/amg_ref.py), which the GPU
V-cycle kernels are compared against: properties fixed by the mathematics,
independent of the reference's own code."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.amg_ref import pcg, vcycle


def _poisson2d(n):
    """SPD 5-point Laplacian with a Dirichlet diagonal shift (n x n cells)."""
    e = np.ones(n)
    T = sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1])
    I = sp.identity(n)
    return (sp.kron(I, T) + sp.kron(T, I) + 0.01 * sp.identity(n * n)).tocsr()


def _aggregation(n, a=2):
    """Piecewise-constant prolongator of a x a aggregates on an n x n grid."""
    m = (n + a - 1) // a
    rows, cols = [], []
    for j in range(n):
        for i in range(n):
            rows.append(j * n + i)
            cols.append((j // a) * m + (i // a))
    return sp.csr_matrix((np.ones(n * n), (rows, cols)), shape=(n * n, m * m))


def _hierarchy(n=12):
    A0 = _poisson2d(n)
    P0 = _aggregation(n)
    A1 = (P0.T @ A0 @ P0).tocsr()
    P1 = _aggregation((n + 1) // 2)
    A2 = (P1.T @ A1 @ P1).tocsr()
    return [A0, A1, A2], [P0, P1], [0.6, 0.6, 0.6]


def test_identity_prolongator_gives_the_exact_solve():
    """With P = I the coarse correction solves the level exactly and the
    post-sweeps leave the solution fixed: V(b) = A^-1 b."""
    A = _poisson2d(8)
    b = np.random.default_rng(0).standard_normal(A.shape[0])
    I = sp.identity(A.shape[0], format="csr")
    z = vcycle([A, A], [I], [0.6, 0.6], b)
    x = spla.spsolve(A.tocsc(), b)
    assert np.abs(z - x).max() <= 1e-12 * np.abs(x).max()


def test_vcycle_is_linear_and_symmetric():
    """Equal pre- and post-sweeps with R = P^T make the V-cycle a symmetric
    linear operator (a transposed restriction or an unmatched sweep breaks it)."""
    As, Ps, om = _hierarchy()
    rng = np.random.default_rng(1)
    u, w = rng.standard_normal(As[0].shape[0]), rng.standard_normal(As[0].shape[0])
    Vu, Vw = vcycle(As, Ps, om, u), vcycle(As, Ps, om, w)
    assert np.abs(vcycle(As, Ps, om, 2.0 * u - 3.0 * w) - (2.0 * Vu - 3.0 * Vw)).max() <= 1e-12 * np.abs(Vu).max()
    assert abs(u @ Vw - w @ Vu) <= 1e-12 * abs(u @ Vw)
    # and positive definite on these vectors
    assert u @ Vu > 0 and w @ Vw > 0


def test_pcg_with_vcycle_converges_to_the_direct_solve():
    As, Ps, om = _hierarchy()
    b = np.random.default_rng(2).standard_normal(As[0].shape[0])
    x, it = pcg(As[0], b, lambda r: vcycle(As, Ps, om, r), tol=1e-12)
    xd = spla.spsolve(As[0].tocsc(), b)
    assert np.abs(x - xd).max() <= 1e-9 * np.abs(xd).max()
    # the V-cycle is a useful preconditioner: far fewer iterations than unknowns
    assert it < 40


def test_jacobi_sweep_on_a_diagonal_operator():
    """For a diagonal A and weight 1 the first damped-Jacobi sweep is already
    the exact solve, so every later step leaves it fixed: V(b) = A^-1 b."""
    rng = np.random.default_rng(3)
    d = rng.uniform(0.5, 2.0, 64)
    A0 = sp.diags(d).tocsr()
    P0 = _aggregation(8)
    A1 = (P0.T @ A0 @ P0).tocsr()
    b = rng.standard_normal(64)
    z = vcycle([A0, A1], [P0], [1.0, 1.0], b)
    assert np.abs(z - b / d).max() <= 1e-13 * np.abs(b / d).max()
