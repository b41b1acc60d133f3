"""The allocation-free residual check (ibm_poisson_residual_norms_noalloc).

Some callers cannot allocate device memory where they call the library (a
fixed device-memory plan, a host callback, a program without a framework
allocator); this entry point keeps its residual and reduction scratch in a
static device array of the library.  The test compares it, through the C ABI,
with the existing operator entry point (ibm_apply_poisson) on two calls in a
row, and checks that an oversized system is rejected.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1109_3524_gb300 as P
    from paper_1109_3524_gb300.build import ensure_built
    ensure_built()
    P.load()
    return P


def test_noalloc_norms_match_apply_poisson_twice(pkg):
    import torch
    case = W.cylinder_re40_128()
    sim = pkg.Sim.from_case(case)
    rng = np.random.default_rng(11)
    for call in range(2):   # two calls in a row share (and reuse) the static scratch
        lam = torch.tensor(rng.standard_normal(sim.n_lambda), device="cuda")
        rhs = torch.tensor(rng.standard_normal(sim.n_lambda), device="cuda")
        bb, rr = sim.residual_norms_noalloc(lam, rhs)
        r = (rhs - sim.apply_poisson(lam)).cpu().numpy()
        b = rhs.cpu().numpy()
        assert abs(bb - b @ b) <= 1e-12 * (b @ b), (call, bb, b @ b)
        assert abs(rr - r @ r) <= 1e-12 * (r @ r), (call, rr, r @ r)


def test_noalloc_just_under_the_static_size(pkg):
    """A body-free 1440^2 grid: 2 073 600 entries, just under the 2^21 limit,
    so the reduction runs at its 1024-block cap (several grid-stride passes)
    and the residual fills the array almost to its end."""
    import torch
    n = 1440
    xf = W.uniform_faces(n, -1.0, 1.0)
    case = W.Case("near_limit", xf, xf.copy(), [], nu=0.01, dt=0.01, nsteps=1, h=2.0 / n)
    sim = pkg.Sim.from_case(case, poisson_precond=pkg.IBM_PRECOND_NONE)
    assert sim.n_lambda == n * n and (1 << 21) - n * n < 1 << 15
    rng = np.random.default_rng(12)
    for call in range(2):
        lam = torch.tensor(rng.standard_normal(sim.n_lambda), device="cuda")
        rhs = torch.tensor(rng.standard_normal(sim.n_lambda), device="cuda")
        bb, rr = sim.residual_norms_noalloc(lam, rhs)
        r = (rhs - sim.apply_poisson(lam)).cpu().numpy()
        b = rhs.cpu().numpy()
        assert abs(bb - b @ b) <= 1e-12 * (b @ b), (call, bb, b @ b)
        assert abs(rr - r @ r) <= 1e-12 * (r @ r), (call, rr, r @ r)
    sim.close()


def test_noalloc_rejects_systems_beyond_the_static_size(pkg):
    import ctypes as C
    n = 1460   # 1460^2 cells > 2^21 lambda entries
    xf = W.uniform_faces(n, -1.0, 1.0)
    case = W.Case("big", xf, xf.copy(), [], nu=0.01, dt=0.01, nsteps=1, h=2.0 / n)
    h = pkg.create_host_only(pkg.Config.for_case(case), case.xf, case.yf)
    out = np.zeros(2)
    # the size check comes before any device work; the pointers are never used
    rc = h.lib.ibm_poisson_residual_norms_noalloc(h.ctx, C.c_void_p(256), C.c_void_p(256),
                                                  out.ctypes.data_as(C.POINTER(C.c_double)))
    assert rc == 1
    assert b"exceeds the static scratch maximum" in h.lib.ibm_last_error(h.ctx)
