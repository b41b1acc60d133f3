"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 results must match the oracle to 1e-8 relative (velocity, lambda, force
coefficients) when both linear systems are solved to 1e-12; reduced-precision
(FP32 V-cycle) results are checked against the bound stated in each test.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import Oracle
from oracle.amg_ref import csr, vcycle

pytestmark = pytest.mark.gpu

TOL_PARITY = 1e-8


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


def _torch():
    import torch
    return torch


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def _uniform_case(nx, ny, nb, moving=False, D=1.0, dt=0.005, re=40.0, noise=1e-3):
    L = 4.0
    xf = W.uniform_faces(nx, -L / 2, L / 2)
    hy = L / nx
    yf = -0.5 * ny * hy + hy * np.arange(ny + 1)
    body = W.Body(nb, 0.02, -0.013, D, heave_amp=0.2 if moving else 0.0, heave_freq=0.2 if moving else 0.0)
    return W.Case(f"u{nx}x{ny}", xf, yf, [body] if nb else [], nu=1.0 / re, dt=dt, nsteps=3,
                  noise_amp=noise, seed=7, h=L / nx)


def _sim(pkg, case, **kw):
    kw.setdefault("tol1", 1e-12)
    kw.setdefault("tol2", 1e-12)
    kw.setdefault("max_iter2", 20000)
    s = pkg.Sim.from_case(case, **kw)
    U0, V0 = case.initial_velocity()
    vr = np.full(case.ny + 1, case.vinf if case.bc == "freestream" else 0.0)
    s.set_state(u=U0, v=V0, v_right=vr, t=0.0, step=0)
    return s


def _step_both(sim, o, case):
    xb, yb, ub, vb = case.body_state(o.t + case.dt)
    if case.n_b:
        sim.set_body(xb, yb, ub, vb)
    st = sim.step(1)[0]
    so = o.step()
    return st, so


def _compare_state(sim, o, tol=TOL_PARITY):
    s = sim.get_state()
    Uo, Vo = o.face_arrays()
    scale = max(np.abs(Uo).max(), np.abs(Vo).max())
    eu = np.abs(s["u"] - Uo).max() / scale
    ev = np.abs(s["v"] - Vo).max() / scale
    el = _rel(s["lambda"], o.lam)
    assert eu < tol and ev < tol and el < tol, (eu, ev, el)
    return eu, ev, el


# ----------------------------------------------------------------------------
# operators and the V-cycle
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(128, 128), (150, 131), (53, 38)])
def test_poisson_operator_matches_oracle(pkg, shape):
    torch = _torch()
    nx, ny = shape
    case = _uniform_case(nx, ny, int(np.pi / (4.0 / nx)))
    sim = _sim(pkg, case)
    o = Oracle(case, factorize=False)
    xb, yb, _, _ = case.body_state(case.dt)
    o.build_poisson(xb, yb, factorize=False)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(o.S.shape[0])
    y = sim.apply_poisson(torch.tensor(x, device="cuda")).cpu().numpy()
    assert _rel(y, o.S @ x) < 1e-13


@pytest.mark.parametrize("mixed", [False, True])
def test_device_body_rows_match_oracle_operator(pkg, mixed):
    """A moving body with the Schur preconditioner: the body rows (E, E^T,
    the coupling rows C and F of Q^T B Q and the force-row diagonal) are
    formed on the device from the host's sparsity pattern.  After three moves
    of the heaving cylinder the library's Poisson operator equals the
    oracle's at the same positions (1e-13), and a step from there equals the
    oracle's step (1e-8)."""
    torch = _torch()
    case = _uniform_case(96, 96, int(np.pi / (4.0 / 96)), moving=True, dt=0.01, re=100.0)
    sim = _sim(pkg, case, poisson_precond=pkg.IBM_PRECOND_SCHUR, amg_rebuild_every=1, moving=1,
               precision=pkg.IBM_PREC_MIXED if mixed else pkg.IBM_PREC_FP64)
    o = Oracle(case)
    for _ in range(3):
        _step_both(sim, o, case)
    xb, yb, ub, vb = case.body_state(o.t + case.dt)
    sim.set_body(xb, yb, ub, vb)
    ob = Oracle(case, factorize=False)
    ob.build_poisson(xb, yb, factorize=False)
    x = np.random.default_rng(21).standard_normal(ob.S.shape[0])
    y = sim.apply_poisson(torch.tensor(x, device="cuda")).cpu().numpy()
    assert _rel(y, ob.S @ x) < 1e-13
    st = sim.step(1)[0]
    so = o.step()
    assert abs(st["cd"] - so.cd) <= TOL_PARITY * abs(so.cd)
    _compare_state(sim, o)


@pytest.mark.parametrize("mixed", [False, True])
def test_vcycle_matches_reference(pkg, mixed):
    torch = _torch()
    case = W.cylinder_re40_128()
    sim = _sim(pkg, case, precision=pkg.IBM_PREC_MIXED if mixed else pkg.IBM_PREC_FP64)
    L = sim.amg_levels()
    As = [csr(*sim.amg_matrix(l, 0)) for l in range(L)]
    Ps = [csr(*sim.amg_matrix(l, 1)) for l in range(L - 1)]
    om = [sim.amg_level_info(l)[1] for l in range(L)]
    rng = np.random.default_rng(5)
    r = rng.standard_normal(As[0].shape[0])
    z = sim.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
    zr = vcycle(As, Ps, om, r)
    # FP64: same arithmetic up to summation order; FP32 V-cycle: single-precision bound
    assert _rel(z, zr) < (2e-5 if mixed else 1e-11)


@pytest.mark.parametrize("mixed", [False, True])
def test_pressure_vcycle_full_size(pkg, mixed):
    """Pressure-block V-cycle of the Schur preconditioner on the 1024^2
    stretched workload against the NumPy V-cycle on the same hierarchy, with
    the coarse levels as one cluster kernel from 16384 rows (operators staged
    in shared memory) and from 65536 rows (too large to stage), and with one
    kernel per sweep throughout."""
    torch = _torch()
    case = W.named("cylinder_re100_1024")
    prec = pkg.IBM_PREC_MIXED if mixed else pkg.IBM_PREC_FP64
    rng = np.random.default_rng(9)
    r = rng.standard_normal(case.nx * case.ny)
    out = {}
    for tail in (65536, 16384, 0):
        sim = _sim(pkg, case, poisson_precond=pkg.IBM_PRECOND_SCHUR, precision=prec, amg_tail_rows=tail,
                   amg_theta=0.02, amg_max_coarse=2048)
        L = sim.amg_levels()
        if tail:
            ns = [sim.amg_level_info(l)[0] for l in range(L)]
            assert ns[1] > 65536 and min(ns[1:]) <= 65536   # both paths in use
            As = [csr(*sim.amg_matrix(l, 0)) for l in range(L)]
            Ps = [csr(*sim.amg_matrix(l, 1)) for l in range(L - 1)]
            om = [sim.amg_level_info(l)[1] for l in range(L)]
            zr = vcycle(As, Ps, om, r)
        out[tail] = sim.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
        sim.close()
    tol = 2e-5 if mixed else 1e-11
    for tail in (65536, 16384, 0):
        assert _rel(out[tail], zr) < tol
        assert _rel(out[tail], out[0]) < tol


@pytest.mark.parametrize("sweeps0", [1, 2, 3, 4, 5, 6])
def test_fused_finest_level_matches_reference(pkg, sweeps0):
    """The temporally blocked finest level of the FP32 pressure-block V-cycle
    (pre-sweeps + residual in one kernel, post-sweeps in another, tiles of
    (64 - 2 S) x 32 cells with an S-cell halo) on a ragged 150 x 131 grid with
    a body and the pinned corner cell, for every supported sweep count S,
    against the NumPy V-cycle on the same hierarchy."""
    torch = _torch()
    case = _uniform_case(150, 131, int(np.pi / (4.0 / 150)))
    sim = _sim(pkg, case, poisson_precond=pkg.IBM_PRECOND_SCHUR, precision=pkg.IBM_PREC_MIXED,
               amg_sweeps0=sweeps0)
    L = sim.amg_levels()
    As = [csr(*sim.amg_matrix(l, 0)) for l in range(L)]
    Ps = [csr(*sim.amg_matrix(l, 1)) for l in range(L - 1)]
    om = [sim.amg_level_info(l)[1] for l in range(L)]
    nc = case.nx * case.ny
    r = np.random.default_rng(13 + sweeps0).standard_normal(sim.n_lambda)
    z = sim.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()[:nc]
    zr = vcycle(As, Ps, om, r[:nc], pre0=sweeps0, post0=sweeps0)
    assert _rel(z, zr) < 2e-5


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_cooperative_coarse_levels_match_reference(pkg, precision, monkeypatch):
    """The coarse levels of the V-cycle as one cooperative kernel (IBM_COOP=1:
    the level-0 restriction, levels 1.. with the FP64 coarsest solve, and the
    prolongation back, phases separated by a bounded grid barrier; the small
    operators staged in shared memory) against the NumPy V-cycle, on the
    1024^2 pressure block and on the ragged coupled 150 x 131 system."""
    torch = _torch()
    monkeypatch.setenv("IBM_COOP", "1")
    prec = pkg.IBM_PREC_MIXED if precision == "mixed" else pkg.IBM_PREC_FP64
    tol = 2e-5 if precision == "mixed" else 1e-11
    for case, kw in ((W.named("cylinder_re100_1024"), dict(poisson_precond=pkg.IBM_PRECOND_SCHUR, amg_theta=0.02,
                                                           amg_max_coarse=2048, amg_sweeps0=3)),
                     (_uniform_case(150, 131, int(np.pi / (4.0 / 150))), {})):
        sim = _sim(pkg, case, precision=prec, **kw)
        L = sim.amg_levels()
        As = [csr(*sim.amg_matrix(l, 0)) for l in range(L)]
        Ps = [csr(*sim.amg_matrix(l, 1)) for l in range(L - 1)]
        om = [sim.amg_level_info(l)[1] for l in range(L)]
        n0 = As[0].shape[0]
        r = np.random.default_rng(17).standard_normal(sim.n_lambda)
        z = sim.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()[:n0]
        # amg_sweeps0 sets the finest level's sweeps of the FP32 pressure-block
        # V-cycle only; in FP64 the finest level takes amg_pre / amg_post
        s0 = kw.get("amg_sweeps0") if precision == "mixed" else None
        zr = vcycle(As, Ps, om, r[:n0], pre0=s0, post0=s0)
        assert _rel(z, zr) < tol
        sim.close()


# ----------------------------------------------------------------------------
# Poisson solve (Eq. 9b) against the direct solve
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("precond,mixed", [(1, False), (2, False), (2, True), (3, False), (3, True)])
def test_poisson_solve_matches_direct(pkg, precond, mixed):
    torch = _torch()
    case = W.cylinder_re40_128()
    o = Oracle(case)
    o.step()
    rhs = o.last_solve["rhs2"]
    # diagonal PCG cannot reach 1e-12 in the true residual on this system
    # (attainable accuracy ~ eps * cond); it is checked at 1e-10
    tol = 1e-10 if precond == 1 else 1e-12
    sim = _sim(pkg, case, poisson_precond=precond, precision=pkg.IBM_PREC_MIXED if mixed else pkg.IBM_PREC_FP64,
               tol2=tol)
    lam, st = sim.solve_poisson(torch.tensor(rhs, device="cuda"))
    assert st["status"] == 0 and st["rel_res"] <= 2 * tol
    assert _rel(lam.cpu().numpy(), o.lam) < TOL_PARITY


@pytest.mark.parametrize("mixed", [False, True])
def test_schur_preconditioner_iterations(pkg, mixed):
    """The Schur block preconditioner (S^-1 formed on the device by Gauss-Jordan)
    keeps the Poisson solve from zero to 1e-10 within a few dozen iterations on
    the 128^2 workload; a wrong S^-1 costs hundreds."""
    torch = _torch()
    case = W.cylinder_re40_128()
    o = Oracle(case)
    o.step()
    rhs = o.last_solve["rhs2"]
    sim = _sim(pkg, case, poisson_precond=pkg.IBM_PRECOND_SCHUR,
               precision=pkg.IBM_PREC_MIXED if mixed else pkg.IBM_PREC_FP64, tol2=1e-10)
    lam, st = sim.solve_poisson(torch.tensor(rhs, device="cuda"))
    print("schur iterations", st["iters"])
    assert st["status"] == 0 and st["iters"] <= 60
    assert _rel(lam.cpu().numpy(), o.lam) < TOL_PARITY


def test_mixed_schur_solve_on_more_tiles_than_blocks(pkg):
    """The temporally blocked finest level loops over its tiles when a grid has
    more of them than one launch has blocks (at most 2048; the 2048^2 workload
    has 36 x 64 = 2304 tiles of 58 x 32 cells), and the post-sweep kernel's
    dot products then stay within their partial-sum slots.  The mixed Schur
    solve there converges like the FP64 one, to the same answer."""
    torch = _torch()
    case = W.named("cylinder_re200_2048")
    rhs = np.random.default_rng(5).standard_normal(case.nx * case.ny + 2 * case.n_b)
    kw = dict(poisson_precond=pkg.IBM_PRECOND_SCHUR, amg_theta=0.02, amg_max_coarse=2048, amg_sweeps0=3,
              amg_omega=0.85, tol2=1e-10)
    lam, st = {}, {}
    for mixed in (False, True):
        sim = _sim(pkg, case, precision=pkg.IBM_PREC_MIXED if mixed else pkg.IBM_PREC_FP64, **kw)
        assert sim.n_lambda == rhs.size
        z, s = sim.solve_poisson(torch.tensor(rhs, device="cuda"))
        lam[mixed], st[mixed] = z.cpu().numpy(), s
        sim.close()
    print("iterations fp64 / mixed", st[False]["iters"], st[True]["iters"])
    for m in (False, True):
        assert st[m]["status"] == 0 and st[m]["rel_res"] <= 2e-10
        assert np.all(np.isfinite(lam[m]))
    assert st[True]["iters"] <= st[False]["iters"] + 3
    assert _rel(lam[True], lam[False]) < 1e-6


def test_poisson_solve_reports_non_convergence(pkg):
    torch = _torch()
    case = W.cylinder_re40_128()
    o = Oracle(case)
    o.step()
    sim = _sim(pkg, case, tol2=1e-14, max_iter2=3)
    lam, st = sim.solve_poisson(torch.tensor(o.last_solve["rhs2"], device="cuda"))
    assert st["status"] == 4 and st["iters"] == 3


def test_zero_rhs_gives_zero(pkg):
    torch = _torch()
    case = W.cylinder_re40_128()
    sim = _sim(pkg, case)
    lam, st = sim.solve_poisson(torch.zeros(sim.n_lambda, dtype=torch.float64, device="cuda"),
                                torch.ones(sim.n_lambda, dtype=torch.float64, device="cuda"))
    assert st["status"] == 0 and float(lam.abs().max()) == 0.0


# ----------------------------------------------------------------------------
# full time steps
# ----------------------------------------------------------------------------
def test_one_step_parity_cylinder_128(pkg):
    case = W.cylinder_re40_128()
    sim = _sim(pkg, case)
    o = Oracle(case)
    st, so = _step_both(sim, o, case)
    _compare_state(sim, o)
    assert abs(st["cd"] - so.cd) <= TOL_PARITY * abs(so.cd)
    assert abs(st["cl"] - so.cl) <= TOL_PARITY * abs(so.cd)


def test_trajectory_parity_cylinder_128_50_steps(pkg):
    """The 128^2 Re 40 workload: 50 steps with both solves at 1e-12."""
    case = W.cylinder_re40_128()
    sim = _sim(pkg, case)
    o = Oracle(case)
    worst = 0.0
    for _ in range(case.nsteps):
        st, so = _step_both(sim, o, case)
        worst = max(worst, abs(st["cd"] - so.cd) / abs(so.cd))
    eu, ev, el = _compare_state(sim, o)
    assert worst < TOL_PARITY, worst


def test_trajectory_at_paper_tolerance_is_bounded(pkg):
    """At the 1e-8 solver tolerance the 50-step C_d trajectory stays within
    1e-6 relative of the direct-solve oracle (stated bound for the iterative
    path at its production tolerance)."""
    case = W.cylinder_re40_128()
    sim = _sim(pkg, case, tol1=1e-8, tol2=1e-8)
    o = Oracle(case)
    worst = 0.0
    for _ in range(case.nsteps):
        st, so = _step_both(sim, o, case)
        worst = max(worst, abs(st["cd"] - so.cd) / abs(so.cd))
    assert worst < 1e-6, worst


# Stated per-step bounds of the production configuration (FP32 V-cycle inside
# FP64 flexible CG, Schur block preconditioner, extrapolated warm start, both
# solves to 1e-8) against the oracle's direct-solve trajectory of the 128^2
# Re 40 workload.  Solves stopped at a relative residual of 1e-8 leave errors
# up to cond x 1e-8; the same configuration with an FP64 V-cycle is run beside
# it, and the reduced-precision bound is on the difference of the two
# trajectories (measured: the two deviations from the oracle agree to four
# digits, so the deviation comes from the tolerances, not from FP32).
PROD_LAMBDA_BOUND = 1e-4     # ||phi - phi_o|| / ||phi_o|| and ||f - f_o|| / ||f_o||, every step
PROD_FORCE_BOUND = 1e-6      # |C_d - C_d,o| / |C_d,o| and |C_l - C_l,o| / |C_d,o|
PROD_MIXED_VS_FP64 = 1e-6    # ||lambda_mixed - lambda_fp64|| / ||lambda_fp64||, every step
PROD_CONSTRAINT = 2e-8       # div_max, slip_max <= this x ||rhs of Eq. 9b||_2 (the Poisson tolerance)


def _production_trajectory(pkg, case, precision):
    sim = _sim(pkg, case, tol1=1e-8, tol2=1e-8, precision=precision,
               poisson_precond=pkg.IBM_PRECOND_SCHUR, warm=pkg.IBM_WARM_EXTRAP)
    o = Oracle(case)
    nc = case.nx * case.ny
    dev = {"phi": [], "f": [], "cd": [], "cl": [], "div": [], "slip": [], "lam": []}
    for _ in range(case.nsteps):
        st, so = _step_both(sim, o, case)
        assert st["solve1"]["status"] == 0 and st["solve2"]["status"] == 0
        lam = sim.get_state()["lambda"]
        dev["lam"].append(lam)
        dev["phi"].append(float(np.linalg.norm(lam[:nc] - o.lam[:nc]) / np.linalg.norm(o.lam[:nc])))
        dev["f"].append(float(np.linalg.norm(lam[nc:] - o.lam[nc:]) / np.linalg.norm(o.lam[nc:])))
        dev["cd"].append(abs(st["cd"] - so.cd) / abs(so.cd))
        dev["cl"].append(abs(st["cl"] - so.cl) / abs(so.cd))
        bn = float(np.linalg.norm(o.last_solve["rhs2"]))
        dev["div"].append(st["div_max"] / bn)
        dev["slip"].append(st["slip_max"] / bn)
    sim.close()
    return {k: np.array(v) for k, v in dev.items()}


def test_production_config_trajectory_bound(pkg):
    """The production configuration over the 50 steps of the 128^2 workload,
    stepped beside the oracle from the same state: per step the relative
    deviations of phi and of the point forces, and those of C_d and C_l, stay
    within the stated bounds; the FP32 V-cycle's trajectory stays within the
    stated bound of the FP64 V-cycle's; the FP64 device check of the
    continuity and no-slip rows (Eq. 8) stays within the Poisson tolerance
    times ||rhs||."""
    case = W.cylinder_re40_128()
    mixed = _production_trajectory(pkg, case, pkg.IBM_PREC_MIXED)
    fp64 = _production_trajectory(pkg, case, pkg.IBM_PREC_FP64)
    mvf = np.array([np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(mixed["lam"], fp64["lam"])])
    for name, d in (("mixed", mixed), ("fp64", fp64)):
        print(f"production config ({name}), 50 steps: max phi dev {d['phi'].max():.3e}, "
              f"max f dev {d['f'].max():.3e}, max C_d dev {d['cd'].max():.3e}, max C_l dev {d['cl'].max():.3e}, "
              f"max div/||b|| {d['div'].max():.3e}, max slip/||b|| {d['slip'].max():.3e}")
    print(f"production config: max ||lambda_mixed - lambda_fp64|| / ||lambda_fp64|| {mvf.max():.3e}")
    d = mixed
    assert d["phi"].max() < PROD_LAMBDA_BOUND and d["f"].max() < PROD_LAMBDA_BOUND, (d["phi"], d["f"])
    assert d["cd"].max() < PROD_FORCE_BOUND and d["cl"].max() < PROD_FORCE_BOUND, (d["cd"], d["cl"])
    assert mvf.max() < PROD_MIXED_VS_FP64, mvf
    assert d["div"].max() < PROD_CONSTRAINT and d["slip"].max() < PROD_CONSTRAINT, (d["div"], d["slip"])
    assert d["div"].min() > 0.0 and d["slip"].min() > 0.0   # the check ran


def test_projection_warm_start_keeps_the_solution(pkg):
    """IBM_WARM_PROJ starts the Poisson solve from the K-norm projection of the
    solution onto the span of up to 24 previous solutions (K = Q^T B Q).
    It changes only where the solve starts: 30 steps of the 128^2 Re 40
    workload in the production configuration (FP32 V-cycle, Schur block
    preconditioner) match the oracle's steps to 1e-8 while the basis fills up
    and starts over, and from the fourth step on the solve starts closer to
    the solution, and takes fewer iterations, than from the extrapolated
    guess."""
    case = W.cylinder_re40_128()
    kw = dict(poisson_precond=pkg.IBM_PRECOND_SCHUR, precision=pkg.IBM_PREC_MIXED)
    stats = {}
    for warm in (pkg.IBM_WARM_PROJ, pkg.IBM_WARM_EXTRAP):
        sim = _sim(pkg, case, warm=warm, **kw)
        o = Oracle(case) if warm == pkg.IBM_WARM_PROJ else None
        st = []
        for _ in range(30):
            if o is not None:
                a, so = _step_both(sim, o, case)
                assert abs(a["cd"] - so.cd) <= TOL_PARITY * abs(so.cd)
            else:
                xb, yb, ub, vb = case.body_state(sim.get_state()["t"] + case.dt)
                sim.set_body(xb, yb, ub, vb)
                a = sim.step(1)[0]
            assert a["solve1"]["status"] == 0 and a["solve2"]["status"] == 0
            st.append((a["solve1"], a["solve2"]))
        if o is not None:
            _compare_state(sim, o)
        stats[warm] = st
        sim.close()
    P, E = stats[pkg.IBM_WARM_PROJ][3:], stats[pkg.IBM_WARM_EXTRAP][3:]
    r_p, r_e = (np.mean([s[1]["rel_res0"] for s in X]) for X in (P, E))
    k_p, k_e = (np.mean([s[1]["iters"] for s in X]) for X in (P, E))
    print(f"projection: rel_res0 {r_p:.3e}, k2 {k_p:.2f}; extrapolation: rel_res0 {r_e:.3e}, k2 {k_e:.2f}")
    assert r_p < r_e and k_p < k_e


def test_constraint_check_matches_oracle_operators(pkg):
    """The device's FP64 constraint maxima after a step equal the maxima of
    |G^T q + bc2| (unpinned cells) and |E q - u_B| formed on the host with the
    oracle's operators from the state the library returns."""
    from oracle import divergence_full
    from oracle.ibpm import interpolation_E
    case = W.cylinder_re40_128()
    sim = _sim(pkg, case, tol1=1e-8, tol2=1e-8)
    o = Oracle(case, factorize=False)
    for _ in range(2):
        xb, yb, ub, vb = case.body_state(sim.get_state()["t"] + case.dt)
        sim.set_body(xb, yb, ub, vb)
        st = sim.step(1)[0]
    s = sim.get_state()
    g = o.g
    q1 = g.q_from_uv(s["u"], s["v"])
    b1 = o.bnd.copy()
    b1.u_right = s["u"][:, -1]
    div = np.delete(divergence_full(g, q1, b1), o.p0)
    E = interpolation_E(g, xb, yb, o.h)
    slip = E @ q1 - np.concatenate([ub, vb])
    assert abs(st["div_max"] - np.abs(div).max()) <= 1e-12 * max(np.abs(q1).max(), 1.0)
    assert abs(st["slip_max"] - np.abs(slip).max()) <= 1e-12 * max(np.abs(q1).max(), 1.0)


@pytest.mark.parametrize("mixed", [False, True])
def test_ragged_grid_steps(pkg, mixed):
    case = _uniform_case(150, 131, int(np.pi / (4.0 / 150)))
    sim = _sim(pkg, case, precision=pkg.IBM_PREC_MIXED if mixed else pkg.IBM_PREC_FP64)
    o = Oracle(case)
    for _ in range(3):
        _step_both(sim, o, case)
    _compare_state(sim, o)


def test_moving_body_parity(pkg):
    case = _uniform_case(96, 96, int(np.pi / (4.0 / 96)), moving=True, dt=0.01, re=100.0)
    sim = _sim(pkg, case, amg_rebuild_every=1, moving=1)
    o = Oracle(case)
    for _ in range(4):
        st, so = _step_both(sim, o, case)
        assert abs(st["cl"] - so.cl) <= TOL_PARITY * max(abs(so.cl), abs(so.cd))
    _compare_state(sim, o)


@pytest.mark.parametrize("N,mixed", [(3, False), (3, True), (2, False)])
def test_bn_steps_parity(pkg, N, mixed):
    """B^N with N > 1 (section 2; Table 2's higher-order columns) on a ragged
    grid with a body: the library's assembled Q^T B^N Q against the oracle's
    operator, then three steps (AMG-preconditioned solve on that operator and
    the N-term projection of Eq. 9c) against the oracle's direct steps."""
    torch = _torch()
    case = _uniform_case(150, 131, int(np.pi / (4.0 / 150)))
    sim = _sim(pkg, case, bn_order=N, precision=pkg.IBM_PREC_MIXED if mixed else pkg.IBM_PREC_FP64)
    ob = Oracle(case, factorize=False, bn_order=N)
    xb, yb, _, _ = case.body_state(case.dt)
    ob.build_poisson(xb, yb, factorize=False)
    x = np.random.default_rng(5).standard_normal(ob.S.shape[0])
    y = sim.apply_poisson(torch.tensor(x, device="cuda")).cpu().numpy()
    assert _rel(y, ob.S @ x) < 1e-13
    o = Oracle(case, bn_order=N)
    for _ in range(3):
        st, so = _step_both(sim, o, case)
        assert st["solve2"]["status"] == 0 and st["solve1"]["status"] == 0
    _compare_state(sim, o)


@pytest.mark.parametrize("N,mixed", [(3, False), (3, True), (2, True)])
def test_bn_matrix_free_steps_parity(pkg, N, mixed):
    """B^N with N > 1 without assembly (section 2; Table 2's higher-order
    columns): with the Schur preconditioner the Poisson operator Q^T B^N Q is
    applied as the projection chain of Eq. 9c on x (B^1 Q x, N - 1 further
    viscous terms, then Q^T) and preconditioned by the Schur block
    preconditioner of Q^T B^1 Q.  On a ragged grid with a body: the applied
    operator against the oracle's assembled one (pinned row included) to
    1e-13, then three steps against the oracle's direct B^N steps to 1e-8."""
    torch = _torch()
    case = _uniform_case(150, 131, int(np.pi / (4.0 / 150)))
    sim = _sim(pkg, case, bn_order=N, poisson_precond=pkg.IBM_PRECOND_SCHUR,
               precision=pkg.IBM_PREC_MIXED if mixed else pkg.IBM_PREC_FP64)
    ob = Oracle(case, factorize=False, bn_order=N)
    xb, yb, _, _ = case.body_state(case.dt)
    ob.build_poisson(xb, yb, factorize=False)
    x = np.random.default_rng(5).standard_normal(ob.S.shape[0])
    y = sim.apply_poisson(torch.tensor(x, device="cuda")).cpu().numpy()
    assert _rel(y, ob.S @ x) < 1e-13, _rel(y, ob.S @ x)
    o = Oracle(case, bn_order=N)
    iters = []
    for _ in range(3):
        st, so = _step_both(sim, o, case)
        assert st["solve2"]["status"] == 0 and st["solve1"]["status"] == 0
        iters.append(st["solve2"]["iters"])
    print(f"B^{N} matrix-free, Schur(B^1) preconditioner: Poisson iterations {iters}")
    _compare_state(sim, o)


def test_re40_impulsive_cylinder_drag(pkg):
    """Section 5.2 on Table 3's 330^2 grid: 6000 steps (t = 60) of the
    impulsively started cylinder at Re 40 against the oracle's drag history
    (golden/re40_drag_330.txt, written by golden/make_re40_drag.py from the
    oracle), and the steady drag against the printed 1.57."""
    import pathlib
    case = W.cylinder_impulsive_re40_330()
    ref = np.loadtxt(pathlib.Path(__file__).parent / "golden" / "re40_drag_330.txt")
    sim = _sim(pkg, case, tol1=1e-10, tol2=1e-10, poisson_precond=pkg.IBM_PRECOND_SCHUR)
    st = sim.step(case.nsteps)
    assert all(s["solve1"]["status"] == 0 and s["solve2"]["status"] == 0 for s in st)
    cd = np.array([s["cd"] for s in st])[49::50]
    assert cd.shape == ref[:, 1].shape
    rel = np.abs(cd - ref[:, 1]) / np.abs(ref[:, 1])
    assert rel.max() < 1e-6, rel.max()
    assert abs(cd[-1] - 1.57) < 0.01 * 1.57


def test_couette_walls_parity(pkg):
    case = W.couette(48, 0.01, 3)
    sim = _sim(pkg, case)
    o = Oracle(case)
    for _ in range(3):
        _step_both(sim, o, case)
    _compare_state(sim, o)


def test_body_free_jacobi_parity(pkg):
    case = _uniform_case(64, 80, 0)
    sim = _sim(pkg, case, poisson_precond=1, tol2=1e-11)
    o = Oracle(case)
    for _ in range(2):
        _step_both(sim, o, case)
    _compare_state(sim, o)


def test_state_roundtrip_and_resume(pkg):
    case = W.cylinder_re40_128()
    sim = _sim(pkg, case)
    sim.step(2)
    s = sim.get_state()
    sim2 = _sim(pkg, case)
    sim2.set_state(u=s["u"], v=s["v"], v_right=s["v_right"], nprev=s["nprev"], lam=s["lambda"], t=s["t"],
                   step=s["step"])
    a = sim.step(1)[0]
    b = sim2.step(1)[0]
    assert a["cd"] == b["cd"] and a["solve2"]["iters"] == b["solve2"]["iters"]
    sa, sb = sim.get_state(), sim2.get_state()
    assert np.array_equal(sa["u"], sb["u"]) and np.array_equal(sa["v"], sb["v"])


def test_bad_body_velocity_is_rejected(pkg):
    case = W.cylinder_re40_128()
    sim = _sim(pkg, case)
    xb, yb, ub, vb = case.body_state(0.0)
    ub = ub.copy()
    ub[3] = np.nan
    with pytest.raises(pkg.IbmError) as e:
        sim.set_body(xb, yb, ub, vb)
    assert e.value.code == 1


# ----------------------------------------------------------------------------
# Schur-complement block preconditioner (pressure-block V-cycle + dense S)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("mixed", [False, True])
def test_schur_pressure_vcycle_matches_reference(pkg, mixed):
    torch = _torch()
    case = W.cylinder_re40_128()
    sim = _sim(pkg, case, poisson_precond=pkg.IBM_PRECOND_SCHUR,
               precision=pkg.IBM_PREC_MIXED if mixed else pkg.IBM_PREC_FP64)
    L = sim.amg_levels()
    As = [csr(*sim.amg_matrix(l, 0)) for l in range(L)]
    Ps = [csr(*sim.amg_matrix(l, 1)) for l in range(L - 1)]
    om = [sim.amg_level_info(l)[1] for l in range(L)]
    assert As[0].shape[0] == case.nx * case.ny   # pressure block only
    r = np.random.default_rng(9).standard_normal(sim.n_lambda)
    z = sim.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()[:case.nx * case.ny]
    zr = vcycle(As, Ps, om, r[:case.nx * case.ny])
    assert _rel(z, zr) < (2e-5 if mixed else 1e-11)


@pytest.mark.parametrize("mixed", [False, True])
def test_schur_steps_parity(pkg, mixed):
    case = _uniform_case(150, 131, int(np.pi / (4.0 / 150)))
    sim = _sim(pkg, case, poisson_precond=pkg.IBM_PRECOND_SCHUR,
               precision=pkg.IBM_PREC_MIXED if mixed else pkg.IBM_PREC_FP64)
    o = Oracle(case)
    for _ in range(3):
        st, so = _step_both(sim, o, case)
        assert st["solve2"]["status"] == 0
        assert abs(st["cd"] - so.cd) <= TOL_PARITY * abs(so.cd)
    _compare_state(sim, o)


@pytest.mark.parametrize("every", [1, 3])
def test_schur_moving_body_parity(pkg, every):
    case = _uniform_case(96, 96, int(np.pi / (4.0 / 96)), moving=True, dt=0.01, re=100.0)
    sim = _sim(pkg, case, poisson_precond=pkg.IBM_PRECOND_SCHUR, amg_rebuild_every=every, moving=1,
               precision=pkg.IBM_PREC_MIXED)
    o = Oracle(case)
    rebuilt = 0
    for _ in range(4):
        st, so = _step_both(sim, o, case)
        rebuilt += st["amg_rebuilt"]
        assert abs(st["cl"] - so.cl) <= TOL_PARITY * max(abs(so.cl), abs(so.cd))
    _compare_state(sim, o)
    # S is built at the first solve, then after every `every` steps of motion
    assert rebuilt == (4 if every == 1 else 2)


def _small_flapping_case(n_b=51):
    """Section 6.2's airfoil and kinematics (translation along x and rotation
    about its centre, fluid at rest) on a small uniform grid."""
    xf = W.uniform_faces(125, -2.5, 2.5)
    yf = W.uniform_faces(50, -1.0, 1.0)
    body = W.FlappingEllipse(n_b)
    return W.Case("flap_small", xf, yf, [body], nu=body.max_speed / 75.0, dt=0.004, nsteps=4,
                  uinf=0.0, vinf=0.0, h=0.04)


@pytest.mark.parametrize("variant", ["schur_mixed", "coupled_fp64"])
def test_flapping_airfoil_steps_parity(pkg, variant):
    """The flapping airfoil of section 6.2 (rotating and translating ellipse
    in fluid at rest) through the CUDA path: body rows of every step formed on
    the device (Schur preconditioner, FP32 V-cycle) or on the host (coupled
    smoothed aggregation rebuilt every step, FP64), four steps against the
    oracle's direct steps, lift and drag to 1e-8 and the final state to 1e-8;
    the device check of the constraints of Eq. 8 at every step."""
    case = _small_flapping_case()
    kw = (dict(poisson_precond=pkg.IBM_PRECOND_SCHUR, precision=pkg.IBM_PREC_MIXED)
          if variant == "schur_mixed" else dict(precision=pkg.IBM_PREC_FP64))
    sim = _sim(pkg, case, amg_rebuild_every=1, moving=1, **kw)
    o = Oracle(case)
    for _ in range(4):
        st, so = _step_both(sim, o, case)
        scale = max(abs(so.cl), abs(so.cd))
        assert abs(st["cl"] - so.cl) <= TOL_PARITY * scale and abs(st["cd"] - so.cd) <= TOL_PARITY * scale
        assert st["div_max"] < 1e-9 and st["slip_max"] < 1e-9, st
    _compare_state(sim, o)
    sim.close()


def test_schur_cache_matches_direct_build(pkg):
    """Moving body: S rebuilt every step from the cache of V-cycle responses
    (one V-cycle per newly touched cell) against building it from 2 n_b
    V-cycles: the same state to 1e-8 (both solves stop at 1e-12) and iteration
    counts of the same size.  The two complements agree only to FP32 rounding
    of the V-cycle outputs, and at this scale the counts move by several
    iterations under rounding-level changes (measured pairs: 25/33/24/29/23/29
    against 31/33/30/29/29/29, and 25/33/30/29/29/29 against 25/33/30/29/28/23)."""
    case = _uniform_case(96, 96, int(np.pi / (4.0 / 96)), moving=True, dt=0.01, re=100.0)
    runs = {}
    for cache in (-1, 0):
        sim = _sim(pkg, case, poisson_precond=pkg.IBM_PRECOND_SCHUR, amg_rebuild_every=1, moving=1,
                   precision=pkg.IBM_PREC_MIXED, schur_cache=cache)
        its, t = [], 0.0
        for _ in range(6):
            xb, yb, ub, vb = case.body_state(t + case.dt)
            sim.set_body(xb, yb, ub, vb)
            st = sim.step(1)[0]
            its.append(st["solve2"]["iters"])
            t += case.dt
        runs[cache] = (its, sim.get_state())
        sim.close()
    (ia, sa), (ib, sb) = runs[-1], runs[0]
    assert max(ia) <= max(ib) + 8 and sum(ia) <= 1.2 * sum(ib), (ia, ib)
    for key in ("u", "v", "lambda"):
        assert _rel(sa[key], sb[key]) < TOL_PARITY


def test_full_size_step_satisfies_discrete_equations(pkg):
    """1024^2 stretched workload, production configuration (FP32 V-cycle in
    FP64 flexible CG with the Schur preconditioner, tolerance 1e-8): one step
    checked through the oracle's operators (no direct solve at this size):
    the divergence and no-slip constraints, Eq. 9a and Eq. 9b residuals."""
    case = W.named("cylinder_re100_1024")
    sim = _sim(pkg, case, tol1=1e-8, tol2=1e-8, poisson_precond=pkg.IBM_PRECOND_SCHUR,
               precision=pkg.IBM_PREC_MIXED)
    o = Oracle(case, factorize=False)
    r1, b_n1, (xb, yb, ub, vb), _ = o.explicit_terms()
    o.build_poisson(xb, yb, factorize=False)
    sim.set_body(xb, yb, ub, vb)
    st = sim.step(1)[0]
    assert st["solve1"]["status"] == 0 and st["solve2"]["status"] == 0
    s = sim.get_state()
    g = o.g
    q1 = g.q_from_uv(s["u"], s["v"])
    lam = s["lambda"]
    from oracle import divergence_full
    b1 = o.bnd.copy()
    b1.u_right = s["u"][:, -1]
    div = divergence_full(g, q1, b1)
    slip = o.E @ q1 - np.concatenate([ub, vb])
    # Eq. 9c inverted: q* = q^{n+1} + B Q lambda; Eq. 9a residual
    qs = q1 + o.Bdiag * (o.Q @ lam)
    # Eq. 9b right-hand side built from q*; after the projection the divergence
    # and slip rows equal the Poisson residual, bounded by tol * ||rhs||.  The
    # pinned cell's row is replaced by phi(p0) = 0, so its divergence collects
    # the residual sum and is checked against the absolute tolerance only.
    rhs = np.concatenate([-divergence_full(g, qs, b1), o.E @ qs - np.concatenate([ub, vb])])
    rhs[o.p0] = 0.0
    bn = np.linalg.norm(rhs)
    d_other = np.delete(div, o.p0)
    assert np.abs(d_other).max() <= 2e-8 * bn
    assert abs(div[o.p0]) <= 1e-6 * bn
    assert np.abs(slip).max() <= 2e-8 * bn
    res1 = np.linalg.norm(o.A @ qs - r1) / np.linalg.norm(r1)
    assert res1 < 1e-7, res1
    # Eq. 9b residual on the pinned system
    res2 = np.linalg.norm(o.S @ lam - rhs) / np.linalg.norm(rhs)
    assert res2 < 1e-7, res2
