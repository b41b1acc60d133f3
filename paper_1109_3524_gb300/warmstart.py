"""Training of the warm-start U-Net on snapshots of the solver itself, and
measurement of what it gains.

A sample predicts the error phi^{n+1} - (2 phi^n - phi^{n-1}) of the
extrapolated warm start from (phi^n, phi^{n-1}, the residual of the
extrapolated guess in step n+1); the library standardises inputs and targets
(ibm_cnn_prepare) and trains with its own forward/backward kernels and Adam.  The split is by time:
the first part of a run trains, the steps after it evaluate.
"""
from __future__ import annotations

import time

import numpy as np

from . import _abi as A
from .sim import Sim, Unet


def generate_snapshots(case, nsteps, device="cuda:0", skip=2, **cfg):
    """Runs `nsteps` steps with the extrapolated warm start and returns
    (phi, r0, state, t): device tensors (nsteps, nx*ny) of lambda's pressure
    part after each step and of the residual of that step's extrapolated
    guess, the final state and time."""
    import torch
    cfg.setdefault("poisson_precond", A.IBM_PRECOND_SCHUR)
    cfg.setdefault("precision", A.IBM_PREC_MIXED)
    cfg["warm"] = A.IBM_WARM_EXTRAP
    sim = Sim.from_case(case, device=device, **cfg)
    U0, V0 = case.initial_velocity()
    sim.set_state(u=U0, v=V0, v_right=np.full(case.ny + 1, case.vinf))
    nc = case.nx * case.ny
    phi = torch.empty((nsteps, nc), dtype=torch.float64, device=device)
    rhs = torch.empty_like(phi)
    sim.snapshot()   # starts recording the residual of the extrapolated guess
    t = 0.0
    for n in range(nsteps + skip):
        xb, yb, ub, vb = case.body_state(t + case.dt)
        if case.n_b:
            sim.set_body(xb, yb, ub, vb)
        sim.step(1)
        t += case.dt
        if n >= skip:
            lam, _, _, r0 = sim.snapshot()
            phi[n - skip] = lam[:nc]
            rhs[n - skip] = r0[:nc]
    state = sim.get_state()
    sim.close()
    return phi, rhs, state, t


def train(net: Unet, phi, r0, nx, ny, steps=300, batch=8, crop=128, lr=2e-3, seed=0, log_every=0):
    """Adam on random crops of samples n = 1 .. len-2 (inputs phi[n], phi[n-1],
    r0[n+1]; target phi[n+1]).  phi and r0 may be lists of runs (a sample
    never spans two runs).  Returns the loss history."""
    rng = np.random.default_rng(seed)
    runs = list(zip(phi, r0)) if isinstance(phi, (list, tuple)) else [(phi, r0)]
    hist = []
    for it in range(steps):
        ph, rr = runs[int(rng.integers(0, len(runs)))]
        n = int(rng.integers(1, ph.shape[0] - 1))
        ch, cw = min(crop, ny), min(crop, nx)
        xy = np.stack([rng.integers(0, nx - cw + 1, batch), rng.integers(0, ny - ch + 1, batch)], axis=1)
        x, tgt = net.prepare(nx, ny, ph[n], ph[n - 1], rr[n + 1], ph[n + 1], xy, ch, cw)
        loss, _ = net.loss_grad(x, tgt)
        net.adam_step(lr)
        hist.append(loss)
        if log_every and it % log_every == 0:
            print(f"[train] step {it} loss {loss:.4e}", flush=True)
    return hist


def prediction_error(net: Unet, phi, r0, nx, ny, samples):
    """Mean of |error of the warm start with the network| / |error of the
    extrapolation alone| over the given samples (below 1: the network helps)."""
    import torch
    ratios = []
    for n in samples:
        x, tgt = net.prepare(nx, ny, phi[n], phi[n - 1], r0[n + 1], phi[n + 1], np.array([[0, 0]]), ny, nx)
        y = net.forward(x)[0].double().reshape(-1)
        t = tgt[0].double().reshape(-1)
        ratios.append(float(torch.linalg.norm(t - y) / torch.linalg.norm(t).clamp_min(1e-300)))
    return float(np.mean(ratios))


def compare_iterations(case, net: Unet, state, t0, nsteps, device="cuda:0", **cfg):
    """Poisson iterations per step from the same state with the previous
    lambda, the extrapolation and the learned warm start."""
    cfg.setdefault("poisson_precond", A.IBM_PRECOND_SCHUR)
    cfg.setdefault("precision", A.IBM_PREC_MIXED)
    out = {}
    for name, warm in (("prev", A.IBM_WARM_PREV), ("extrap", A.IBM_WARM_EXTRAP), ("cnn", A.IBM_WARM_CNN)):
        sim = Sim.from_case(case, device=device, warm=warm, **cfg)
        if warm == A.IBM_WARM_CNN:
            sim.attach_cnn(net)
        sim.set_state(u=state["u"], v=state["v"], v_right=state["v_right"], nprev=state["nprev"],
                      lam=state["lambda"], t=t0, step=state["step"])
        t = t0
        its, r0 = [], []
        tic = time.perf_counter()
        for _ in range(nsteps):
            xb, yb, ub, vb = case.body_state(t + case.dt)
            if case.n_b:
                sim.set_body(xb, yb, ub, vb)
            st = sim.step(1)[0]
            t += case.dt
            its.append(st["solve2"]["iters"])
            r0.append(st["solve2"]["rel_res0"])
        import torch
        torch.cuda.synchronize()
        el = time.perf_counter() - tic
        # the first two steps rebuild lambda^{n-1} and do not extrapolate
        out[name] = {"k2_mean": float(np.mean(its[2:])), "rel_res0_mean": float(np.mean(r0[2:])),
                     "steps_per_s": nsteps / el}
        sim.close()
    return out
