#!/usr/bin/env python
"""Benchmark of the immersed-boundary projection step on GB300.

One step = one time step of the method (explicit right-hand side, velocity
solve Eq. 9a, Poisson solve Eq. 9b, projection Eq. 9c, forces) on the
1024^2 stretched-grid cylinder workload (Re 100, 630 body points).  Prints
one JSON line (rank 0).  `--impl reference` times the CPU oracle instead.

Multi-GPU: the path is run as independent replicas (one per rank); the value
is the steps of all replicas divided by the slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time steps/s and Poisson GB/s (% HBM roofline), learned+mixed vs plain FP64 AMG-PCG"
WORKLOAD = "cylinder_re100_1024"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-kernel-profile", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned warm-start variant")
    ap.add_argument("--no-moving", action="store_true", help="skip the moving-body workload")
    ap.add_argument("--snapshots", type=int, default=200, help="solver snapshots per training run")
    ap.add_argument("--train-re", type=float, nargs="+", default=[90.0, 110.0],
                    help="Reynolds numbers of the training runs (same grid and body; not the timed flow)")
    ap.add_argument("--train-steps", type=int, default=1200, help="Adam steps of the U-Net")
    ap.add_argument("--cnn-window", type=int, nargs=2, default=[512, 256], metavar=("W", "H"),
                    help="inference window (cells) of the learned warm start around the body; 0 0: whole grid")
    ap.add_argument("--trunc", type=float, default=0.1, help="AMG prolongator truncation")
    ap.add_argument("--profile-out", default=None, help="write the per-kernel profile (JSON) here")
    ap.add_argument("--poisson-micro", action="store_true",
                    help="instead of the step benchmark: Poisson solves to 1e-5 with CG, Jacobi-PCG and "
                         "SA-AMG-PCG on 5-point systems and the four Table 1 systems (one JSON line each)")
    ap.add_argument("--micro-sizes", type=int, nargs="+", default=[50, 100, 200, 400, 700, 1000, 1400, 2000],
                    help="grid sides of the body-free 5-point systems (2500 .. 4e6 unknowns)")
    ap.add_argument("--micro-systems", type=int, nargs="*", default=[1, 2, 3, 4], help="Table 1 systems")
    ap.add_argument("--micro-out", default=None, help="also append the lines to this file")
    return ap.parse_args()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v, device=None):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.idx = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                rows.append((float(f[0]), float(f[1]), f[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def make_sim(P, case, device, **kw):
    import numpy as np
    sim = P.Sim.from_case(case, device=device, **kw)
    U0, V0 = case.initial_velocity()
    sim.set_state(u=U0, v=V0, v_right=np.full(case.ny + 1, case.vinf), t=0.0, step=0)
    return sim


def run_variant(P, case, device, steps, warmup, ws, kernel_profile=True, setup=None, **kw):
    """Device-timed steps (CUDA events on the library's stream), then a second
    pass with per-kernel events for the roofline."""
    import torch
    sim = make_sim(P, case, device, **kw)
    if setup is not None:
        setup(sim)
    body = case.body_state
    t = 0.0

    def advance(n):
        nonlocal t
        out = []
        for _ in range(n):
            xb, yb, ub, vb = body(t + case.dt)
            if case.moving:
                sim.set_body(xb, yb, ub, vb)
            out.append(sim.step(1)[0])
            t += case.dt
        return out

    advance(warmup)
    print(f"[bench] launches before the timed region: {sim.launch_count()}", file=sys.stderr, flush=True)
    stream = sim.stream
    torch.cuda.synchronize(device)
    barrier(ws)
    l0 = sim.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    gpu_index = torch.cuda.current_device()
    with Clocks(gpu_index) as clk:
        # the profiler range brackets the timed steps (ncu --profile-from-start off)
        torch.cuda.profiler.start()
        e0.record(stream)
        stats = advance(steps)
        e1.record(stream)
        torch.cuda.synchronize(device)
        torch.cuda.profiler.stop()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    launches = sim.launch_count() - l0
    if not kernel_profile:
        return sim, stats, ms, launches, clk.summary(), {}, 0
    # profiled pass (per-kernel CUDA events on the library's stream)
    sim.profile(True)
    sim.profile_reset()
    nprof = max(3, min(steps, 20))
    advance(nprof)
    prof = sim.profile_read()
    sim.profile(False)
    return sim, stats, ms, launches, clk.summary(), prof, nprof


def poisson_classes():
    return ["pois_spmv", "pois_coupling", "pois_update", "pois_pupdate", "vc_smooth0", "vc_coupling0",
            "vc_restrict", "vc_prolong", "vc_csr", "vc_coarsest", "schur", "pw_precond"]


# DRAM bytes per launch of a kernel class from one ncu capture of the current
# kernels (profiles/ncu_level_sweeps_cylinder_re100_1024.md): mean over the class's
# launches in one step of cylinder_re100_1024 (cold cache).  Null for other classes.
NCU_TRAFFIC = {"vc_csr": 12.823e6, "vc_smooth0": 10.166e6}


def roofline(prof, peak, peak_kind):
    # dominant kernel class by device time
    k = max(prof, key=lambda n: prof[n]["ms"])
    p = prof[k]
    per_launch_ms = p["ms"] / max(p["launches"], 1)
    per_launch_bytes = p["bytes"] / max(p["launches"], 1)
    ach = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9 if per_launch_ms > 0 else 0.0
    return {"kernel": k, "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4), "traffic": NCU_TRAFFIC.get(k), "peak_source": peak_kind,
            "bytes_per_launch": per_launch_bytes, "ms_per_launch": per_launch_ms,
            "share_of_profiled_time": round(p["ms"] / sum(v["ms"] for v in prof.values()), 4)}


def e2e_run(P, case, device, steps, warmup, **kw):
    """End to end through the public API with host buffers: every step sends
    the body state from pinned host memory and reads back the step's forces
    and solver statistics."""
    import numpy as np
    import torch
    sim = make_sim(P, case, device, **kw)
    pin = [torch.empty(case.n_b, dtype=torch.float64).pin_memory() for _ in range(4)]
    t = 0.0

    def one():
        nonlocal t
        xb, yb, ub, vb = case.body_state(t + case.dt)
        for buf, a in zip(pin, (xb, yb, ub, vb)):
            buf.numpy()[:] = a
        sim.set_body(*(b.numpy() for b in pin))
        st = sim.step(1)[0]
        t += case.dt
        return st

    for _ in range(warmup):
        one()
    torch.cuda.synchronize(device)
    h0, d0 = sim.transfer_bytes()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize(device)
    el = time.perf_counter() - t0
    h1, d1 = sim.transfer_bytes()
    sim.close()
    return steps / el, (h1 - h0) / steps, (d1 - d0) / steps


def cpu_baseline(case, nsteps=3):
    """The CPU oracle (direct sparse solves, FP64) on the same workload: the
    one-time LU factorisations are timed separately; the value is steps/s over
    `nsteps` steps."""
    import numpy as np
    from oracle import Oracle
    t0 = time.perf_counter()
    o = Oracle(case)
    xb, yb, _, _ = case.body_state(case.dt)
    o.build_poisson(xb, yb)
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    for _ in range(nsteps):
        o.step()
    el = time.perf_counter() - t0
    return {"value": nsteps / el, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{case.name}: steps 1-{nsteps} after the one-time LU factorisations "
                      f"({setup:.1f} s, not in the value); SuperLU and the NumPy step run single-threaded",
            "setup_s": round(setup, 2), "host_cpus": os.cpu_count()}


def run_ours(args):
    import numpy as np
    import torch
    import workloads as W
    import paper_1109_3524_gb300 as P
    ws, rank, local = dist_setup()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    case = W.named(args.workload)
    peak, peak_kind = load_peaks()
    # pressure-block smoothed aggregation tuned on this workload: weaker strength
    # threshold (larger aggregates), dense coarsest up to 2048 unknowns, three
    # sweeps each way on the finest level, Jacobi weight 0.85 * 2 / rho(D^-1 A)
    common = dict(tol1=1e-8, tol2=1e-8, poisson_precond=P.IBM_PRECOND_SCHUR, amg_trunc=args.trunc,
                  amg_theta=0.02, amg_max_coarse=2048, amg_tail_rows=16384, amg_sweeps0=3, amg_omega=0.85)
    # headline: FP32 V-cycle inside FP64 flexible CG, extrapolated warm start
    sim, stats, ms, launches, clocks, prof, nprof = run_variant(
        P, case, device, args.steps, args.warmup, ws, kernel_profile=not args.no_kernel_profile,
        precision=P.IBM_PREC_MIXED, warm=P.IBM_WARM_EXTRAP, **common)
    ms_max = max_over_ranks(ws, ms, device)
    value = ws * args.steps / (ms_max * 1e-3)
    k1 = [s["solve1"]["iters"] for s in stats]
    k2 = [s["solve2"]["iters"] for s in stats]
    pois = {k: prof[k] for k in poisson_classes() if k in prof}
    pois_bytes = sum(v["bytes"] for v in pois.values())
    pois_ms = sum(v["ms"] for v in pois.values())
    pois_gbs = pois_bytes / (pois_ms * 1e-3) / 1e9 if pois_ms > 0 else 0.0
    roof = roofline(prof, peak, peak_kind) if prof else None
    if args.profile_out and rank == 0:
        with open(args.profile_out, "w") as f:
            json.dump({"steps": nprof, "classes": prof}, f, indent=1)
    sim.close()
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": case.name, "grid": f"{case.nx}x{case.ny} stretched 1.02 outside [-2,2]^2",
                   "domain": "[-15,15]^2", "n_b": case.n_b, "Re": round(1.0 / case.nu), "dt": case.dt,
                   "variant": "FP32 SA V-cycle (Schur block) in FP64 flexible CG, extrapolated warm start",
                   "tol": 1e-8, "parallelism": "replicas" if ws > 1 else "single GPU",
                   "l2": "working set ~0.6 GB > 129 MB L2 (no flush needed)"},
        "iters": {"k1_mean": round(float(np.mean(k1)), 2), "k2_mean": round(float(np.mean(k2)), 2),
                  "k2_max": int(max(k2))},
        "poisson": {"gbs": round(pois_gbs, 1), "frac_hbm": round(pois_gbs / peak, 4),
                    "ms_per_step": round(pois_ms / nprof, 4) if nprof else None},
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "cd_last": stats[-1]["cd"],
        # force coefficients over the timed steps; from the uniform start the
        # timed window (steps * dt time units) is far shorter than one shedding
        # period, so no Strouhal number is formed from it
        "forces": {"cd_last": stats[-1]["cd"], "cl_last": stats[-1]["cl"],
                   "cd_mean": float(np.mean([s["cd"] for s in stats])),
                   "cl_max_abs": float(np.max(np.abs([s["cl"] for s in stats]))),
                   "time_units": round(len(stats) * case.dt, 6), "strouhal": None},
    }
    if not args.no_plain:
        # plain FP64 AMG-PCG with the same preconditioner structure, warm start lambda^n
        psim, pstats, pms, _, _, pprof, pn = run_variant(
            P, case, device, args.steps, args.warmup, ws, precision=P.IBM_PREC_FP64,
            warm=P.IBM_WARM_PREV, **common)
        pms = max_over_ranks(ws, pms, device)
        ppois = {k: pprof[k] for k in poisson_classes() if k in pprof}
        pb = sum(v["bytes"] for v in ppois.values())
        pm = sum(v["ms"] for v in ppois.values())
        out["plain_fp64"] = {"value": round(ws * args.steps / (pms * 1e-3), 3), "unit": "steps/s",
                             "k2_mean": round(float(np.mean([s["solve2"]["iters"] for s in pstats])), 2),
                             "poisson_gbs": round(pb / (pm * 1e-3) / 1e9, 1) if pm > 0 else None}
        psim.close()
    if not args.no_learned:
        out["learned_mixed"] = learned_variant(P, case, device, args, ws, common)
    if not args.no_moving:
        # the moving-body path (E and the coupling rows rebuilt every step, the
        # Schur complement rebuilt every step from the cache of V-cycle responses)
        mcase = W.named("oscillating_cylinder_re100_1024")
        msteps = max(10, min(args.steps, 50))
        msim, mstats, mms, mlaunch, _, _, _ = run_variant(
            P, mcase, device, msteps, args.warmup, ws, kernel_profile=False, precision=P.IBM_PREC_MIXED,
            warm=P.IBM_WARM_EXTRAP, moving=1, amg_rebuild_every=1, **common)
        mms = max_over_ranks(ws, mms, device)
        out["moving"] = {"workload": mcase.name, "value": round(ws * msteps / (mms * 1e-3), 3), "unit": "steps/s",
                         "steps": msteps, "k2_mean": round(float(np.mean([s["solve2"]["iters"] for s in mstats])), 2),
                         "schur_rebuilds": int(sum(s["amg_rebuilt"] for s in mstats)), "gpu_launches": int(mlaunch)}
        msim.close()
    if not args.no_e2e:
        e2e_v, h2d, d2h = e2e_run(P, case, device, args.steps, args.warmup, precision=P.IBM_PREC_MIXED,
                                  warm=P.IBM_WARM_EXTRAP, **common)
        out["e2e"] = {"value": round(e2e_v, 3), "unit": "steps/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(case)
    if rank == 0:
        print(json.dumps(out), flush=True)


def learned_variant(P, case, device, args, ws, common):
    """The learned warm start on top of the headline variant: the U-Net is
    trained (untimed) with the library's kernels on this workload's own
    snapshots, then the same steps are timed with it attached."""
    import numpy as np
    import torch
    from paper_1109_3524_gb300 import warmstart as WS
    import workloads as W
    t0 = time.perf_counter()
    # training runs: the same geometry at other Reynolds numbers, so the timed
    # flow is never part of the training data
    phis, r0s = [], []
    for re in args.train_re:
        tcase = W.cylinder_stretched(case.nx, float(re), case.dt, args.snapshots)
        ph, rr, _, _ = WS.generate_snapshots(tcase, args.snapshots, device=device, precision=P.IBM_PREC_MIXED,
                                             **common)
        phis.append(ph)
        r0s.append(rr)
    net = P.Unet(16, 4, max_pixels=max(case.nx * case.ny, 8 * 128 * 128), device=device)
    net.init_params(seed=0)
    hist = WS.train(net, phis, r0s, case.nx, case.ny, steps=args.train_steps, batch=8, crop=128, lr=1e-3)
    torch.cuda.synchronize(device)
    train_s = time.perf_counter() - t0
    del phis, r0s
    win = None
    if args.cnn_window and args.cnn_window[0] > 0:
        # inference on a window of cells around the body and its near wake
        import numpy as np
        xc = 0.5 * (case.xf[:-1] + case.xf[1:])
        yc = 0.5 * (case.yf[:-1] + case.yf[1:])
        w, h = args.cnn_window
        x0 = int(np.searchsorted(xc, -0.8))
        y0 = int(np.searchsorted(yc, 0.0)) - h // 2
        win = (min(max(x0, 0), case.nx - w), min(max(y0, 0), case.ny - h), w, h)
        net.set_window(*win)
    lsim, lstats, lms, llaunch, _, lprof, ln = run_variant(
        P, case, device, args.steps, args.warmup, ws, kernel_profile=not args.no_kernel_profile,
        setup=lambda s: s.attach_cnn(net), precision=P.IBM_PREC_MIXED, warm=P.IBM_WARM_CNN, **common)
    lms = max_over_ranks(ws, lms, device)
    res = {"value": round(ws * args.steps / (lms * 1e-3), 3), "unit": "steps/s",
           "k2_mean": round(float(np.mean([s["solve2"]["iters"] for s in lstats])), 2),
           "train": {"runs_re": list(args.train_re), "snapshots_per_run": args.snapshots,
                     "adam_steps": args.train_steps, "batch": 8, "crop": 128,
                     "loss_first": round(float(hist[0]), 5), "loss_last20": round(float(np.mean(hist[-20:])), 5),
                     "seconds_incl_snapshots": round(train_s, 2)},
           "gpu_launches": int(llaunch), "window": list(win) if win else "whole grid"}
    lsim.close()
    net.close()
    return res


def run_reference(args):
    """The CPU oracle as the reference arm (rank 0 only)."""
    ws, rank, _ = (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0)
    if rank != 0:
        return
    import workloads as W
    from oracle import Oracle
    case = W.named(args.workload)
    k = max(1, min(args.steps, 10))
    w = max(0, min(args.warmup, 1))
    t0 = time.perf_counter()
    o = Oracle(case)
    setup = time.perf_counter() - t0
    for _ in range(w):
        o.step()
    t0 = time.perf_counter()
    for _ in range(k):
        o.step()
    el = time.perf_counter() - t0
    v = k / el
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "steps/s", "n_gpus": ws,
           "steps": k, "warmup": w, "ms_per_step": round(1e3 * el / k, 2), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": case.name, "solver": "direct sparse LU (SuperLU), FP64"},
           "cpu_baseline": {"value": round(v, 4), "unit": "steps/s", "cores": 1, "kind": "oracle",
                            "sample": f"{k} steps of {case.name} after {w} warm-up step(s); LU factorisations "
                                      f"({setup:.1f} s) before the timed region"},
           "e2e": {"value": round(v, 4), "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_poisson_micro(args):
    """Section 3's solver comparison: wall time of one Poisson solve to a
    relative residual of 1e-5 from a zero guess, on the 5-point systems of
    2500 to 4e6 unknowns and on the coupled systems of Table 1 (rebuilt with
    cylinders), with CG, Jacobi-PCG and PCG with the smoothed-aggregation
    V-cycle (FP64).  Set-up (host) and solve (device, synchronised wall
    clock, median of three after one untimed solve) are reported apart."""
    import numpy as np
    import torch
    import workloads as W
    import paper_1109_3524_gb300 as P
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    systems = [(f"table1_system{k}", W.table1_system(k)) for k in args.micro_systems]
    systems += [(f"poisson5_{n}x{n}", W.body_free(n)) for n in args.micro_sizes]
    precs = [("cg", P.IBM_PRECOND_NONE), ("pcg_jacobi", P.IBM_PRECOND_JACOBI), ("pcg_sa", P.IBM_PRECOND_AMG)]
    for name, case in systems:
        for pname, pc in precs:
            t0 = time.perf_counter()
            sim = make_sim(P, case, device, tol2=1e-5, max_iter2=200000, poisson_precond=pc)
            setup_s = time.perf_counter() - t0
            rhs = torch.tensor(np.random.default_rng(11).standard_normal(sim.n_lambda), device=device)
            rhs[0] = 0.0   # the pinned cell
            sim.solve_poisson(rhs)
            times = []
            for _ in range(3):
                torch.cuda.synchronize(device)
                t1 = time.perf_counter()
                _, st = sim.solve_poisson(rhs)
                torch.cuda.synchronize(device)
                times.append(time.perf_counter() - t1)
            line = {"bench": "poisson_micro", "system": name, "unknowns": sim.n_lambda, "n_b": case.n_b,
                    "solver": pname, "iters": st["iters"], "status": st["status"], "rel_res": st["rel_res"],
                    "ms_per_solve": 1e3 * statistics.median(times), "setup_s": setup_s, "tol": 1e-5}
            print(json.dumps(line), flush=True)
            if args.micro_out:
                with open(args.micro_out, "a") as f:
                    f.write(json.dumps(line) + "\n")
            del sim
            torch.cuda.empty_cache()


if __name__ == "__main__":
    a = parse()
    if a.poisson_micro:
        run_poisson_micro(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
