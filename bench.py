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
    ap.add_argument("--spinup", type=int, default=1000,
                    help="untimed steps from the uniform start before every variant's warm-up (the timed window "
                         "then lies past the impulsive-start transient); 0: time from the start")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-kernel-profile", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned warm-start variant")
    ap.add_argument("--no-moving", action="store_true", help="skip the moving-body workload")
    ap.add_argument("--no-bn3", action="store_true", help="skip the N = 3 (B^3) line")
    ap.add_argument("--no-extrap", action="store_true", help="skip the extrapolated warm-start line")
    ap.add_argument("--no-flapping", action="store_true", help="skip the flapping-airfoil workload (section 6.2)")
    ap.add_argument("--no-c5", action="store_true", help="skip the 4096^2 four-cylinder workload")
    ap.add_argument("--no-coupled", action="store_true", help="skip the coupled-SA (section 3) arm")
    ap.add_argument("--coupled-steps", type=int, default=5, help="timed steps of the coupled-SA arm")
    ap.add_argument("--no-c1", action="store_true", help="skip the 128^2 Re 40 line (parity with the oracle)")
    ap.add_argument("--no-c3", action="store_true", help="skip the 2048^2 Re 200 mixed-precision line")
    ap.add_argument("--c3-steps", type=int, default=50, help="steps of the 2048^2 line")
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
    ap.add_argument("--cnn-only", action="store_true",
                    help="instead of the step benchmark: time the forward convolutions of the warm-start U-Net "
                         "(base 16, 4 levels, He-initialised) on the inference window and a training batch, "
                         "tcgen05 beside mma.sync (one JSON line)")
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

class optional_line:
    """Runs one secondary bench line; an exception there is printed to stderr
    and recorded as {"error": ...} under its key, so that the headline line is
    still printed."""

    def __init__(self, out, key):
        self.out, self.key = out, key

    def __enter__(self):
        return self

    def __exit__(self, et, ev, tb):
        if et is None or not issubclass(et, Exception):
            return False
        import gc
        import traceback
        traceback.print_exception(et, ev, tb, file=sys.stderr)
        self.out[self.key] = {"error": f"{et.__name__}: {ev}"}
        del tb
        gc.collect()
        try:
            import torch
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        except Exception:
            pass
        return True


def make_sim(P, case, device, state=None, **kw):
    """A context at the uniform start, or at `state` (a get_state() dict)."""
    import numpy as np
    sim = P.Sim.from_case(case, device=device, **kw)
    if state is None:
        U0, V0 = case.initial_velocity()
        sim.set_state(u=U0, v=V0, v_right=np.full(case.ny + 1, case.vinf), t=0.0, step=0)
    else:
        sim.set_state(**state)
        if case.n_b:
            xb, yb, ub, vb = case.body_state(state["t"] + case.dt)
            sim.set_body(xb, yb, ub, vb)
    return sim


def spin_up(P, case, device, nsteps, **kw):
    """Untimed steps from the uniform start; returns the state to time from."""
    if nsteps <= 0:
        return None
    sim = make_sim(P, case, device, **kw)
    t = 0.0
    for _ in range(nsteps):
        if case.moving:
            xb, yb, ub, vb = case.body_state(t + case.dt)
            sim.set_body(xb, yb, ub, vb)
        sim.step(1)
        t += case.dt
    s = sim.get_state()
    sim.close()
    return {"u": s["u"], "v": s["v"], "v_right": s["v_right"], "nprev": s["nprev"], "lam": s["lambda"],
            "t": s["t"], "step": s["step"]}


def run_variant(P, case, device, steps, warmup, ws, kernel_profile=True, setup=None, state=None, **kw):
    """Device-timed steps (CUDA events on the library's stream), then a second
    pass with per-kernel events (launch counts and bytes per kernel class)."""
    import torch
    sim = make_sim(P, case, device, state=state, **kw)
    if setup is not None:
        setup(sim)
    body = case.body_state
    t = 0.0 if state is None else state["t"]

    host_ms = []   # wall time of ibm_set_body per step (moving bodies)

    def advance(n):
        nonlocal t
        out = []
        for _ in range(n):
            xb, yb, ub, vb = body(t + case.dt)
            if case.moving:
                t0 = time.perf_counter()
                sim.set_body(xb, yb, ub, vb)
                host_ms.append(1e3 * (time.perf_counter() - t0))
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
    sim.set_body_ms = float(sum(host_ms[-steps:]) / steps) if host_ms else 0.0
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


# DRAM bytes per launch of a kernel class, from one ncu capture (the summary
# named in "capture"), valid only while the kernel sources hash to "src": a
# changed kernel reports traffic null until it is captured again.
NCU_TRAFFIC = {}


# classes whose kernels are bound by GB300's FP64 units rather than by HBM
# (ncu: FP64 pipe 68-81 % busy at 22-26 % of DRAM bandwidth for the FP64 CG
# vector kernels); their HBM fraction understates how close they run
FP64_CLASSES = {
    "warm": "FP64 ALU (about 2m + (4m + 12)/2 FP64 operations per unknown for m basis vectors)",
    "vel_resid": "FP64 ALU (6 FP64 operations per unknown)",
    "rhs": "FP64 ALU (about 46 FP64 operations per velocity unknown)",
    "pois_update": "FP64 ALU and HBM (3 FP64 operations and 48 B per unknown)",
    "pois_spmv": "FP64 ALU (6 FP64 operations per unknown)",
}


def kernel_source_hash():
    import hashlib
    d = os.path.join(ROOT, "paper_1109_3524_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def roofline(gclass, counts, peak, peak_kind):
    """Dominant kernel class by graph-mode time per step (graph-mode time per
    launch x launches per step); achieved = its algorithmic bytes per launch /
    its graph-mode time per launch."""
    per_step = {k: v["ms_per_launch"] * counts.get(k, 0) for k, v in gclass.items()}
    k = max(per_step, key=per_step.get)
    g = gclass[k]
    ach = g["bytes_per_launch"] / (g["ms_per_launch"] * 1e-3) / 1e9 if g["ms_per_launch"] > 0 else 0.0
    tr = NCU_TRAFFIC.get(k)
    traffic = tr["bytes"] if tr and tr.get("src") == kernel_source_hash() else None
    return {"kernel": k, "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4), "traffic": traffic, "peak_source": peak_kind,
            "limiter": FP64_CLASSES.get(k, "HBM bytes or launch latency"),
            "bytes_per_launch": g["bytes_per_launch"], "ms_per_launch": g["ms_per_launch"],
            "timing": "CUDA-graph replay of the class's launches of one step, back to back, CUDA events",
            "class_ms_per_step": {c: round(v, 4) for c, v in sorted(per_step.items(), key=lambda x: -x[1])}}


def e2e_run(P, case, device, steps, warmup, state=None, **kw):
    """End to end through the public API with host buffers: every step sends
    the body state from pinned host memory and reads back the step's forces
    and solver statistics."""
    import numpy as np
    import torch
    sim = make_sim(P, case, device, state=state, **kw)
    pin = [torch.empty(case.n_b, dtype=torch.float64).pin_memory() for _ in range(4)]
    t = 0.0 if state is None else state["t"]

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


def graph_class_times(sim, prof, reps=20):
    """Graph-mode time per launch of every kernel class the step launches (each
    call runs one more step on `sim`; use it last)."""
    out = {}
    for k in sorted(prof, key=lambda n: -prof[n]["ms"]):
        if prof[k]["launches"] <= 0:
            continue
        try:
            out[k] = sim.profile_graph_class(k, reps)
        except Exception as e:   # a class that the extra step did not launch
            print(f"[bench] graph timing of {k}: {e}", file=sys.stderr, flush=True)
    return out


def constraint_maxima(stats):
    return {"div_max": float(max(s["div_max"] for s in stats)),
            "slip_max": float(max(s["slip_max"] for s in stats)),
            "what": "max over the timed steps of the FP64 device check of q^{n+1}: |G^T q + bc2| (unpinned "
                    "cells) and |E q - u_B| (Eq. 8)"}


def c1_line(P, device):
    """The 128^2 Re 40 workload as configured (FP64, Jacobi-PCG velocity solve,
    AMG-PCG Poisson solve, both to 1e-8, 50 steps from the seeded noisy start):
    steps/s and the per-step deviation of C_d from the oracle stepped beside it."""
    import numpy as np
    import torch
    import workloads as W
    from oracle import Oracle
    case = W.cylinder_re40_128()
    sim = make_sim(P, case, device, tol1=1e-8, tol2=1e-8, precision=P.IBM_PREC_FP64, warm=P.IBM_WARM_PREV)
    o = Oracle(case)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ms, dev, k2 = 0.0, [], []
    for _ in range(case.nsteps):
        xb, yb, ub, vb = case.body_state(o.t + case.dt)
        sim.set_body(xb, yb, ub, vb)
        e0.record(sim.stream)
        st = sim.step(1)[0]
        e1.record(sim.stream)
        torch.cuda.synchronize(device)
        ms += e0.elapsed_time(e1)
        so = o.step()
        dev.append(abs(st["cd"] - so.cd) / abs(so.cd))
        k2.append(st["solve2"]["iters"])
    sim.close()
    return {"workload": case.name, "value": round(case.nsteps / (ms * 1e-3), 3), "unit": "steps/s",
            "steps": case.nsteps, "k2_mean": round(float(np.mean(k2)), 2),
            "cd_dev_max_vs_oracle": float(max(dev)),
            "variant": "FP64 V-cycle (coupled SA) in PCG, warm start lambda^n, tol 1e-8; steps timed one by one"}


def c3_line(P, device, steps, common):
    """The 2048^2 Re 200 workload in the production mixed configuration:
    steps/s over `steps` steps after a short untimed start, and per step the
    relative deviation of C_d, C_l and the velocity from the same steps taken
    with the FP64 V-cycle at tolerance 1e-12 from the same state.  A direct
    factorisation at this size (4.2 M cells) is beyond a bench run; the FP64
    path is tied to the oracle by the parity tests."""
    import numpy as np
    import torch
    import workloads as W
    case = W.named("cylinder_re200_2048")
    kw = dict(common, precision=P.IBM_PREC_MIXED, warm=P.IBM_WARM_EXTRAP)
    state = spin_up(P, case, device, 20, **kw)
    sim = make_sim(P, case, device, state=state, **kw)
    ref = make_sim(P, case, device, state=state, **dict(kw, precision=P.IBM_PREC_FP64, tol1=1e-12, tol2=1e-12,
                                                          max_iter2=5000))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ms, k2, dcd, dcl, dq = 0.0, [], [], [], []
    for _ in range(steps):
        e0.record(sim.stream)
        a = sim.step(1)[0]
        e1.record(sim.stream)
        torch.cuda.synchronize(device)
        ms += e0.elapsed_time(e1)
        b = ref.step(1)[0]
        k2.append(a["solve2"]["iters"])
        dcd.append(abs(a["cd"] - b["cd"]) / abs(b["cd"]))
        dcl.append(abs(a["cl"] - b["cl"]) / abs(b["cd"]))
    sa, sb = sim.get_state(), ref.get_state()
    dq = max(float(np.abs(sa["u"] - sb["u"]).max()), float(np.abs(sa["v"] - sb["v"]).max())) / \
        float(np.abs(sb["u"]).max())
    sim.close()
    ref.close()
    return {"workload": case.name, "value": round(steps / (ms * 1e-3), 3), "unit": "steps/s", "steps": steps,
            "k2_mean": round(float(np.mean(k2)), 2), "start_t": state["t"],
            "cd_dev_max_vs_fp64": float(max(dcd)), "cl_dev_max_vs_fp64": float(max(dcl)),
            "velocity_dev_vs_fp64_last": dq,
            "reference": "the same steps with the FP64 V-cycle at tolerance 1e-12 from the same state",
            "variant": "FP32 SA V-cycle (Schur block) in FP64 flexible CG, extrapolated warm start, tol 1e-8"}


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
    # sweeps each way on the finest level (one temporally blocked kernel each
    # way), Jacobi weight 0.85 * 2 / rho(D^-1 A), one kernel per phase on the
    # coarse levels (measured faster than the single-cluster coarse kernel
    # once the coarsest solve is FP64)
    common = dict(tol1=1e-8, tol2=1e-8, poisson_precond=P.IBM_PRECOND_SCHUR, amg_trunc=args.trunc,
                  amg_theta=0.02, amg_max_coarse=2048, amg_tail_rows=0, amg_sweeps0=3, amg_omega=0.85)
    # headline: FP32 V-cycle in FP64 flexible CG, the warm start projected onto
    # the span of the previous solutions; the spin-up and the other variants
    # start from the same state (spun up with the extrapolated warm start)
    headline = dict(precision=P.IBM_PREC_MIXED, warm=P.IBM_WARM_PROJ, **common)
    extrap = dict(headline, warm=P.IBM_WARM_EXTRAP)
    t_spin = time.perf_counter()
    state = spin_up(P, case, device, args.spinup, **extrap)
    t_spin = time.perf_counter() - t_spin
    t_start = state["t"] if state else 0.0
    window = [round(t_start + args.warmup * case.dt, 6), round(t_start + (args.warmup + args.steps) * case.dt, 6)]
    sim, stats, ms, launches, clocks, prof, nprof = run_variant(
        P, case, device, args.steps, args.warmup, ws, kernel_profile=not args.no_kernel_profile,
        state=state, **headline)
    ms_max = max_over_ranks(ws, ms, device)
    value = ws * args.steps / (ms_max * 1e-3)
    k1 = [s["solve1"]["iters"] for s in stats]
    k2 = [s["solve2"]["iters"] for s in stats]
    # the Poisson solves of the timed steps themselves (events around each solve)
    pois_ms = float(sum(s["poisson_ms"] for s in stats))
    pois_bytes = float(sum(s["poisson_bytes"] for s in stats))
    pois_gbs = pois_bytes / (pois_ms * 1e-3) / 1e9 if pois_ms > 0 else 0.0
    roof = None
    if prof:
        counts = {k: v["launches"] / nprof for k, v in prof.items()}
        gclass = graph_class_times(sim, prof)
        roof = roofline(gclass, counts, peak, peak_kind)
        if args.profile_out and rank == 0:
            with open(args.profile_out, "w") as f:
                json.dump({"steps": nprof, "classes": prof, "graph": gclass}, f, indent=1)
    sim.close()
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": case.name, "grid": f"{case.nx}x{case.ny} stretched 1.02 outside [-2,2]^2",
                   "domain": "[-15,15]^2", "n_b": case.n_b, "Re": round(1.0 / case.nu), "dt": case.dt,
                   "variant": "FP32 SA V-cycle (Schur block) in FP64 flexible CG, warm start projected onto the span "
                              "of up to 24 previous solutions",
                   "tol": 1e-8, "parallelism": "replicas" if ws > 1 else "single GPU",
                   "timed_window": {"t": window, "spinup_steps": args.spinup, "spinup_s": round(t_spin, 2),
                                    "note": "every variant starts from the same spun-up state"},
                   "l2": "working set ~0.5 GB > 129 MB L2 (no flush needed)"},
        "iters": {"k1_mean": round(float(np.mean(k1)), 2), "k2_mean": round(float(np.mean(k2)), 2),
                  "k2_max": int(max(k2))},
        "poisson": {"gbs": round(pois_gbs, 1), "frac_hbm": round(pois_gbs / peak, 4),
                    "ms_per_step": round(pois_ms / len(stats), 4),
                    "bytes_per_step": round(pois_bytes / len(stats)),
                    "timing": "CUDA events around each Poisson solve of the timed steps"},
        "roofline": roof,
        "constraints": constraint_maxima(stats),
        "gpu_launches": int(launches),
        "clocks": clocks,
        "cd_last": stats[-1]["cd"],
        "forces": {"cd_last": stats[-1]["cd"], "cl_last": stats[-1]["cl"],
                   "cd_mean": float(np.mean([s["cd"] for s in stats])),
                   "cl_max_abs": float(np.max(np.abs([s["cl"] for s in stats]))),
                   "time_units": round(len(stats) * case.dt, 6), "strouhal": None},
    }
    if not args.no_plain:
        with optional_line(out, "plain_fp64"):
            # plain FP64 AMG-PCG with the same preconditioner structure, warm start lambda^n
            psim, pstats, pms, _, _, _, _ = run_variant(
                P, case, device, args.steps, args.warmup, ws, kernel_profile=False, state=state,
                precision=P.IBM_PREC_FP64, warm=P.IBM_WARM_PREV, **common)
            pms = max_over_ranks(ws, pms, device)
            pm = sum(s["poisson_ms"] for s in pstats)
            pb = sum(s["poisson_bytes"] for s in pstats)
            out["plain_fp64"] = {"value": round(ws * args.steps / (pms * 1e-3), 3), "unit": "steps/s",
                                 "k2_mean": round(float(np.mean([s["solve2"]["iters"] for s in pstats])), 2),
                                 "poisson_gbs": round(pb / (pm * 1e-3) / 1e9, 1) if pm > 0 else None,
                                 "variant": "FP64 V-cycle (Schur block) in PCG, warm start lambda^n"}
            psim.close()
    if not args.no_coupled:
        with optional_line(out, "plain_coupled_sa"):
            # section 3's method as the paper runs it: SA on the whole coupled Q^T B Q, FP64 PCG, lambda^n
            cs = max(1, min(args.coupled_steps, args.steps))
            ckw = dict(common, poisson_precond=P.IBM_PRECOND_AMG, amg_theta=0.08, amg_max_coarse=256,
                       amg_sweeps0=0, amg_omega=2.0 / 3.0, max_iter2=5000)
            csim, cstats, cms, _, _, _, _ = run_variant(
                P, case, device, cs, 1, ws, kernel_profile=False, state=state, precision=P.IBM_PREC_FP64,
                warm=P.IBM_WARM_PREV, **ckw)
            cms = max_over_ranks(ws, cms, device)
            out["plain_coupled_sa"] = {
                "value": round(ws * cs / (cms * 1e-3), 3), "unit": "steps/s", "steps": cs,
                "k2_mean": round(float(np.mean([s["solve2"]["iters"] for s in cstats])), 2),
                "status": [s["solve2"]["status"] for s in cstats],
                "variant": "FP64 smoothed aggregation on the whole coupled Q^T B Q (section 3) in PCG, lambda^n"}
            csim.close()
    if not args.no_learned:
        with optional_line(out, "learned_mixed"):
            out["learned_mixed"] = learned_variant(P, case, device, args, ws, common, state)
    if not args.no_extrap:
        with optional_line(out, "extrap_mixed"):
            # the headline variant with the extrapolated warm start
            # 2 lambda^n - lambda^{n-1} instead of the projection
            jsim, jstats, jms, jlaunch, _, _, _ = run_variant(
                P, case, device, args.steps, args.warmup, ws, kernel_profile=False, state=state, **extrap)
            jms = max_over_ranks(ws, jms, device)
            out["extrap_mixed"] = {
                "value": round(ws * args.steps / (jms * 1e-3), 3), "unit": "steps/s", "steps": args.steps,
                "k2_mean": round(float(np.mean([s["solve2"]["iters"] for s in jstats])), 2),
                "rel_res0_mean": float(np.mean([s["solve2"]["rel_res0"] for s in jstats])),
                "poisson_ms_per_step": round(float(np.mean([s["poisson_ms"] for s in jstats])), 4),
                "gpu_launches": int(jlaunch), "constraints": constraint_maxima(jstats),
                "variant": "FP32 SA V-cycle (Schur block) in FP64 flexible CG, extrapolated warm start, tol 1e-8"}
            jsim.close()
    if not args.no_bn3:
        with optional_line(out, "bn3"):
            # section 4 / Table 2: B^3 (third-order series for A^-1) in the
            # projection and in Q^T B^3 Q, applied matrix-free on the device,
            # preconditioned by the Schur block preconditioner of Q^T B^1 Q
            bsteps = max(5, min(args.steps, 20))
            bkw = dict(extrap, bn_order=3)
            bsim, bstats, bms, blaunch, _, _, _ = run_variant(
                P, case, device, bsteps, args.warmup, ws, kernel_profile=False, state=state, **bkw)
            bms = max_over_ranks(ws, bms, device)
            out["bn3"] = {"value": round(ws * bsteps / (bms * 1e-3), 3), "unit": "steps/s", "steps": bsteps,
                          "k2_mean": round(float(np.mean([s["solve2"]["iters"] for s in bstats])), 2),
                          "poisson_ms_per_step": round(float(np.mean([s["poisson_ms"] for s in bstats])), 4),
                          "gpu_launches": int(blaunch), "constraints": constraint_maxima(bstats),
                          "variant": "N = 3: Q^T B^3 Q matrix-free (projection chain), Schur block "
                                     "preconditioner of Q^T B^1 Q, FP32 V-cycle in FP64 flexible CG, "
                                     "extrapolated warm start, tol 1e-8, from the same spun-up state"}
            bsim.close()
    if not args.no_moving:
        with optional_line(out, "moving"):
            # the moving-body path (E and the coupling rows rebuilt every step, the
            # Schur complement rebuilt every step from the cache of V-cycle responses)
            mcase = W.named("oscillating_cylinder_re100_1024")
            msteps = max(10, min(args.steps, 50))
            mkw = dict(precision=P.IBM_PREC_MIXED, warm=P.IBM_WARM_EXTRAP, moving=1, amg_rebuild_every=1, **common)
            mstate = spin_up(P, mcase, device, min(args.spinup, 100), **mkw)
            msim, mstats, mms, mlaunch, _, _, _ = run_variant(
                P, mcase, device, msteps, args.warmup, ws, kernel_profile=False, state=mstate, **mkw)
            mms = max_over_ranks(ws, mms, device)
            out["moving"] = {"workload": mcase.name, "value": round(ws * msteps / (mms * 1e-3), 3), "unit": "steps/s",
                             "steps": msteps, "k2_mean": round(float(np.mean([s["solve2"]["iters"] for s in mstats])), 2),
                             "schur_rebuilds": int(sum(s["amg_rebuilt"] for s in mstats)), "gpu_launches": int(mlaunch),
                             "poisson_ms_per_step": round(float(np.mean([s["poisson_ms"] for s in mstats])), 4),
                             "set_body_ms_per_step": round(msim.set_body_ms, 4),
                             "body_rows": "pattern on the host (integer work), values on the device",
                             "spinup_steps": min(args.spinup, 100), "constraints": constraint_maxima(mstats)}
            msim.close()
            if not args.no_learned:
                # the learned warm start on the moving workload, trained on the
                # oscillating cylinder at the training Reynolds numbers
                out["moving"]["learned_mixed"] = learned_variant(P, mcase, device, args, ws, common, state=mstate,
                                                                 moving=True, roofline=False)
    if not args.no_flapping:
        with optional_line(out, "flapping"):
            # section 6.2: the flapping airfoil (Table 1's system 3) with the body
            # rows formed on the device every step; the paper's context figure is
            # 164 s for one period (4000 steps) on a C2050
            fcase = W.named("flapping_ellipse_re75_930x654")
            fsteps = max(10, min(args.steps * 5, 100))
            fkw = dict(precision=P.IBM_PREC_MIXED, warm=P.IBM_WARM_EXTRAP, moving=1, amg_rebuild_every=1, **common)
            fspin = min(args.spinup, 400)
            fstate = spin_up(P, fcase, device, fspin, **fkw)
            fsim, fstats, fms, flaunch, _, _, _ = run_variant(
                P, fcase, device, fsteps, args.warmup, ws, kernel_profile=False, state=fstate, **fkw)
            fms = max_over_ranks(ws, fms, device)
            fv = ws * fsteps / (fms * 1e-3)
            out["flapping"] = {"workload": fcase.name, "value": round(fv, 3), "unit": "steps/s", "steps": fsteps,
                               "spinup_steps": fspin, "k2_mean": round(float(np.mean([s["solve2"]["iters"] for s in fstats])), 2),
                               "poisson_ms_per_step": round(float(np.mean([s["poisson_ms"] for s in fstats])), 4),
                               "set_body_ms_per_step": round(fsim.set_body_ms, 4), "gpu_launches": int(flaunch),
                               "seconds_per_period": round(4000.0 / fv, 2),
                               "paper_seconds_per_period_c2050": 164.0,
                               "constraints": constraint_maxima(fstats)}
            fsim.close()
    if not args.no_c5:
        with optional_line(out, "c5"):
            # 4096^2, four cylinders, the downstream pair heaving: body rows and S
            # (5040 force unknowns) rebuilt every step
            ccase = W.named("four_cylinders_re150_4096")
            csteps = 10
            ckw = dict(precision=P.IBM_PREC_MIXED, warm=P.IBM_WARM_EXTRAP, moving=1, amg_rebuild_every=1, **common)
            csim, cstats, cms, claunch, _, _, _ = run_variant(P, ccase, device, csteps, min(args.warmup, 3), ws,
                                                              kernel_profile=False, **ckw)
            cms = max_over_ranks(ws, cms, device)
            out["c5"] = {"workload": ccase.name, "value": round(ws * csteps / (cms * 1e-3), 3), "unit": "steps/s",
                         "steps": csteps, "cells": ccase.nx * ccase.ny, "n_b": ccase.n_b,
                         "k2_mean": round(float(np.mean([s["solve2"]["iters"] for s in cstats])), 2),
                         "poisson_ms_per_step": round(float(np.mean([s["poisson_ms"] for s in cstats])), 3),
                         "set_body_ms_per_step": round(csim.set_body_ms, 3), "gpu_launches": int(claunch),
                         "timed_window": "steps 4-13 from the uniform start",
                         "constraints": constraint_maxima(cstats)}
            csim.close()
    if not args.no_c1 and rank == 0:
        with optional_line(out, "c1"):
            out["c1"] = c1_line(P, device)
    if not args.no_c3 and rank == 0:
        with optional_line(out, "c3"):
            out["c3"] = c3_line(P, device, args.c3_steps, common)
    if not args.no_e2e:
        with optional_line(out, "e2e"):
            e2e_v, h2d, d2h = e2e_run(P, case, device, args.steps, args.warmup, state=state, **headline)
            out["e2e"] = {"value": round(e2e_v, 3), "unit": "steps/s", "h2d_bytes_per_step": int(h2d),
                          "d2h_bytes_per_step": int(d2h)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        with optional_line(out, "cpu_baseline"):
            out["cpu_baseline"] = cpu_baseline(case)
    if rank == 0:
        print(json.dumps(out), flush=True)


def learned_variant(P, case, device, args, ws, common, state=None, moving=False, roofline=True):
    """The learned warm start on top of the headline variant: the U-Net is
    trained (untimed) with the library's kernels on snapshots of the same
    geometry at other Reynolds numbers, then the same steps are timed with it
    attached.  moving: the oscillating cylinder (body rows and S rebuilt every
    step, in training and in the timed steps)."""
    import numpy as np
    import torch
    from paper_1109_3524_gb300 import warmstart as WS
    import workloads as W
    t0 = time.perf_counter()
    mkw = dict(moving=1, amg_rebuild_every=1) if moving else {}
    # training runs: the same geometry at other Reynolds numbers, so the timed
    # flow is never part of the training data
    phis, r0s = [], []
    for re in args.train_re:
        if moving:
            tcase = W.oscillating_cylinder(case.nx, float(re), case.dt, args.snapshots)
        else:
            tcase = W.cylinder_stretched(case.nx, float(re), case.dt, args.snapshots)
        ph, rr, _, _ = WS.generate_snapshots(tcase, args.snapshots, device=device, precision=P.IBM_PREC_MIXED,
                                             **mkw, **common)
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
    lsteps = max(10, min(args.steps, 50)) if moving else args.steps
    lsim, lstats, lms, llaunch, _, lprof, ln = run_variant(
        P, case, device, lsteps, args.warmup, ws, kernel_profile=False, state=state,
        setup=lambda s: s.attach_cnn(net), precision=P.IBM_PREC_MIXED, warm=P.IBM_WARM_CNN, **mkw, **common)
    lms = max_over_ranks(ws, lms, device)
    res = {"value": round(ws * lsteps / (lms * 1e-3), 3), "unit": "steps/s", "steps": lsteps,
           "k2_mean": round(float(np.mean([s["solve2"]["iters"] for s in lstats])), 2),
           "train": {"runs_re": list(args.train_re), "snapshots_per_run": args.snapshots,
                     "adam_steps": args.train_steps, "batch": 8, "crop": 128,
                     "loss_first": round(float(hist[0]), 5), "loss_last20": round(float(np.mean(hist[-20:])), 5),
                     "seconds_incl_snapshots": round(train_s, 2)},
           "gpu_launches": int(llaunch), "window": list(win) if win else "whole grid"}
    lsim.close()
    if roofline:
        res["cnn_roofline"] = cnn_roofline(P, net, device, max(case.nx * case.ny, 8 * 128 * 128))
    net.close()
    return res


def cnn_roofline(P, net, device, max_pixels, reps=20):
    """The forward convolutions of the warm-start U-Net, each timed with CUDA
    events (ibm_cnn_time_forward), on the inference window and on a training
    batch: algorithmic FLOPs 2 P K cout (K = ks^2 cin) and bytes (input and
    output activations once, BF16, plus the weights) per convolution.  The
    dominant convolution is reported against the measured BF16 tensor peak
    when it has 64 or more output channels, else against HBM.  The same
    network with every convolution on mma.sync (IBM_CNN_NO_TC=1) is timed
    beside it."""
    import numpy as np
    d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    tpeak, hpeak = float(d.get("bf16_tflops", 1900.0)), float(d.get("hbm_gbs", 6800.0))
    src = "measured" if d else "fallback"
    os.environ["IBM_CNN_NO_TC"] = "1"
    try:
        ref = P.Unet(net.base, net.levels, max_pixels=max_pixels, device=device)
    finally:
        del os.environ["IBM_CNN_NO_TC"]
    ref.set_params(net.get_params())
    lay = net.layers()
    out = {}
    for name, (B, H, W) in (("inference_window", (1, 256, 512)), ("training_batch", (8, 128, 128))):
        ms_tc = net.time_forward(B, H, W, reps=reps)
        ms_ms = ref.time_forward(B, H, W, reps=reps)
        rows, tot_f, tot_ms = [], 0.0, 0.0
        for i, ly in enumerate(lay):
            px = B * (H >> ly["level"]) * (W >> ly["level"])
            fl = 2.0 * px * ly["ks"] ** 2 * ly["cin"] * ly["cout"]
            by = 2.0 * px * (ly["cin"] + ly["cout"]) + 2.0 * ly["ks"] ** 2 * ly["cin"] * ly["cout"] + 4.0 * ly["cout"]
            rows.append({"conv": i, "cin": ly["cin"], "cout": ly["cout"], "pixels": px, "tcgen05": ly["tcgen05"],
                         "us": round(1e3 * ms_tc[i], 2), "us_mma_sync": round(1e3 * ms_ms[i], 2),
                         "tflops": round(fl / (ms_tc[i] * 1e-3) / 1e12, 2),
                         "gbs": round(by / (ms_tc[i] * 1e-3) / 1e9, 1)})
            tot_f += fl
            tot_ms += ms_tc[i]
        dom = max(rows, key=lambda r: r["us"])
        tensor = dom["cout"] >= 64
        ach = dom["tflops"] if tensor else dom["gbs"]
        out[name] = {"batch_hw": [B, H, W], "convs_us": round(1e3 * tot_ms, 1),
                     "convs_us_mma_sync": round(1e3 * float(np.sum(ms_ms)), 1),
                     "tflops": round(tot_f / (tot_ms * 1e-3) / 1e12, 2),
                     "dominant": {"conv": dom["conv"], "bound": "tensor" if tensor else "hbm", "achieved": ach,
                                  "peak": tpeak if tensor else hpeak, "unit": "TFLOP/s" if tensor else "GB/s",
                                  "frac": round(ach / (tpeak if tensor else hpeak), 4), "peak_source": src},
                     "layers": rows}
    ref.close()
    return out


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


def run_cnn_only(args):
    import torch
    import paper_1109_3524_gb300 as P
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    P.load()
    net = P.Unet(16, 4, max_pixels=1 << 20, device=device)
    net.init_params(seed=0)
    print(json.dumps({"bench": "cnn_forward", "network": "U-Net base 16, 4 levels (16-32-64-128)",
                      "cnn_roofline": cnn_roofline(P, net, device, 1 << 20)}))
    net.close()


if __name__ == "__main__":
    a = parse()
    if a.poisson_micro:
        run_poisson_micro(a)
    elif a.cnn_only:
        run_cnn_only(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
