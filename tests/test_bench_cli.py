"""bench.py pieces that run without a GPU: the reference arm (the CPU oracle
timed on the host) prints one JSON line with the contract's keys, and the
roofline entry is algorithmic bytes per launch over the mean launch time of
the dominant kernel class."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "cylinder_re40_128", "--steps", "2", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["value"] > 0
    assert d["config"]["workload"] == "cylinder_re40_128"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert abs(d["ms_per_step"] - 1e3 / d["value"]) < 0.02 * d["ms_per_step"]


def test_roofline_of_the_dominant_class():
    """The dominant class is the one with the largest graph-mode time per
    step (time per launch x launches per step); achieved = its algorithmic
    bytes per launch / its graph-mode time per launch; traffic only when the
    recorded capture's kernel-source hash is the current one."""
    sys.path.insert(0, ROOT)
    import bench
    gclass = {"vc_smooth0": {"launches": 14, "ms_per_launch": 4.0e-3, "bytes_per_launch": 12.0e6},
              "pois_spmv": {"launches": 2, "ms_per_launch": 10.0e-3, "bytes_per_launch": 40.0e6}}
    counts = {"vc_smooth0": 300.0, "pois_spmv": 20.0}
    old = dict(bench.NCU_TRAFFIC)
    try:
        bench.NCU_TRAFFIC.clear()
        bench.NCU_TRAFFIC["vc_smooth0"] = {"bytes": 11.0e6, "src": bench.kernel_source_hash()}
        r = bench.roofline(gclass, counts, 6704.5, "measured")
        # 12 MB per launch in 4 us: 3000 GB/s; 1.2 ms per step against 0.2 ms
        assert r["kernel"] == "vc_smooth0" and r["bound"] == "hbm" and r["unit"] == "GB/s"
        assert abs(r["achieved"] - 3000.0) < 0.1
        assert abs(r["frac"] - 3000.0 / 6704.5) < 1e-4
        assert r["traffic"] == 11.0e6
        assert abs(r["class_ms_per_step"]["vc_smooth0"] - 1.2) < 1e-9
        assert r["limiter"] == "HBM bytes or launch latency"
        bench.NCU_TRAFFIC["vc_smooth0"]["src"] = "stale"
        assert bench.roofline(gclass, counts, 6704.5, "measured")["traffic"] is None
        # a class bound by the FP64 units names that limit
        gclass["vel_resid"] = {"launches": 3, "ms_per_launch": 40.0e-3, "bytes_per_launch": 84.0e6}
        counts["vel_resid"] = 60.0
        r = bench.roofline(gclass, counts, 6704.5, "measured")
        assert r["kernel"] == "vel_resid" and r["limiter"].startswith("FP64 ALU")
    finally:
        bench.NCU_TRAFFIC.clear()
        bench.NCU_TRAFFIC.update(old)


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 times the oracle; any other rank exits 0
    without work and prints nothing."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "cylinder_re40_128", "--steps", "2", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""


def test_own_arm_fails_loudly_without_a_gpu():
    """The library's arm has no CPU fallback: on a machine without a CUDA
    device it exits non-zero and prints no result line."""
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "1", "--warmup", "3",
                          "--no-cpu-baseline"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode != 0
    assert out.stdout.strip() == ""
