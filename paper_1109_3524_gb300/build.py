"""Builds libibm.so (the C-ABI library) in-tree for sm_103a.

Host code is compiled with g++ and the CUDA sources with nvcc, in parallel;
the CUDA runtime is linked statically so the library loads on machines
without a GPU (its CUDA calls then fail with an error status).
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libibm.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cu = ["k_solve.cu", "k_level0.cu", "k_coop.cu", "k_body.cu", "k_step.cu", "k_vel32.cu", "k_tail.cu", "api.cu", "noalloc.cu", "unet.cu", "k_conv_tc.cu"]
    cpp = ["host.cpp"]
    jobs = []
    for f in cu:
        o = os.path.join(BUILD, f + ".o")
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", "-c", os.path.join(CSRC, f), "-o", o]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, o))
    for f in cpp:
        o = os.path.join(BUILD, f + ".o")
        jobs.append((["g++", "-O2", "-fPIC", "-std=c++17", "-c", os.path.join(CSRC, f), "-o", o], o))
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose:
        for o in outs:
            if o:
                print(o)
    tmp = OUT + ".tmp"
    _run([NVCC, *ARCH, "-shared", "-cudart", "static", "-o", tmp] + [o for _, o in jobs])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv))


def ensure_built() -> str:
    """Rebuilds when the library is missing or older than a source file."""
    srcs = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "ibm.h")]
    if os.path.exists(OUT):
        t = os.path.getmtime(OUT)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return OUT
    return build()
