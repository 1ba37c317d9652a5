"""Build libmps.so in-tree: CUDA sources for sm_103a (GB300) plus the C++ host builders.

Usage: python -m paper_2211_07983_gb300.build   (or paper_2211_07983_gb300.build.build())
Translation units compile in parallel; the result is paper_2211_07983_gb300/libmps.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libmps.so")
PEAKS_OUT = os.path.join(HERE, "libpeaks.so")   # arithmetic peak microbenchmarks (roofline denominators)
BUILD = os.path.join(HERE, "_build")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
CU_SOURCES = ["mps_api.cu", "gemm.cu", "gate_kernels.cu", "energy_kernels.cu", "noalloc.cu", "arena.cu", "gemm_tf32.cu", "svd_coop.cu", "gemm_tc.cu"]
CXX_SOURCES = ["host_builders.cpp"]


def _nvcc() -> str:
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(cuda, "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _stale(objs, srcs) -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "mps.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile every translation unit and link libmps.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    objs = []
    for f in CU_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append([nvcc, "-std=c++17", "-O3", ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-Xptxas", "-v" if verbose else "-O3", "-c", os.path.join(CSRC, f), "-o", o])
    for f in CXX_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-c", os.path.join(CSRC, f),
                     "-o", o])
    peaks_job = [nvcc, "-std=c++17", "-O3", ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
                 os.path.join(CSRC, "peaks.cu"), "-o", PEAKS_OUT + ".tmp"]
    if not force and not _stale(objs, CU_SOURCES + CXX_SOURCES) and os.path.exists(PEAKS_OUT):
        return OUT
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs) + 1)) as ex:
        logs = list(ex.map(_run, jobs + [peaks_job]))
    os.replace(PEAKS_OUT + ".tmp", PEAKS_OUT)
    if verbose:
        for lg in logs:
            sys.stdout.write(lg)
    tmp = OUT + ".tmp"
    _run([nvcc, "-shared", ARCH, "-o", tmp] + objs)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force=True))
