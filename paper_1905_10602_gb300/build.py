"""Builds libifmm.so in-tree for sm_103a (GB300).

Four CUDA translation units compiled by nvcc (runtime.cu: every kernel of the
main path; noalloc.cu: the allocation-free matvec; mlp.cu: the rank
predictor's training and inference kernels; probe.cu: the arithmetic-peak
probes) and the host translation units compiled by g++, in parallel, then
linked against the CUDA runtime.  `python -m paper_1905_10602_gb300.build` or build() from Python.
"""

from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libifmm.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

CU_SOURCES = ["runtime.cu", "noalloc.cu", "mlp.cu", "probe.cu"]
CPP_SOURCES = ["tree.cpp", "factor.cpp", "solve.cpp", "batch.cpp", "bd.cpp", "fmm.cpp"]


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + p.stdout)
    return p.stdout


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "ifmm.h"))
    jobs = []
    objs = []
    for src in CU_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([os.path.join(CUDA, "bin", "nvcc"), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler",
                         "-fPIC", "-Xptxas", "-v" if verbose else "-O3", "-c", s, "-o", o])
    for src in CPP_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", "-Wno-unused-function",
                         "-I" + os.path.join(CUDA, "include"), "-c", s, "-o", o])
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    if force or jobs or not os.path.exists(LIB):
        _run(["g++", "-shared", "-o", LIB] + objs + ["-L" + os.path.join(CUDA, "lib64"), "-lcudart", "-lpthread",
                                                     "-Wl,-rpath," + os.path.join(CUDA, "lib64")])
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
