"""Builds ``libdgsl.so`` in-tree for sm_103a.

Translation units are compiled in parallel (host C++ with g++, CUDA with
nvcc, one ``-gencode`` for compute_103a/sm_103a) and linked into
``paper_2401_17806_gb300/_lib/libdgsl.so`` with the static CUDA runtime.
Host code is compiled with ``-ffp-contract=off`` so that the geometry and
index maps come out the same on x86-64 and on Arm hosts.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUTDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUTDIR, "libdgsl.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

HOST_SOURCES = ["host.cpp", "mg_host.cpp"]
CUDA_SOURCES = ["api.cu", "steps.cu", "k_apply.cu", "k_cg.cu", "k_batch.cu", "k_batch_pc.cu", "k_sl.cu", "server.cu",
                "k_mg.cu"]


def _nvcc():
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand) and not shutil.which(cand):
        raise RuntimeError("nvcc not found; set NVCC or put the CUDA toolkit on PATH")
    return cand


def _sources():
    names = HOST_SOURCES + CUDA_SOURCES
    hdrs = [f for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return [os.path.join(CSRC, f) for f in names + hdrs] + [os.path.join(INCLUDE, "dgsl.h")]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile and link libdgsl.so if any source is newer; return its path."""
    if not force and not stale():
        return LIB
    os.makedirs(OUTDIR, exist_ok=True)
    nvcc = _nvcc()
    objdir = os.path.join(OUTDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    jobs = []
    for src in HOST_SOURCES:
        obj = os.path.join(objdir, src + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall",
                     "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj])
    for src in CUDA_SOURCES:
        obj = os.path.join(objdir, src + ".o")
        cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
               "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE,
               "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info:
            cmd.insert(2, "-Xptxas=-v")
        jobs.append(cmd)
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o, file=sys.stderr)
    objs = [os.path.join(objdir, s + ".o") for s in HOST_SOURCES + CUDA_SOURCES]
    tmp = LIB + ".tmp"
    _run([nvcc, ARCH, "-shared", "-cudart", "static", "-o", tmp] + objs + ["-lpthread", "-ldl", "-lrt"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
