"""Build libgbstokes.so in-tree for sm_103a.

Host setup code is compiled by g++ with -ffp-contract=off (the
aggregation's strength test must round like plain multiply/add); the CUDA
translation units by nvcc for compute_103a/sm_103a only.  Units compile
in parallel; the link uses nvcc's static CUDA runtime.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libgbstokes.so")

CU_UNITS = ["capi.cu", "amg_fp64.cu", "amg_fp32.cu", "amg_bf16.cu", "noalloc.cu", "peak.cu"]
CPP_UNITS = ["setup.cpp"]
GENCODE = "arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _sources_newer(obj: str, srcs) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(s) > t for s in srcs)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".hpp", ".cuh", ".h"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "gbstokes.h"))
    jobs = []
    objs = []
    for u in CU_UNITS:
        src = os.path.join(CSRC, u)
        obj = os.path.join(OUT_DIR, u + ".o")
        objs.append(obj)
        if force or _sources_newer(obj, [src] + headers):
            jobs.append([nvcc, "-gencode", GENCODE, "-O3", "-lineinfo", "-std=c++17",
                         "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                         "--expt-relaxed-constexpr", "-c", src, "-o", obj])
    for u in CPP_UNITS:
        src = os.path.join(CSRC, u)
        obj = os.path.join(OUT_DIR, u + ".o")
        objs.append(obj)
        if force or _sources_newer(obj, [src] + headers):
            jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-c", src,
                         "-o", obj])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), p.stdout, p.stderr))
        return p.stderr

    with ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for err in ex.map(run, jobs):
            if verbose and err:
                print(err)
    if jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        run([nvcc, "-gencode", GENCODE, "-shared", "-o", tmp] + objs)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose=True, force="--force" in sys.argv))
