"""Compile the simulator's shared library (libsnn.so) for sm_103a, in-tree.

Sources are compiled in parallel to objects under _build/ and linked into
paper_2405_02019_gb300/libsnn.so against the shared CUDA runtime.  Device code uses
-fmad=false and host code -ffp-contract=off so that no product-sum is fused.
"""

from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libsnn.so")
BUILD = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)

SOURCES = ["builder.cpp", "kernels.cu", "resident.cu", "abi.cu", "noalloc.cu"]
HEADERS = ["internal.hpp", "philox.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _flags(verbose_ptx: bool = False):
    f = ["-std=c++17", "-O3", ARCH, "-lineinfo", "-fmad=false", f"-I{ROOT}",
         "-Xcompiler", "-fPIC,-O2,-ffp-contract=off,-fno-fast-math,-pthread,-Wall"]
    if verbose_ptx:
        f += ["-Xptxas", "-v"]
    return f


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src, os.path.join(ROOT, "include", "snn.h")] + [os.path.join(CSRC, h) for h in HEADERS]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s + ".o")
        objs.append(obj)
        if force or _stale(obj, src):
            jobs.append([cc, *_flags(verbose and s.endswith(".cu")), "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"compile failed: {' '.join(cmd)}")
    if force or jobs or not os.path.exists(OUT):
        tmp = OUT + ".tmp"
        cmd = [cc, "-shared", ARCH, "-cudart", "shared", "-o", tmp, *objs,
               "-Xlinker", "-rpath,/usr/local/cuda/lib64", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(OUT)
