"""Build libmpcg.so (the C-ABI library) for sm_103a with nvcc.

Usage: python -m paper_2402_12833_gb300.build [--force]

The translation units compile in parallel; the shared library lands next to
this file in ``lib/`` and links the CUDA runtime statically.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "lib")
LIB = os.path.join(OUT, "libmpcg.so")
SOURCES = ["api.cu", "stencil.cu", "stencil_dw.cu", "stencil_sym.cu", "block.cu", "small.cu", "matfree.cu", "ell.cu", "learned.cu", "learned_tc.cu", "learned_train_tc.cu", "learned3_tc.cu",
           "batch.cu", "noalloc.cu", "amg_setup.cpp", "tune.cpp"]
# host-only units: no fused multiply-add contraction, so the hierarchy built on
# the host rounds the same way on every machine
HOST_FLAGS = ["-Xcompiler", "-ffp-contract=off"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libmpcg")
    return path


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(HERE, "..", "include", "mpcg.h"))
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(SRC, src)
        o = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
        objs.append(o)
        # a translation unit that includes another .cu (stencil_dw.cu) depends on it
        with open(s) as f:
            inc = [os.path.join(SRC, ln.split('"')[1]) for ln in f
                   if ln.startswith('#include "') and ln.split('"')[1].endswith(".cu")]
        if force or _stale(o, [s] + headers + inc):
            host = HOST_FLAGS if src.endswith(".cpp") else []
            cmd = [nvcc(), *ARCH, *FLAGS, *host, *(extra or []), "-c", s, "-o", o]
            jobs.append(cmd)
    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stderr
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for err in ex.map(run, jobs):
            if verbose and err:
                print(err)
    if jobs or _stale(LIB, objs):
        run([nvcc(), *ARCH, "-shared", "-o", LIB, *objs])
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
