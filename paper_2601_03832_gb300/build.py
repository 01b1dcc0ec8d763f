"""Builds the in-tree CUDA libraries for sm_103a with nvcc (no CMake).

libgrover_mps.so   the iterative-Grover engine behind include/grover_mps.h
libgmps_peaks.so   peak-rate microbenchmarks behind include/gmps_peaks.h

Every translation unit is compiled in parallel, then each library is linked
next to this file.  Run: python -m paper_2601_03832_gb300.build
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
SOURCES = ["gmps_form_c128.cu", "gmps_form_c64.cu", "gmps_form_dw.cu", "gmps_launch.cu", "gmps_capi.cu", "gmps_sv.cu"]
LIB = os.path.join(HERE, "libgrover_mps.so")
PEAK_SOURCES = ["gmps_peaks.cu"]
PEAK_LIB = os.path.join(HERE, "libgmps_peaks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(lib, deps):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link both libraries if any source changed; returns the
    engine library's path."""
    objdir = os.path.join(ROOT, "_build")
    os.makedirs(objdir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers += [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]
    libs = [(LIB, [os.path.join(CSRC, x) for x in SOURCES]),
            (PEAK_LIB, [os.path.join(CSRC, x) for x in PEAK_SOURCES])]
    todo = [(lib, srcs) for lib, srcs in libs if force or _stale(lib, srcs + headers)]
    if not todo:
        return LIB
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    all_srcs = [src for _, srcs in todo for src in srcs]
    with ThreadPoolExecutor(max_workers=len(all_srcs)) as ex:
        objs = dict(zip(all_srcs, ex.map(compile_one, all_srcs)))
    for lib, srcs in todo:
        tmp = lib + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[objs[x] for x in srcs], "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
