"""Builds libppl.so (the sm_103a CUDA library behind include/ppl.h) in-tree with nvcc."""
from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libppl.so")
# translation unit -> extra nvcc flags; the FP32 step uses approximate division and
# square root (its error is budgeted against the FP64 oracle), the FP64 step is IEEE
UNITS = {
    "ppl.cu": [],
    "tools.cu": [],
    "thermo.cu": [],
    "adjoint.cu": [],
    "step_fp64.cu": [],
    "step_fp32.cu": ["--use_fast_math"],
    "batch_persist.cu": ["--use_fast_math"],
    "step_tangent.cu": [],
    "step_tangent32.cu": ["--use_fast_math"],
}
SOURCES = [os.path.join(CSRC, u) for u in UNITS]
DEPS = SOURCES + [os.path.join(CSRC, h) for h in ("common.cuh", "dual.cuh", "lane2.cuh", "row_step.cuh", "row_step_pair.cuh", "sim.cuh", "step_variants.h")] + [
    os.path.join(ROOT, "include", "ppl.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libppl")
    return cand


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile libppl.so if it is missing or older than its sources; return its path."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    nvcc = nvcc_path()
    common = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC"]
    objs, procs = [], []
    for unit, extra in UNITS.items():
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        cmd = [nvcc, *common, *extra, "-c", os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append(subprocess.Popen(cmd))
        objs.append(obj)
    if any(p.wait() != 0 for p in procs):
        raise RuntimeError("nvcc failed")
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
