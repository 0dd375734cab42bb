"""Compile the CUDA library ``libff.so`` in-tree for sm_103a (GB300)."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
SOURCES = [os.path.join(CSRC, "ff.cu")]
DEPS = SOURCES + [os.path.join(CSRC, h) for h in ("ff_kernels.cuh", "ff_sweep.cuh", "ff_seed.cuh",
                                                  "ff_wht_tc.cuh", "ff_seed_tc.cuh",
                                                  "ff_peaks.cuh")] \
    + [os.path.join(ROOT, "include", "ff.h")]
LIB = os.path.join(HERE, "libff.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libff.so")


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    m = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= m for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-cudart", "shared", "-I", os.path.join(ROOT, "include"), "-o", tmp, *SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
