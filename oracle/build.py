"""Compile the C oracle into ``oracle/libffo.so`` (test infrastructure only)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ffo.c")
HDR = os.path.join(HERE, "ffo.h")
LIB = os.path.join(HERE, "libffo.so")


def build(force: bool = False) -> str:
    """Build the shared library if it is missing or older than its sources."""
    if not force and os.path.exists(LIB):
        lib_m = os.path.getmtime(LIB)
        if lib_m >= os.path.getmtime(SRC) and lib_m >= os.path.getmtime(HDR):
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-ffp-contract=off", "-o", tmp, SRC, "-lpthread", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
