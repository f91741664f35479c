"""Compile the C part of the oracle (gcc, no CUDA) into oracle/_build/."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libargus_oracle.so")
SOURCES = ["kalman.c", "gwb.c"]
HEADERS = ["kf_body.h", "ou_phi.h", "gwb_body.h"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in SOURCES + HEADERS)


def build(force: bool = False) -> str:
    if force or _stale():
        os.makedirs(OUT_DIR, exist_ok=True)
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-D_GNU_SOURCE", "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
