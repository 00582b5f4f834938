"""Compile the FP64 Allen-Cahn oracle (test infrastructure) into a shared library.

The oracle is plain C, built with gcc without FMA contraction so that each
operation rounds as written.  OpenMP is used when the compiler supports it.
Run as ``python -m oracle.build`` or call :func:`build`.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ac_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")

BASE_FLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
              "-std=c11", "-Wall", "-Wextra"]


def _compile(extra: list[str]) -> None:
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", *BASE_FLAGS, *extra, SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, LIB)


def build(force: bool = False) -> str:
    """Build ``_build/liboracle.so`` if missing or older than the source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    try:
        _compile(["-fopenmp"])
    except subprocess.CalledProcessError:
        _compile([])
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
