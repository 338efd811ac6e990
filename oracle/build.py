"""Compile the C oracle (test infrastructure) into oracle/libptsne_oracle.so."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ptsne_oracle.c")
LIB = os.path.join(HERE, "libptsne_oracle.so")


def build(force: bool = False) -> str:
    alt = os.environ.get("PTSNE_ORACLE_LIB")
    if alt:  # a separately built copy (used to check that the pins catch planted mistakes)
        return alt
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-Wno-unused-parameter", SRC, "-o", LIB, "-lm"]
    subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
