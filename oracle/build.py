"""Compile the FP64 CPU oracle (test infrastructure) into oracle/_build/liboracle.so.

Plain gcc, -O2 without fast-math so that IEEE double arithmetic is kept,
OpenMP for the site loops. Run as a script or through build().
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = [os.path.join(HERE, "wilson_oracle.c"), os.path.join(HERE, "heatbath.c")]
HEADERS = [os.path.join(HERE, "wilson_oracle.h"), os.path.join(HERE, "heatbath.h")]


def build(force: bool = False) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    newest_src = max(os.path.getmtime(p) for p in SOURCES + HEADERS)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest_src:
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp] + SOURCES + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
