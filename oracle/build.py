"""Build the oracle shared library (plain C, FP64, OpenMP) in-tree under ``oracle/_build``.

Test infrastructure: the CUDA library never links or loads it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "feod_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False, verbose: bool = False, plant: int = 0) -> str:
    """Compile ``liboracle.so`` if it is missing or older than its source; return its path.

    ``plant`` > 0 builds a deliberately wrong variant (``liboracle_plantN.so``) for the test that
    checks the pins catch mistakes; the regular oracle always has ``plant == 0``.
    """
    lib = LIB if plant == 0 else os.path.join(OUT_DIR, f"liboracle_plant{plant}.so")
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-Wall", "-Wno-unknown-pragmas", f"-DORC_PLANT={int(plant)}", SRC, "-o", tmp, "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
