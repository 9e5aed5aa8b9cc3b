"""Build liboracle.so: plain C, binary64 without FMA contraction. Everything is single-threaded except
oracle_omp.c (the all-cores baseline), built with OpenMP when the compiler has it."""
from __future__ import annotations

import glob
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def build() -> str:
    out = os.path.join(_HERE, "liboracle.so")
    srcs = sorted(glob.glob(os.path.join(_HERE, "*.c")))
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-o", out]
    r = subprocess.run(base + ["-fopenmp", *srcs, "-lm"], capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP: oracle_omp_threads() then reports one thread
        r = subprocess.run(base + [*srcs, "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stdout + r.stderr)
    return out


if __name__ == "__main__":
    print(build())
