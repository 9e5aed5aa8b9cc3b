"""Build the generator's host library (gcc) and device twin (nvcc, sm_103a)."""
from __future__ import annotations

import os
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)


def build_host() -> str:
    out = os.path.join(_HERE, "libgsrgen_host.so")
    src = os.path.join(_HERE, "gsrgen_host.c")
    _run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp", "-o", out, src, "-lm"])
    return out


def build_dev() -> str:
    out = os.path.join(_HERE, "libgsrgen_dev.so")
    src = os.path.join(_HERE, "gsrgen_dev.cu")
    _run(["nvcc", ARCH, "-O3", "-fmad=false", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-o", out, src])
    return out


def build() -> None:
    build_host()
    build_dev()


if __name__ == "__main__":
    build()
    print("built", file=sys.stderr)
