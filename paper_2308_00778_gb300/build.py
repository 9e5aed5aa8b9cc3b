"""Build libgsr.so in-tree: every csrc/*.cu compiled for sm_103a in parallel, then linked."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(_HERE, "csrc")
OBJ = os.path.join(_HERE, "_build")
LIB = os.path.join(_HERE, "libgsr.so")
NVCC_FLAGS = ["-gencode=arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr"]


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(extra_flags=None, verbose=False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    flags = NVCC_FLAGS + list(extra_flags or [])

    def one(src):
        obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
        out = _run(["nvcc", *flags, "-c", src, "-o", obj])
        if verbose and out:
            print(out)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(one, srcs))
    _run(["nvcc", "-gencode=arch=compute_103a,code=sm_103a", "-shared", "-o", LIB, *objs])
    return LIB


if __name__ == "__main__":
    import sys

    print(build(verbose="-v" in sys.argv))
