"""Build liboracle.so: plain C, single-threaded, binary64 without FMA contraction."""
from __future__ import annotations

import glob
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def build() -> str:
    out = os.path.join(_HERE, "liboracle.so")
    srcs = sorted(glob.glob(os.path.join(_HERE, "*.c")))
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-o", out,
           *srcs, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stdout + r.stderr)
    return out


if __name__ == "__main__":
    print(build())
