"""Record, for a named workload, the oracle's LSQR iteration count that first
brings every block within 1e-9 of its tightly converged solution (calls only
gsrgen + oracle). The benchmark's reference arm (the oracle timed on the host)
reads it to extrapolate a bounded sample to a whole solve.

The coefficients are rounded to binary32 once, as in the benchmark. Block
error: |x_blk - x*_blk| / max(|x*_blk|, 1e-3) for astro / attitude /
instrumental / global.

    python tests/golden/make_itn.py [workload]      # default c2
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gsrgen  # noqa: E402
import oracle  # noqa: E402

TOL = 1e-9


def block_err(x, ref, s):
    worst = 0.0
    for a, z in s.blocks().values():
        if z > a:
            worst = max(worst, np.linalg.norm(x[a:z] - ref[a:z]) / max(np.linalg.norm(ref[a:z]), 1e-3))
    return worst


def main():
    name = sys.argv[1] if len(sys.argv) > 1 else "c2"
    w = gsrgen.workloads()[name]
    h = gsrgen.generate(w.cfg, fp32=True)
    s = oracle.from_host_system(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    t0 = time.time()
    xs, info = oracle.lsqr(s, b, 400, 1e-15, 1e-15, 0.0, w.damp)

    def err(k):
        x, _ = oracle.lsqr(s, b, k, 0.0, 0.0, 0.0, w.damp)
        return block_err(x, xs, s)

    hi = 8
    while err(hi) > TOL and hi < info["itn"]:
        hi *= 2
    lo = hi // 2
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if err(mid) <= TOL:
            hi = mid
        else:
            lo = mid
    out = {"workload": name, "rows": s.n_rows, "cols": s.n_cols, "damp": w.damp,
           "reference": {"atol": 1e-15, "btol": 1e-15, "itn": info["itn"], "istop": info["istop"]},
           "itn_to_1e-9": hi, "seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, f"{name}_oracle_itn.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
