"""Write the stored oracle values under tests/golden/ (calls only gsrgen + oracle).

The paper prints no worked numeric example (its systems are proprietary Gaia
data), so the stored values here are the oracle's own results on the
synthetic config-1 system: a regression pin on the oracle. Any later change
to them must name, in its commit message, the passage of the paper (or the
reading of it) that justifies the change.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gsrgen  # noqa: E402
import oracle  # noqa: E402


def main():
    w = gsrgen.workloads()["c1"]
    h = gsrgen.generate(w.cfg)
    s = oracle.from_host_system(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    out = {"workload": "c1: 1,000 stars x 100 obs, 100 knots/axis, 60 instr, 1 global, seed 0, damp 1e-6",
           "b_head": b[:8].tolist()}
    x, info = oracle.lsqr(s, b, w.itnlim, w.atol, w.btol, 1e12, w.damp)
    out["converged"] = {"info": info, "x_head": {k: x[a:a + 6].tolist() for k, (a, z) in s.blocks().items()}}
    x50, info50 = oracle.lsqr(s, b, 10, 0.0, 0.0, 0.0, w.damp)
    out["itn10"] = {"info": info50, "x_head": {k: x50[a:a + 6].tolist() for k, (a, z) in s.blocks().items()}}
    with open(os.path.join(HERE, "c1_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
