"""The benchmark's acceptance arithmetic on the host: the parameter blocks, the 1e-9 per-block
relative error that decides when a solver leg has converged, and the consistency ratio q of
Eq. 5 between a solution and the binary64 reference."""
import math
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
import gsrgen  # noqa: E402


def test_block_ranges_follow_the_unknown_order():
    c = gsrgen.workloads()["c2"].cfg
    r = bench.block_ranges(c)
    assert r == {"astro": (0, 500000), "att": (500000, 509000), "instr": (509000, 510000), "glob": (510000, 510001)}
    assert r["glob"][1] == c.ncols()
    v = gsrgen.workloads()["c2a2"].cfg  # 2 astrometric unknowns per star, no global
    rv = bench.block_ranges(v)
    assert rv["astro"] == (0, 2 * v.n_stars) and rv["glob"][0] == rv["glob"][1] == v.ncols()


def test_max_block_err_is_the_worst_block_relative_norm():
    c = gsrgen.make_cfg(0, 10, 20, 8, 6, n_glob=1)
    r = bench.block_ranges(c)
    rng = np.random.default_rng(3)
    ref = torch.tensor(rng.standard_normal(c.ncols()))
    x = ref.clone()
    a, z = r["att"]
    d = torch.zeros(c.ncols(), dtype=torch.float64)
    d[a:z] = torch.tensor(rng.standard_normal(z - a)) * 1e-7
    x += d
    want = float(torch.linalg.vector_norm(d[a:z]) / torch.linalg.vector_norm(ref[a:z]))
    # x = ref + d rounds each entry by up to 2^-53 |ref| (~1e-16 against d ~ 1e-7)
    assert math.isclose(bench.max_block_err(x, ref, c), want, rel_tol=1e-8)
    # a block whose reference is (near) zero is measured against 1e-3, not against its own norm
    ref2 = ref.clone()
    g0, g1 = r["glob"]
    ref2[g0:g1] = 0.0
    x2 = ref2.clone()
    x2[g0:g1] = 2e-12
    assert math.isclose(bench.max_block_err(x2, ref2, c), 2e-12 / 1e-3, rel_tol=1e-12)
    assert bench.max_block_err(ref, ref, c) == 0.0


def test_eq5_q_per_section():
    c = gsrgen.make_cfg(0, 10, 20, 8, 6, n_glob=1)
    r = bench.block_ranges(c)
    n = c.ncols()
    xr = torch.zeros(n, dtype=torch.float64)
    se = torch.full((n,), 0.5, dtype=torch.float64)
    x = xr.clone()
    i0 = r["instr"][0] + 2
    x[i0] = 0.3  # q = 0.3 / sqrt(0.5^2 + 0.5^2)
    q = bench.eq5_q(x, xr, se, c)
    assert set(q) == {"astro", "att", "instr", "glob"}
    assert math.isclose(q["instr"], 0.3 / math.sqrt(0.5), rel_tol=1e-12)
    assert q["astro"] == q["att"] == q["glob"] == 0.0
