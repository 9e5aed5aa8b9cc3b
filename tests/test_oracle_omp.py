"""The all-cores oracle (oracle/oracle_omp.c) against the single-threaded oracle.

aprod 1 splits whole rows over threads, so it is bitwise the single-threaded
product; aprod 2 and the norms sum in another order, so they agree to
rounding (1e-13 of the sum of |terms| for the products); the LSQR solve on
config 1 then matches the single-threaded solve per block to 1e-10.
"""
import numpy as np
import pytest

import gsrgen
import oracle


def _abs_sys(s):
    return oracle.System(s.star_ptr, np.abs(s.A), s.knot, s.instr, s.n_dfa, s.n_instr, s.n_glob,
                         n_astro=s.n_astro, n_ipr=s.n_ipr)


@pytest.mark.parametrize("sections", [(5, 6, 1), (3, 2, 4)])
def test_omp_aprods_vs_single_thread(sections):
    na, ni, ng = sections
    cfg = gsrgen.make_cfg(31, 700, (1, 90), 40, 25, n_astro=na, n_ipr=ni, n_glob=ng)
    h = gsrgen.generate(cfg)
    s = oracle.from_host_system(h)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(s.n_cols)
    y = rng.standard_normal(s.n_rows)
    y0 = rng.standard_normal(s.n_rows)
    np.testing.assert_array_equal(oracle.aprod1_omp(s, x, y0.copy()), oracle.aprod1(s, x, y0.copy()))
    x0 = rng.standard_normal(s.n_cols)
    got = oracle.aprod2_omp(s, y, x0.copy())
    ref = oracle.aprod2(s, y, x0.copy())
    mag = oracle.aprod2(_abs_sys(s), np.abs(y), np.abs(x0).copy())
    assert np.all(np.abs(got - ref) <= 1e-13 * mag)


def test_omp_lsqr_vs_single_thread_c1():
    w = gsrgen.workloads()["c1"]
    h = gsrgen.generate(w.cfg)
    s = oracle.from_host_system(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    x1, i1 = oracle.lsqr(s, b, 200, 1e-12, 1e-12, 0.0, w.damp)
    xo, io = oracle.lsqr_omp(s, b, 200, 1e-12, 1e-12, 0.0, w.damp)
    assert abs(io["itn"] - i1["itn"]) <= 1
    for a, z in s.blocks().values():
        if z > a:
            d = np.linalg.norm(xo[a:z] - x1[a:z]) / max(np.linalg.norm(x1[a:z]), 1e-3)
            assert d <= 1e-10, (a, z, d)
    assert oracle.omp_threads() >= 1
