"""Pins of the CPU oracle against things other than itself.

* aprod 1 / aprod 2 (Eqs. 2-3) against an explicit dense matrix built entry by
  entry (brute force), and the adjoint identity <Ax, y> = <x, A^T y>.
* The Eq. 4 norm against exact math (fsum / hypot) including overflow and
  underflow cases the unscaled form gets wrong.
* The column preconditioner of Alg. 1 against dense column norms.
* LSQR against dense least squares (numpy lstsq of [A~; damp I]), against the
  normal equations (Cholesky of the Gram matrix on config 1), against exact
  recovery of a planted solution, and its residual estimates against the true
  residuals.
"""
import math

import numpy as np
import pytest

import gsrgen
import oracle
from conftest import dense_matrix


def _sys(cfg, fp32=False):
    h = gsrgen.generate(cfg, fp32=fp32)
    return h, oracle.from_host_system(h)


def _dense(h):
    c = h.cfg
    return dense_matrix(h.star_ptr, h.A, h.knot, h.instr, c.n_dfa, c.n_instr, c.n_glob, c.n_astro, c.n_ipr)


CASES = [
    gsrgen.make_cfg(7, 20, 30, 12, 8),             # tiny, fixed obs per star
    gsrgen.make_cfg(21, 13, (1, 37), 9, 6, n_glob=0),  # ragged stars, no global column, n_instr = 6
    gsrgen.make_cfg(22, 4, (3, 5), 4, 7),          # minimal attitude: n_dfa = 4, one knot position
]
# section variants (Sec. 2: 0..5 astrometric and 0..6 instrumental coefficients per row; several
# global unknowns or none): compact rows of n_astro + 12 + n_ipr + n_glob coefficients
VARIANTS = [
    gsrgen.make_cfg(31, 17, (2, 29), 10, 9, n_glob=2, n_astro=3, n_ipr=4),
    gsrgen.make_cfg(32, 11, 20, 8, 5, n_glob=5, n_astro=2, n_ipr=1),
    gsrgen.make_cfg(33, 9, (4, 25), 7, 6, n_glob=0, n_astro=0, n_ipr=6),   # no astrometric section
    gsrgen.make_cfg(34, 14, (1, 30), 9, 0, n_glob=1, n_astro=5, n_ipr=0),  # no instrumental section
    gsrgen.make_cfg(35, 12, 18, 6, 8, n_glob=3, n_astro=5, n_ipr=6),       # the standard row plus 2 globals
]


@pytest.mark.parametrize("cfg", CASES + VARIANTS)
def test_aprod_vs_dense(cfg):
    h, s = _sys(cfg)
    D = _dense(h)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(s.n_cols)
    y0 = rng.standard_normal(s.n_rows)
    y = oracle.aprod1(s, x, y0.copy())
    np.testing.assert_allclose(y, y0 + D @ x, rtol=0, atol=1e-13 * (np.abs(D) @ np.abs(x)).max())
    u = rng.standard_normal(s.n_rows)
    x0 = rng.standard_normal(s.n_cols)
    z = oracle.aprod2(s, u, x0.copy())
    np.testing.assert_allclose(z, x0 + D.T @ u, rtol=0, atol=1e-13 * (np.abs(D.T) @ np.abs(u)).max())


def test_adjoint_identity_c1():
    h, s = _sys(gsrgen.workloads()["c1"].cfg)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(s.n_cols)
    y = rng.standard_normal(s.n_rows)
    Ax = oracle.aprod1(s, x, np.zeros(s.n_rows))
    Aty = oracle.aprod2(s, y, np.zeros(s.n_cols))
    # scale: sum |A_ij x_j y_i|
    absA = oracle.System(s.star_ptr, np.abs(s.A), s.knot, s.instr, s.n_dfa, s.n_instr, s.n_glob)
    scale = float(np.abs(y) @ oracle.aprod1(absA, np.abs(x), np.zeros(s.n_rows)))
    assert abs(math.fsum(Ax * y) - math.fsum(x * Aty)) <= 1e-13 * scale


@pytest.mark.parametrize("sections", [(3, 4, 2), (0, 2, 5), (5, 0, 0)])
def test_adjoint_identity_section_variants(sections):
    na, ni, ng = sections
    c = gsrgen.workloads()["c1"].cfg
    h, s = _sys(gsrgen.make_cfg(c.seed, c.n_stars, (c.obs_min, c.obs_max), c.n_dfa, c.n_instr, n_glob=ng,
                                n_astro=na, n_ipr=ni))
    rng = np.random.default_rng(11)
    x = rng.standard_normal(s.n_cols)
    y = rng.standard_normal(s.n_rows)
    Ax = oracle.aprod1(s, x, np.zeros(s.n_rows))
    Aty = oracle.aprod2(s, y, np.zeros(s.n_cols))
    absA = oracle.System(s.star_ptr, np.abs(s.A), s.knot, s.instr, s.n_dfa, s.n_instr, s.n_glob, na, ni)
    scale = float(np.abs(y) @ oracle.aprod1(absA, np.abs(x), np.zeros(s.n_rows)))
    assert abs(math.fsum(Ax * y) - math.fsum(x * Aty)) <= 1e-13 * scale


def test_norm_eq4():
    rng = np.random.default_rng(2)
    a = rng.standard_normal(1001)
    assert oracle.norm2(a) == pytest.approx(math.sqrt(math.fsum(a * a)), rel=1e-15)
    assert oracle.norm2(np.zeros(5)) == 0.0
    assert oracle.norm2(np.array([-3.0])) == 3.0
    # values whose squares overflow / underflow binary64: the scaled form still works
    assert oracle.norm2(np.array([3e200, 4e200])) == pytest.approx(5e200, rel=1e-15)
    assert oracle.norm2(np.array([3e-200, -4e-200])) == pytest.approx(5e-200, rel=1e-15)
    big = a * 1e300
    assert oracle.norm2(big) == pytest.approx(1e300 * math.sqrt(math.fsum(a * a)), rel=1e-14)


def test_precond_vs_dense_and_empty_column():
    # n_instr = 40 with only 8 rows: some instrumental columns are never hit
    cfg = gsrgen.make_cfg(5, 2, 4, 6, 40)
    h, s = _sys(cfg)
    D = _dense(h)
    norms = np.linalg.norm(D, axis=0)
    assert (norms == 0).any()
    p = oracle.precond(s)
    expect = np.where(norms > 0, 1.0 / np.where(norms > 0, norms, 1.0), 1.0)
    np.testing.assert_allclose(p, expect, rtol=1e-14)


def _lstsq_solution(D, b, damp, precond=True):
    c = D.shape[1]
    norms = np.linalg.norm(D, axis=0)
    p = np.where(norms > 0, 1.0 / np.where(norms > 0, norms, 1.0), 1.0) if precond else np.ones(c)
    M = np.vstack([D * p, damp * np.eye(c)])
    rhs = np.concatenate([b, np.zeros(c)])
    y = np.linalg.lstsq(M, rhs, rcond=None)[0]
    return p * y


@pytest.mark.parametrize("damp", [0.0, 1e-6, 0.3])
@pytest.mark.parametrize("precond", [True, False])
def test_lsqr_vs_dense_lstsq(damp, precond):
    h, s = _sys(gsrgen.make_cfg(7, 20, 30, 12, 8))
    D = _dense(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    x, info = oracle.lsqr(s, b, itnlim=2000, atol=1e-15, btol=1e-15, damp=damp, precond=precond)
    ref = _lstsq_solution(D, b, damp, precond)
    assert info["istop"] in (1, 2, 4, 5)
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("cfg", VARIANTS)
def test_lsqr_section_variants_vs_lstsq(cfg):
    h, s = _sys(cfg)
    D = _dense(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    x, info = oracle.lsqr(s, b, itnlim=5000, atol=1e-15, btol=1e-15, damp=1e-6)
    ref = _lstsq_solution(D, b, 1e-6)
    assert info["istop"] in (1, 2, 4, 5)
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)
    assert s.n_cols == D.shape[1] and s.blocks()["glob"][1] == s.n_cols


def test_lsqr_ragged_vs_lstsq():
    h, s = _sys(gsrgen.make_cfg(21, 13, (6, 37), 9, 6, n_glob=0))
    D = _dense(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    x, info = oracle.lsqr(s, b, itnlim=5000, atol=1e-15, btol=1e-15, damp=1e-6)
    ref = _lstsq_solution(D, b, 1e-6)
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("sections", [(5, 6, 1), (2, 3, 4)])
def test_lsqr_planted_recovery(sections):
    na, ni, ng = sections
    cfg = gsrgen.make_cfg(8, 40, 40, 20, 10, noise_sigma=0.0, n_astro=na, n_ipr=ni, n_glob=ng)
    h, s = _sys(cfg)
    b = oracle.rhs(s, h.x_true, h.eps)
    x, info = oracle.lsqr(s, b, itnlim=2000, atol=1e-15, btol=1e-15, damp=0.0)
    assert info["istop"] in (1, 4)  # consistent system: the residual test stops it
    for name, (a, z) in s.blocks().items():
        assert np.linalg.norm(x[a:z] - h.x_true[a:z]) <= 1e-10 * max(np.linalg.norm(h.x_true[a:z]), 1e-3), name


def test_lsqr_estimates_match_true_residuals():
    h, s = _sys(gsrgen.make_cfg(7, 20, 30, 12, 8))
    b = oracle.rhs(s, h.x_true, h.eps)
    damp = 0.05
    x, info = oracle.lsqr(s, b, itnlim=30, damp=damp)  # fixed iterations, not converged
    r = b - oracle.aprod1(s, x, np.zeros(s.n_rows))
    p = oracle.precond(s)
    y = x / p
    # r2norm = sqrt(|r|^2 + damp^2 |y|^2), r1norm = |r|, arnorm = |A~^T r - damp^2 y|
    assert info["r1norm"] == pytest.approx(np.linalg.norm(r), rel=1e-8)
    assert info["r2norm"] == pytest.approx(math.sqrt(np.linalg.norm(r) ** 2 + damp ** 2 * y @ y), rel=1e-8)
    g = p * oracle.aprod2(s, r, np.zeros(s.n_cols)) - damp ** 2 * y
    assert info["arnorm"] == pytest.approx(np.linalg.norm(g), rel=1e-6)
    assert info["xnorm"] == pytest.approx(np.linalg.norm(y), rel=1e-8)
    assert info["istop"] == 7 and info["itn"] == 30
    D = _dense(h)
    assert info["anorm"] <= np.linalg.norm(np.vstack([D * p, damp * np.eye(s.n_cols)]), "fro") * (1 + 1e-12)


def test_lsqr_c1_normal_equations():
    w = gsrgen.workloads()["c1"]
    h, s = _sys(w.cfg)
    b = oracle.rhs(s, h.x_true, h.eps)
    x, info = oracle.lsqr(s, b, w.itnlim, w.atol, w.btol, 1e12, w.damp)
    assert info["istop"] in (1, 2)
    p = oracle.precond(s)
    # Gram matrix of A~ from per-row outer products (24 entries per row)
    n = s.n_cols
    a0 = 5 * s.n_stars
    i0 = a0 + 3 * s.n_dfa
    star = np.repeat(np.arange(s.n_stars), np.diff(s.star_ptr))
    cols = np.empty((s.n_rows, 24), dtype=np.int64)
    cols[:, :5] = 5 * star[:, None] + np.arange(5)
    for ax in range(3):
        cols[:, 5 + 4 * ax:9 + 4 * ax] = a0 + ax * s.n_dfa + s.knot[:, None] + np.arange(4)
    cols[:, 17:23] = i0 + s.instr
    cols[:, 23] = i0 + s.n_instr
    vals = s.A * p[cols]
    G = np.zeros((n, n))
    np.add.at(G, (np.repeat(cols, 24, axis=1).ravel(), np.tile(cols, (1, 24)).ravel()),
              (vals[:, :, None] * vals[:, None, :]).ravel())
    G += w.damp ** 2 * np.eye(n)
    rhs = np.zeros(n)
    np.add.at(rhs, cols.ravel(), (vals * b[:, None]).ravel())
    L = np.linalg.cholesky(G)
    y_ref = np.linalg.solve(L.T, np.linalg.solve(L, rhs))
    x_ref = p * y_ref
    for name, (a, z) in s.blocks().items():
        err = np.linalg.norm(x[a:z] - x_ref[a:z]) / max(np.linalg.norm(x_ref[a:z]), 1e-3)
        assert err <= 1e-10, (name, err)


def test_lsqr_itnlim_and_zero_rhs():
    h, s = _sys(gsrgen.make_cfg(7, 20, 30, 12, 8))
    x, info = oracle.lsqr(s, np.zeros(s.n_rows), itnlim=10)
    assert info["istop"] == 0 and info["itn"] == 0 and not x.any()
    b = oracle.rhs(s, h.x_true, h.eps)
    x, info = oracle.lsqr(s, b, itnlim=3)
    assert info["istop"] == 7 and info["itn"] == 3


def test_oracle_matches_stored_c1_values():
    """Regression pin: tests/golden/c1_oracle.json (written by tests/golden/make_golden.py)."""
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "c1_oracle.json")) as f:
        g = json.load(f)
    w = gsrgen.workloads()["c1"]
    h, s = _sys(w.cfg)
    b = oracle.rhs(s, h.x_true, h.eps)
    np.testing.assert_allclose(b[:8], g["b_head"], rtol=1e-13)
    x, info = oracle.lsqr(s, b, w.itnlim, w.atol, w.btol, 1e12, w.damp)
    assert info["itn"] == g["converged"]["info"]["itn"] and info["istop"] == g["converged"]["info"]["istop"]
    for k, (a, z) in s.blocks().items():
        np.testing.assert_allclose(x[a:a + 6], g["converged"]["x_head"][k], rtol=1e-11, atol=1e-13)
