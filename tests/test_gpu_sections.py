"""Section variants on the GPU against the CPU oracle.

Sec. 2 allows 0 to 5 astrometric and 0 to 6 instrumental coefficients per
row beside the 12 attitude ones, and a global section or none; Sec. 4.2 runs
systems with five global unknowns. A context made by gsr_create_sections for
such a choice stores compact tiles and runs the kernels' run-time-geometry
instances. The bars are those of the standard-row tests:
* aprod 1 / aprod 2 (binary64 arithmetic): per element |gpu - oracle| <=
  1e-13 (sum of |terms| + |oracle|);
* the binary32 inner kernels: 25 u and 2e3 u of the sum of |terms|
  (u = 2^-24), the double-float residual u |r| + 2^-40 sum|terms|;
* LSQR at a fixed iteration count and converged: 1e-10 per block;
* mixed precision and warm-started solves: 1e-9 per block against the
  oracle's converged solution.
Cases cover no astrometric section, no instrumental section, five globals,
empty and single-row stars, accumulators too large for shared memory and
32-bit instrumental planes; the LSQR cases have at least ten observations per
star (fewer than n_astro make a star's block rank deficient).
"""
import ctypes

import numpy as np
import pytest
import torch

import gsrgen
import oracle
import paper_2308_00778_gb300 as g
from gpu_util import abs_system, block_errors, context_for

pytestmark = pytest.mark.gpu

APROD_CASES = {
    "a3_i4_g2": gsrgen.make_cfg(141, 300, (1, 80), 60, 40, n_glob=2, n_astro=3, n_ipr=4),
    "a0_i6_g0": gsrgen.make_cfg(142, 200, 50, 40, 30, n_glob=0, n_astro=0, n_ipr=6),
    "a5_i0_g1_empty_stars": gsrgen.make_cfg(143, 250, (0, 60), 50, 0, n_glob=1, n_astro=5, n_ipr=0),
    "a2_i1_g5": gsrgen.make_cfg(144, 400, 40, 30, 9, n_glob=5, n_astro=2, n_ipr=1),
    "a5_i6_g5_many_tiles": gsrgen.make_cfg(145, 3000, (20, 200), 300, 200, n_glob=5),
    "a4_i6_g3_wide": gsrgen.make_cfg(146, 500, 100, 9000, 20000, n_glob=3, n_astro=4, n_ipr=6),
    "a1_i2_g0_instr32": gsrgen.make_cfg(147, 1200, 100, 80, 70000, n_glob=0, n_astro=1, n_ipr=2),
}
SOLVE_CASES = {
    "a3_i4_g2": gsrgen.make_cfg(151, 400, (10, 90), 40, 25, n_glob=2, n_astro=3, n_ipr=4),
    "a0_i6_g0": gsrgen.make_cfg(152, 300, (10, 60), 30, 20, n_glob=0, n_astro=0, n_ipr=6),
    "a5_i0_g1": gsrgen.make_cfg(153, 300, (10, 80), 30, 0, n_glob=1, n_astro=5, n_ipr=0),
    "a5_i6_g5": gsrgen.make_cfg(154, 500, (10, 120), 50, 30, n_glob=5, att_kind=1),
}


def _setup(cfg, fp32=False, rhs=True):
    h = gsrgen.generate(cfg, fp32=fp32)
    s = oracle.from_host_system(h)
    b = oracle.rhs(s, h.x_true, h.eps) if rhs else None
    ctx = context_for(h, fp32=fp32)
    ctx.set_system(h.A32 if fp32 else h.A, h.knot, h.instr, b)
    return h, s, b, ctx


def _check(got, want, scale, tol=1e-13):
    err = np.abs(got - want)
    bound = tol * (scale + np.abs(want)) + 1e-300
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3g}"


@pytest.mark.parametrize("name", sorted(APROD_CASES))
@pytest.mark.parametrize("fp32", [False, True])
def test_aprod_sections_vs_oracle(name, fp32):
    cfg = APROD_CASES[name]
    h, s, _, ctx = _setup(cfg, fp32, rhs=False)
    assert (ctx.n_astro, ctx.n_ipr, ctx.n_glob) == (cfg.n_astro, cfg.n_ipr, cfg.n_glob)
    assert ctx.row_width == cfg.npar and ctx.n_cols == s.n_cols
    rng = np.random.default_rng(3)
    x = rng.standard_normal(s.n_cols)
    y0 = rng.standard_normal(s.n_rows)
    yd = torch.tensor(y0, device="cuda")
    ctx.aprod1(torch.tensor(x, device="cuda"), yd)
    _check(yd.cpu().numpy(), oracle.aprod1(s, x, y0.copy()), oracle.aprod1(abs_system(s), np.abs(x), np.abs(y0)))
    u = rng.standard_normal(s.n_rows)
    z0 = rng.standard_normal(s.n_cols)
    zd = torch.tensor(z0, device="cuda")
    ctx.aprod2(torch.tensor(u, device="cuda"), zd)
    _check(zd.cpu().numpy(), oracle.aprod2(s, u, z0.copy()), oracle.aprod2(abs_system(s), np.abs(u), np.abs(z0)))
    ctx.close()


@pytest.mark.parametrize("name", sorted(APROD_CASES))
def test_binary32_kernels_sections(name):
    cfg = APROD_CASES[name]
    h, s, b, ctx = _setup(cfg, fp32=True)
    u = 2.0 ** -24
    rng = np.random.default_rng(9)
    x = rng.standard_normal(s.n_cols).astype(np.float32).astype(np.float64)
    y0 = rng.standard_normal(s.n_rows).astype(np.float32).astype(np.float64)
    yd = torch.tensor(y0, dtype=torch.float32, device="cuda")
    ctx.aprod1_f32(torch.tensor(x, dtype=torch.float32, device="cuda"), yd)
    want = oracle.aprod1(s, x, y0.copy())
    scale = oracle.aprod1(abs_system(s), np.abs(x), np.abs(y0).copy())
    assert np.all(np.abs(yd.cpu().numpy() - want) <= 25 * u * scale)
    z0 = rng.standard_normal(s.n_cols)
    zd = torch.tensor(z0, device="cuda")
    ctx.aprod2_f32(torch.tensor(y0, dtype=torch.float32, device="cuda"), zd)
    want2 = oracle.aprod2(s, y0, z0.copy())
    scale2 = oracle.aprod2(abs_system(s), np.abs(y0), np.abs(z0).copy())
    assert np.all(np.abs(zd.cpu().numpy() - want2) <= 2e3 * u * scale2)
    xs = rng.standard_normal(s.n_cols)
    rd = torch.zeros(s.n_rows, dtype=torch.float32, device="cuda")
    ctx.residual(torch.tensor(xs, device="cuda"), rd)
    r_ref = b - oracle.aprod1(s, xs, np.zeros(s.n_rows))
    rscale = oracle.aprod1(abs_system(s), np.abs(xs), np.abs(b).copy())
    assert np.all(np.abs(rd.cpu().numpy() - r_ref) <= u * np.abs(r_ref) + 2.0 ** -40 * rscale)
    ctx.close()


@pytest.mark.parametrize("name", sorted(SOLVE_CASES))
@pytest.mark.parametrize("fp32", [False, True])
def test_lsqr_sections_vs_oracle(name, fp32):
    """Binary64 LSQR (on binary64 or binary32 storage): the iterate at 12 iterations (a small
    system may meet a machine-precision stop test first: both sides then stop at the same
    iteration) and the converged solution."""
    cfg = SOLVE_CASES[name]
    h, s, b, ctx = _setup(cfg, fp32)
    x = np.zeros(s.n_cols)
    info = ctx.solve(x, itnlim=12, atol=0.0, btol=0.0, conlim=0.0, damp=1e-6)
    xo, io = oracle.lsqr(s, b, 12, 0.0, 0.0, 0.0, 1e-6)
    assert info["itn"] == io["itn"] and info["istop"] == io["istop"], (info, io)
    for k, e in block_errors(x, xo, s).items():
        assert e <= 1e-10, (k, e)
    for key in ("r1norm", "anorm", "arnorm", "xnorm"):
        assert info[key] == pytest.approx(io[key], rel=1e-9), key
    xc = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
    ctx.solve(xc, itnlim=3000, atol=1e-14, btol=1e-14, conlim=0.0, damp=1e-6)
    xoc, _ = oracle.lsqr(s, b, 3000, 1e-14, 1e-14, 0.0, 1e-6)
    for k, e in block_errors(xc.cpu().numpy(), xoc, s).items():
        assert e <= 1e-10, (k, e)
    ctx.close()


@pytest.mark.parametrize("name", sorted(SOLVE_CASES))
def test_mixed_and_warm_sections_vs_oracle(name):
    """Mixed precision from x0 = 0, from the Jacobi start and from the learned start (the shipped
    network), and the binary64 solve from the learned start: every block within 1e-9 of the oracle's
    converged solution of the same (binary32-rounded) values."""
    cfg = SOLVE_CASES[name]
    h, s, b, ctx = _setup(cfg, fp32=True)
    xo, _ = oracle.lsqr(s, b, 3000, 1e-14, 1e-14, 0.0, 1e-6)
    learned = dict(warm=g.GSR_WARM_LEARNED, weights_path=g.WARM_WEIGHTS)
    for kw in (dict(mode=g.GSR_MIXED), dict(mode=g.GSR_MIXED, warm=g.GSR_WARM_JACOBI), dict(mode=g.GSR_MIXED, **learned),
               dict(itnlim=3000, atol=1e-14, btol=1e-14, conlim=0.0, **learned)):
        x = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
        info = ctx.solve(x, damp=1e-6, **kw)
        errs = block_errors(x.cpu().numpy(), xo, s)
        assert max(errs.values()) <= 1e-9, (kw, errs, info)
    ctx.close()


@pytest.mark.parametrize("fp32", [False, True])
def test_warm_start_astro_solve_sections(fp32):
    """The warm start's per-star solve has n_astro unknowns per star: against the oracle's
    n_astro x n_astro solve given the same attitude, instrumental and global parts."""
    cfg = gsrgen.make_cfg(155, 800, (10, 90), 60, 30, n_glob=3, n_astro=3, n_ipr=2, att_kind=1)
    h, s, b, ctx = _setup(cfg, fp32)
    x0 = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
    ctx.warm_start(x0)
    got = x0.cpu().numpy()
    a0 = s.blocks()["att"][0]
    ref = np.zeros(s.n_cols)
    ref[a0:] = got[a0:]
    assert oracle.astro_solve(s, b, ref) == 0
    bar = 1e-4 if fp32 else 1e-12  # binary32 / binary64 normal equations (as in test_gpu_warm.py)
    for st in range(cfg.n_stars):
        r, gg = ref[3 * st:3 * st + 3], got[3 * st:3 * st + 3]
        assert np.linalg.norm(gg - r) <= bar * np.linalg.norm(r) + bar * 1e-5, st
    ctx.close()


@pytest.mark.parametrize("n_glob", [0, 1])
def test_create_sections_with_the_standard_sections(n_glob):
    """gsr_create_sections with 5 astrometric, 6 instrumental and at most one global takes compact
    rows (23 or 24 coefficients) and runs the standard tiles: its aprods equal gsr_create's bit for
    bit on the same rows."""
    cfg = gsrgen.make_cfg(156, 700, (1, 90), 50, 40, n_glob=n_glob)
    h = gsrgen.generate(cfg)
    ref = context_for(h)
    ref.set_system(h.A, h.knot, h.instr)
    L = g.lib()
    hh = ctypes.c_void_p()
    sp = np.ascontiguousarray(h.star_ptr)
    assert L.gsr_create_sections(ctypes.byref(hh), cfg.n_stars, 0, sp.ctypes.data, 5, cfg.n_dfa, cfg.n_instr, 6,
                                 n_glob, g.GSR_FP64, 0) == 0
    w = 23 + n_glob
    A = np.ascontiguousarray(h.A[:, :w])
    assert g.gsr_set_system(hh.value, A.ctypes.data, 0, h.knot.ctypes.data, h.instr.ctypes.data, 0, g.GSR_HOST) == 0
    assert g.gsr_sections(hh.value) == (0, 5, 6, n_glob, w)
    rng = np.random.default_rng(4)
    x = torch.tensor(rng.standard_normal(ref.n_cols), device="cuda")
    y1 = torch.zeros(ref.n_rows, dtype=torch.float64, device="cuda")
    y2 = torch.zeros_like(y1)
    ref.aprod1(x, y1)
    assert g.gsr_aprod1(hh.value, x.data_ptr(), y2.data_ptr()) == 0
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    g.gsr_destroy(hh.value)
    ref.close()


def test_sections_argument_errors():
    h = gsrgen.generate(APROD_CASES["a3_i4_g2"])
    ctx = context_for(h)
    with pytest.raises(g.GsrError) as e:  # a value out of range is rejected before anything is stored
        bad = h.instr.copy()
        bad[5, 3] = h.cfg.n_instr
        ctx.set_system(h.A, h.knot, bad)
    assert e.value.status == g.Status.EINVAL
    ctx.close()
    # no instrumental section: instr_col may be NULL
    h0 = gsrgen.generate(APROD_CASES["a5_i0_g1_empty_stars"])
    c0 = context_for(h0)
    assert g.gsr_set_rows(c0.h, 0, c0.n_rows, h0.A.ctypes.data, 0, g.GSR_AOS, 0, h0.knot.ctypes.data, 0,
                          g.GSR_HOST) == 0
    c0.close()
