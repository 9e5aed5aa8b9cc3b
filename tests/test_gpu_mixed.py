"""Mixed precision (binary32 inner LSQR, binary64 refinement) against binary64 solutions.

Both sides solve the same system: coefficients rounded to binary32 once, the
binary64 references use exactly those values widened. Bar: every block
within 1e-9 relative (|x_blk - ref_blk| / max(|ref_blk|, 1e-3)) of the
binary64 solution. The refinement converges to the least-squares solution of
the undamped problem; with damp 1e-6 the damped reference differs by
O(damp^2) ~ 1e-12, far below the bar.
"""
import numpy as np
import pytest
import torch

import gsrgen
import oracle
import paper_2308_00778_gb300 as g
from gpu_util import block_errors, context_for

pytestmark = pytest.mark.gpu


def _setup32(cfg):
    h = gsrgen.generate(cfg, fp32=True)
    s = oracle.from_host_system(h)  # h.A holds the binary32-rounded values, widened
    b = oracle.rhs(s, h.x_true, h.eps)
    ctx = context_for(h, fp32=True)
    ctx.set_system(h.A32, h.knot, h.instr, b)
    return h, s, b, ctx


def test_mixed_c1_vs_oracle():
    w = gsrgen.workloads()["c1"]
    h, s, b, ctx = _setup32(w.cfg)
    x = np.zeros(s.n_cols)
    info = ctx.solve(x, mode=g.GSR_MIXED, damp=w.damp)
    xo, io = oracle.lsqr(s, b, 500, 1e-14, 1e-14, 0.0, w.damp)
    errs = block_errors(x, xo, s)
    assert max(errs.values()) <= 1e-9, (errs, info)
    assert 2 <= info["outer_itn"] <= 6, info
    ctx.close()


@pytest.mark.parametrize("name,fused", [("ragged_sinusoid", 0), ("wide_instr_global", 1), ("wide_instr_global", -1),
                                        ("wide_ragged_instr_global", 1), ("wide_ragged_instr_global", -1)])
def test_mixed_vs_plain_fp64_on_gpu(name, fused):
    """Mixed solves against the binary64-arithmetic GPU solve of the same stored values. The wide
    cases (60,000 attitude columns: the attitude products go to the L2 window reductions) run the inner
    iterations both as one fused pass per iteration (inner_fused 1: aprod 1 and aprod 2 from one read
    of each tile) and as the two separate passes (-1); the ragged one has stars of 10 to 300 rows, so
    tiles hold many stars and a warp's range ends inside stars (at least 10 rows a star: with fewer
    than 5 a star's astrometric unknowns are not determined by its rows, and the refinement's
    undamped fixed point and the damped reference may differ in them by far more than 1e-9)."""
    cfg = {"ragged_sinusoid": gsrgen.make_cfg(51, 20000, (50, 150), 1500, 300, att_kind=1),
           "wide_instr_global": gsrgen.make_cfg(52, 3000, 100, 20000, 15000),
           "wide_ragged_instr_global": gsrgen.make_cfg(53, 4000, (10, 300), 20000, 40000)}[name]
    h, s, b, ctx = _setup32(cfg)
    xp = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
    ctx.solve(xp, damp=1e-6, atol=1e-14, btol=1e-14, conlim=0.0, itnlim=5000)  # binary64 arithmetic, same values
    xm = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
    info = ctx.solve(xm, mode=g.GSR_MIXED, damp=1e-6, inner_fused=fused)
    errs = block_errors(xm.cpu().numpy(), xp.cpu().numpy(), s)
    assert max(errs.values()) <= 1e-9, (errs, info)
    ctx.close()


def test_mixed_fixed_schedule_and_x0():
    """A fixed schedule (inner iterations x outer steps) and a warm start x0."""
    w = gsrgen.workloads()["c1"]
    h, s, b, ctx = _setup32(w.cfg)
    xo, _ = oracle.lsqr(s, b, 500, 1e-14, 1e-14, 0.0, w.damp)
    x = np.zeros(s.n_cols)
    info = ctx.solve(x, mode=g.GSR_MIXED, damp=w.damp, inner_itn=12, max_outer=3, refine_tol=-1.0,
                     atol=0.0, btol=0.0, inner_tol=1e-30)
    assert info["outer_itn"] == 3 and info["itn"] == 36, info
    assert max(block_errors(x, xo, s).values()) <= 1e-9
    # a shorter inner limit for the refinement steps after the first
    xs = np.zeros(s.n_cols)
    info = ctx.solve(xs, mode=g.GSR_MIXED, damp=w.damp, inner_itn=14, inner_itn_next=9, max_outer=3,
                     refine_tol=-1.0, atol=0.0, btol=0.0, inner_tol=1e-30)
    assert info["outer_itn"] == 3 and info["itn"] == 14 + 2 * 9, info
    assert max(block_errors(xs, xo, s).values()) <= 1e-9
    with pytest.raises(TypeError):
        ctx.solve(xs, mode=g.GSR_MIXED, inner_iterations=3)  # misspelt parameter
    with pytest.raises(g.GsrError) as e:
        ctx.solve(xs, mode=g.GSR_MIXED, inner_itn_next=-1)
    assert e.value.status == g.Status.EINVAL
    x1 = np.zeros(s.n_cols)
    info = ctx.solve(x1, x0=xo, mode=g.GSR_MIXED, damp=w.damp)
    assert info["outer_itn"] <= 2 and max(block_errors(x1, xo, s).values()) <= 1e-9, info
    with pytest.raises(g.GsrError) as e:
        ctx.solve(x1, mode=g.GSR_MIXED, se_out=np.zeros(s.n_cols))
    assert e.value.status == g.Status.EINVAL
    ctx.close()


def _abs_sys(s):
    return oracle.System(s.star_ptr, np.abs(s.A), s.knot, s.instr, s.n_dfa, s.n_instr, s.n_glob)


@pytest.mark.parametrize("name", ["c1", "ragged_wide", "instr_32bit"])
def test_binary32_kernels_and_residual(name):
    """The inner kernels against the oracle on the same (rounded) values.

    aprod1_f32: 24 binary32 products and sums per row, error <= 25 u sum|terms|
    (u = 2^-24). aprod2_f32: binary32 partial sums of up to ~10^3 terms before
    the binary64 flush; bound 2e3 u sum|terms|. residual: double-float, then
    rounded to binary32: |r - r_ref| <= u |r_ref| + 2^-40 sum|terms|."""
    cfg = {"c1": gsrgen.workloads()["c1"].cfg, "ragged_wide": gsrgen.make_cfg(61, 2000, (10, 300), 9000, 9000),
           "instr_32bit": gsrgen.make_cfg(62, 2000, 100, 100, 70000)}[name]
    h, s, b, ctx = _setup32(cfg)
    u = 2.0 ** -24
    rng = np.random.default_rng(9)
    x = rng.standard_normal(s.n_cols).astype(np.float32).astype(np.float64)
    y0 = rng.standard_normal(s.n_rows).astype(np.float32).astype(np.float64)
    yd = torch.tensor(y0, dtype=torch.float32, device="cuda")
    ctx.aprod1_f32(torch.tensor(x, dtype=torch.float32, device="cuda"), yd)
    want = oracle.aprod1(s, x, y0.copy())
    scale = oracle.aprod1(_abs_sys(s), np.abs(x), np.abs(y0).copy())
    assert np.all(np.abs(yd.cpu().numpy() - want) <= 25 * u * scale)

    z0 = rng.standard_normal(s.n_cols)
    zd = torch.tensor(z0, device="cuda")
    ctx.aprod2_f32(torch.tensor(y0, dtype=torch.float32, device="cuda"), zd)
    want2 = oracle.aprod2(s, y0, z0.copy())
    scale2 = oracle.aprod2(_abs_sys(s), np.abs(y0), np.abs(z0).copy())
    assert np.all(np.abs(zd.cpu().numpy() - want2) <= 2e3 * u * scale2)

    xs = rng.standard_normal(s.n_cols)
    rd = torch.zeros(s.n_rows, dtype=torch.float32, device="cuda")
    ctx.residual(torch.tensor(xs, device="cuda"), rd)
    r_ref = b - oracle.aprod1(s, xs, np.zeros(s.n_rows))
    rscale = oracle.aprod1(_abs_sys(s), np.abs(xs), np.abs(b).copy())
    assert np.all(np.abs(rd.cpu().numpy() - r_ref) <= u * np.abs(r_ref) + 2.0 ** -40 * rscale)
    ctx.close()


def test_binary32_entry_points_need_fp32_context():
    cfg = gsrgen.make_cfg(7, 20, 30, 12, 8)
    h = gsrgen.generate(cfg)
    ctx = context_for(h)
    ctx.set_system(h.A, h.knot, h.instr, np.ones(h.n_rows))
    with pytest.raises(g.GsrError) as e:
        ctx.aprod1_f32(torch.zeros(ctx.n_cols, dtype=torch.float32, device="cuda"),
                       torch.zeros(ctx.n_rows, dtype=torch.float32, device="cuda"))
    assert e.value.status == g.Status.EINVAL
    with pytest.raises(g.GsrError) as e:
        ctx.residual(torch.zeros(ctx.n_cols, dtype=torch.float64, device="cuda"),
                     torch.zeros(ctx.n_rows, dtype=torch.float32, device="cuda"))
    assert e.value.status == g.Status.EINVAL
    ctx.close()


def test_binary32_instrumental_sums_are_order_independent():
    """The binary32 aprod 2 keeps the instrumental sums in 32-bit fixed point
    per block (scaled per column by a power of two) and adds the blocks in
    binary64, where those sums are exact: the instrumental entries of A^T y are
    bitwise the same from run to run, and match the oracle within the rounding
    of the fixed point (at most 2^-20 of the column's largest |a| max|y| per
    contribution) plus the binary32 products."""
    cfg = gsrgen.workloads()["c1"].cfg
    h, s, b, ctx = _setup32(cfg)
    rng = np.random.default_rng(21)
    y = rng.standard_normal(s.n_rows).astype(np.float32)
    yd = torch.tensor(y, device="cuda")
    a0, a1 = s.blocks()["instr"]
    outs = []
    for _ in range(3):
        z = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
        ctx.aprod2_f32(yd, z)
        outs.append(z.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o[a0:a1], outs[0][a0:a1])
    want = oracle.aprod2(s, y.astype(np.float64), np.zeros(s.n_cols))
    ic = s.instr.reshape(-1, 6)
    av = np.abs(s.A.reshape(-1, 24)[:, 17:23])
    amax = np.zeros(s.n_instr)
    np.maximum.at(amax, ic.ravel(), av.ravel())
    count = np.bincount(ic.ravel(), minlength=s.n_instr)
    bound = count * (2.0 ** -20 * amax * np.abs(y).max())
    scale = oracle.aprod2(_abs_sys(s), np.abs(y).astype(np.float64), np.zeros(s.n_cols))
    err = np.abs(outs[0][a0:a1] - want[a0:a1])
    assert np.all(err <= bound + 2.0 ** -23 * scale[a0:a1]), (err / (bound + 1e-300)).max()
    ctx.close()


def test_reload_that_changes_the_one_pass_choice():
    """The binary32 aprod 2 runs in one pass when every attitude column gets at least 20 fixed-point
    bits over the pass's partition. A reload whose rows all start at knot 0 (every row on the same
    4 columns per axis) leaves too few, so the context switches to the attitude reductions into L2
    windows and drops the iteration graphs it captured for the one-pass kernel. Mixed solves before and after the reload,
    and after reloading the first system again, match the oracle."""
    w = gsrgen.workloads()["c1"]
    h, s, b, ctx = _setup32(w.cfg)
    knot0 = np.zeros_like(h.knot)
    s0 = oracle.System(s.star_ptr, h.A, knot0, h.instr, s.n_dfa, s.n_instr, s.n_glob)
    b0 = oracle.rhs(s0, h.x_true, h.eps)
    for sys_, bb, kn in ((s, b, h.knot), (s0, b0, knot0), (s, b, h.knot)):
        ctx.set_system(h.A32, kn, h.instr, bb)
        x = np.zeros(s.n_cols)
        info = ctx.solve(x, mode=g.GSR_MIXED, damp=w.damp, inner_itn=30, max_outer=4)
        xo, _ = oracle.lsqr(sys_, bb, 2000, 1e-14, 1e-14, 0.0, w.damp)
        errs = block_errors(x, xo, sys_)
        assert max(errs.values()) <= 1e-9, (errs, info)
    ctx.close()


@pytest.mark.parametrize("spread", ["instr", "instr_and_att"])
def test_spread_coefficients_keep_per_column_precision(spread):
    """The one-pass aprod 2 gives the attitude columns one fixed-point scale, and the instrumental
    ones too, only when no column then loses precision: the group's fewest bits minus log2(largest /
    smallest column max |a|) must stay >= 20. Here the odd instrumental columns (and, in the second
    case, the third attitude axis) have coefficients 2^-4 times the others (4 bits of spread against
    about 21 bits on this system): the instrumental sums keep their per-column scales in the
    one-pass aprod 2 (first case), the attitude columns go to the vector reductions into L2 windows
    (form 3, second case).
    aprod2_f32 keeps its bounds (binary32 sums 2e3 u, the instrumental fixed point 2^-20 of each
    column's own bound) and the mixed solve matches the oracle. (The mixed solver's accuracy on
    columns of small norm is limited by the binary32 rounding of the refinement's right-hand side,
    about 2^-24 |r*| / |A_:,j| for the noise residual r*: 5e-10 here, 1.2e-7 with a spread of
    2^-12.)"""
    cfg = gsrgen.workloads()["c1"].cfg
    h = gsrgen.generate(cfg, fp32=True)
    A32 = h.A32.copy()
    small = (h.instr % 2) == 1                        # odd instrumental columns: 2^-4 smaller
    A32[:, 17:23][small] *= np.float32(2.0 ** -4)
    if spread == "instr_and_att":
        A32[:, 13:17] *= np.float32(2.0 ** -4)       # attitude axis 2
    A = A32.astype(np.float64)
    s = oracle.System(h.star_ptr, A, h.knot, h.instr, cfg.n_dfa, cfg.n_instr, cfg.n_glob)
    b = oracle.rhs(s, h.x_true, h.eps)
    ctx = context_for(h, fp32=True)
    ctx.set_system(A32, h.knot, h.instr, b)
    plan = ctx.aprod2_plan()
    assert plan["fx_bits"] >= 20 and plan["ins_group"] == 0
    assert plan["passes"] == (1 if spread == "instr" else 3)
    u = 2.0 ** -24
    rng = np.random.default_rng(17)
    y = rng.standard_normal(s.n_rows).astype(np.float32)
    z = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
    ctx.aprod2_f32(torch.tensor(y, device="cuda"), z)
    want = oracle.aprod2(s, y.astype(np.float64), np.zeros(s.n_cols))
    scale = oracle.aprod2(_abs_sys(s), np.abs(y).astype(np.float64), np.zeros(s.n_cols))
    err = np.abs(z.cpu().numpy() - want)
    a0, a1 = s.blocks()["instr"]
    assert np.all(err[:a0] <= 2e3 * u * scale[:a0])
    amax = np.zeros(s.n_instr)
    np.maximum.at(amax, h.instr.ravel(), np.abs(A[:, 17:23]).ravel())
    count = np.bincount(h.instr.ravel(), minlength=s.n_instr)
    bound = count * 2.0 ** -20 * amax * np.abs(y).max() + 2.0 ** -23 * scale[a0:a1]
    assert np.all(err[a0:a1] <= bound)
    x = np.zeros(s.n_cols)
    info = ctx.solve(x, mode=g.GSR_MIXED, damp=1e-6, inner_itn=30, max_outer=4)
    xo, _ = oracle.lsqr(s, b, 3000, 1e-14, 1e-14, 0.0, 1e-6)
    errs = block_errors(x, xo, s)
    assert max(errs.values()) <= 1e-9, (errs, info)
    ctx.close()


@pytest.mark.parametrize("case", ["odd_instr_2^-12", "glob_2^-10"])
def test_mixed_reaches_1e9_on_ill_scaled_columns(case):
    """Columns of very different norm: the odd instrumental columns 2^-12 times the others, or the
    global column 2^-10 times its usual size. Rounding the refinement's residual r to binary32 limits
    column j to about 2^-24 |r| / |A_:,j| (1.2e-7 in the instrumental block in the first case); the
    binary64 gradient A~^T r of the inner solves' start, which the refinement switches to when a step
    stops halving the correction (refine_grad 0) or uses from the second step on (refine_grad 1),
    brings every block within 1e-9 of the binary64 solution. With refine_grad -1 (binary32 start
    throughout) the first case stays above 1e-9."""
    cfg = gsrgen.workloads()["c1"].cfg
    h = gsrgen.generate(cfg, fp32=True)
    A32 = h.A32.copy()
    if case.startswith("odd_instr"):
        small = (h.instr % 2) == 1
        A32[:, 17:23][small] *= np.float32(2.0 ** -12)
    else:
        A32[:, 23] *= np.float32(2.0 ** -10)
    A = A32.astype(np.float64)
    s = oracle.System(h.star_ptr, A, h.knot, h.instr, cfg.n_dfa, cfg.n_instr, cfg.n_glob)
    b = oracle.rhs(s, h.x_true, h.eps)
    xo, _ = oracle.lsqr(s, b, 5000, 1e-15, 1e-15, 0.0, 1e-6)
    ctx = context_for(h, fp32=True)
    ctx.set_system(A32, h.knot, h.instr, b)
    for grad in (0, 1):
        x = np.zeros(s.n_cols)
        info = ctx.solve(x, mode=g.GSR_MIXED, damp=1e-6, refine_grad=grad)
        errs = block_errors(x, xo, s)
        assert max(errs.values()) <= 1e-9, (grad, errs, info)
    if case.startswith("odd_instr"):
        x = np.zeros(s.n_cols)
        info = ctx.solve(x, mode=g.GSR_MIXED, damp=1e-6, refine_grad=-1, max_outer=8)
        errs = block_errors(x, xo, s)
        assert errs["instr"] > 1e-9, (errs, info)
    ctx.close()


@pytest.mark.parametrize("name", ["c1", "wide_one_scale", "wide_ragged"])
def test_aprod12_f32_vs_oracle(name):
    """One Golub-Kahan step's two products (gsr_aprod12_f32): y <- A x + coef y, then z += A^T y with
    the new y. On the wide systems (60,000 attitude columns) both come from one read of each tile (the
    inner iterations' fused pass); on c1 the two separate products run. y within 25 u sum|terms| of the
    oracle's; z within 2e3 u sum|terms| of the oracle's A^T y for the GPU's own new y."""
    cfg = {"c1": gsrgen.workloads()["c1"].cfg, "wide_one_scale": gsrgen.make_cfg(64, 3000, 100, 20000, 15000),
           "wide_ragged": gsrgen.make_cfg(65, 4000, (1, 300), 20000, 40000)}[name]
    h, s, b, ctx = _setup32(cfg)
    assert ctx.aprod2_plan()["passes"] == (1 if name == "c1" else 3)
    u = 2.0 ** -24
    rng = np.random.default_rng(23)
    x = rng.standard_normal(s.n_cols).astype(np.float32).astype(np.float64)
    y0 = rng.standard_normal(s.n_rows).astype(np.float32).astype(np.float64)
    z0 = rng.standard_normal(s.n_cols)
    coef = -0.75
    yd = torch.tensor(y0, dtype=torch.float32, device="cuda")
    zd = torch.tensor(z0, device="cuda")
    ctx.aprod12_f32(torch.tensor(x, dtype=torch.float32, device="cuda"), yd, zd, coef)
    torch.cuda.synchronize()
    want = oracle.aprod1(s, x, coef * y0)
    scale = oracle.aprod1(_abs_sys(s), np.abs(x), np.abs(coef * y0))
    yn = yd.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(yn - want) <= 25 * u * scale)
    want2 = oracle.aprod2(s, yn, z0.copy())
    scale2 = oracle.aprod2(_abs_sys(s), np.abs(yn), np.abs(z0).copy())
    assert np.all(np.abs(zd.cpu().numpy() - want2) <= 2e3 * u * scale2)
    ctx.close()


@pytest.mark.parametrize("name", ["c1", "wide_ragged"])
def test_f32_products_on_vectors_at_odd_offsets(name):
    """The binary32 products on caller vectors that start 4 bytes past a 16-byte boundary (views at
    offset 1 of larger buffers): the kernels' 16-byte row-vector loads and stores apply only to aligned
    vectors, so these take the per-row path. aprod 1, aprod 2 and the fused pair against the oracle
    with the bounds of the aligned tests."""
    cfg = {"c1": gsrgen.workloads()["c1"].cfg, "wide_ragged": gsrgen.make_cfg(65, 4000, (1, 300), 20000, 40000)}[name]
    h, s, b, ctx = _setup32(cfg)
    u = 2.0 ** -24
    rng = np.random.default_rng(29)
    x = rng.standard_normal(s.n_cols).astype(np.float32).astype(np.float64)
    y0 = rng.standard_normal(s.n_rows).astype(np.float32).astype(np.float64)
    z0 = rng.standard_normal(s.n_cols)

    def view(v, dtype):
        buf = torch.zeros(v.size + 1, dtype=dtype, device="cuda")
        buf[1:] = torch.tensor(v, dtype=dtype, device="cuda")
        out = buf[1:]
        assert out.data_ptr() % 16 == 4
        return out

    xd, yd = view(x, torch.float32), view(y0, torch.float32)
    ctx.aprod1_f32(xd, yd)
    torch.cuda.synchronize()
    want = oracle.aprod1(s, x, y0)
    scale = oracle.aprod1(_abs_sys(s), np.abs(x), np.abs(y0))
    assert np.all(np.abs(yd.cpu().numpy().astype(np.float64) - want) <= 25 * u * scale)

    yv = view(y0, torch.float32)
    zd = torch.tensor(z0, device="cuda")
    ctx.aprod2_f32(yv, zd)
    torch.cuda.synchronize()
    want2 = oracle.aprod2(s, y0, z0.copy())
    scale2 = oracle.aprod2(_abs_sys(s), np.abs(y0), np.abs(z0).copy())
    assert np.all(np.abs(zd.cpu().numpy() - want2) <= 2e3 * u * scale2)

    coef = -0.75
    yv = view(y0, torch.float32)
    zd = torch.tensor(z0, device="cuda")
    ctx.aprod12_f32(xd, yv, zd, coef)
    torch.cuda.synchronize()
    want = oracle.aprod1(s, x, coef * y0)
    scale = oracle.aprod1(_abs_sys(s), np.abs(x), np.abs(coef * y0))
    yn = yv.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(yn - want) <= 25 * u * scale)
    want2 = oracle.aprod2(s, yn, z0.copy())
    scale2 = oracle.aprod2(_abs_sys(s), np.abs(yn), np.abs(z0).copy())
    assert np.all(np.abs(zd.cpu().numpy() - want2) <= 2e3 * u * scale2)
    ctx.close()


def test_wide_attitude_windows_at_the_edge_knots():
    """The attitude window accumulators and window copies at the ends of each axis: a wide system
    (20,000 knots per axis: the window forms) whose first 300 rows start at knot 0 and last 300 rows at
    knot n_dfa - 4 (the last window, whose columns end the axis), so the fold's first and last windows
    of every axis carry many products. The binary32 kernels and the fused pair against the oracle,
    and aprod 2 run twice (its binary32 sums in L2 arrive in any order) agreeing within that bound."""
    cfg = gsrgen.make_cfg(66, 2000, 100, 20000, 500)
    h = gsrgen.generate(cfg, fp32=True)
    knot = h.knot.copy()
    knot[:300] = 0
    knot[-300:] = cfg.n_dfa - 4
    s = oracle.System(h.star_ptr, h.A, knot, h.instr, cfg.n_dfa, cfg.n_instr, cfg.n_glob)
    b = oracle.rhs(s, h.x_true, h.eps)
    ctx = context_for(h, fp32=True)
    ctx.set_system(h.A32, knot, h.instr, b)
    assert ctx.aprod2_plan()["passes"] == 3
    u = 2.0 ** -24
    rng = np.random.default_rng(31)
    x = rng.standard_normal(s.n_cols).astype(np.float32).astype(np.float64)
    y0 = rng.standard_normal(s.n_rows).astype(np.float32).astype(np.float64)
    yd = torch.tensor(y0, dtype=torch.float32, device="cuda")
    ctx.aprod1_f32(torch.tensor(x, dtype=torch.float32, device="cuda"), yd)
    want = oracle.aprod1(s, x, y0.copy())
    scale = oracle.aprod1(_abs_sys(s), np.abs(x), np.abs(y0).copy())
    assert np.all(np.abs(yd.cpu().numpy() - want) <= 25 * u * scale)
    y32 = torch.tensor(y0, dtype=torch.float32, device="cuda")
    want2 = oracle.aprod2(s, y0, np.zeros(s.n_cols))
    scale2 = oracle.aprod2(_abs_sys(s), np.abs(y0), np.zeros(s.n_cols))
    runs = []
    for _ in range(2):
        zd = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
        ctx.aprod2_f32(y32, zd)
        runs.append(zd.cpu().numpy())
        assert np.all(np.abs(runs[-1] - want2) <= 2e3 * u * scale2)
    assert np.all(np.abs(runs[0] - runs[1]) <= 4e3 * u * scale2)
    a0 = s.blocks()["att"][0]
    for ax in range(3):  # the first and the last column of each axis got contributions
        for col in (a0 + ax * cfg.n_dfa, a0 + ax * cfg.n_dfa + cfg.n_dfa - 1):
            assert scale2[col] > 0 and abs(runs[0][col] - want2[col]) <= 2e3 * u * scale2[col]
    xs = rng.standard_normal(s.n_cols)
    rd = torch.zeros(s.n_rows, dtype=torch.float32, device="cuda")
    ctx.residual(torch.tensor(xs, device="cuda"), rd)
    r_ref = b - oracle.aprod1(s, xs, np.zeros(s.n_rows))
    rscale = oracle.aprod1(_abs_sys(s), np.abs(xs), np.abs(b).copy())
    assert np.all(np.abs(rd.cpu().numpy() - r_ref) <= u * np.abs(r_ref) + 2.0 ** -40 * rscale)
    ctx.close()


@pytest.mark.parametrize("name,fused", [("c1", 1), ("wide", 1), ("wide", -1)])
def test_closing_iteration_gives_the_same_iterate(name, fused):
    """An inner solve that runs to its iteration limit m ends with a closing iteration (aprod 1 and the
    x update; inner_close 1): LSQR's x_m = x_{m-1} + (phi_m / rho_m) w_m needs beta_{m+1}, not v_{m+1}.
    One refinement step of m inner iterations from x0 = 0, closing against every iteration in full
    (inner_close 0), for m = 4 and 5 (one graph of m iterations each) and m = 12 (two graphs of 6): the
    two differ only by the rounding of the last binary32 aprod 1 and its norm, far below the last LSQR
    step |x_m - x_{m-1}| that a wrong closing update would miss or repeat. c1 takes the one-pass
    shared-memory aprod 2; 'wide' (20,000 knots per axis) the fused pass (1) or the two passes (-1)."""
    cfg = {"c1": gsrgen.workloads()["c1"].cfg, "wide": gsrgen.make_cfg(54, 3000, 100, 20000, 3000)}[name]
    h, s, b, ctx = _setup32(cfg)
    kw = dict(mode=g.GSR_MIXED, damp=1e-6, max_outer=1, refine_tol=-1.0, inner_tol=1e-30, atol=0.0, btol=0.0,
              conlim=0.0, inner_fused=fused)
    res = {}
    for m in (3, 4, 5, 11, 12):
        for close in (0, 1):
            if close and m in (3, 11):
                continue
            x = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
            info = ctx.solve(x, inner_itn=m, inner_close=close, **kw)
            assert info["itn"] == m and info["outer_itn"] == 1 and info["istop"] == 7, info
            res[m, close] = x.cpu().numpy()
    for m in (4, 5, 12):
        step = np.linalg.norm(res[m, 0] - res[m - 1, 0])
        assert step > 0.0
        assert np.linalg.norm(res[m, 1] - res[m, 0]) <= 1e-3 * step, (m, step)
    # the whole refinement with closing inner solves still reaches 1e-9 of the oracle's solution
    xo, _ = oracle.lsqr(s, b, 2000, 1e-14, 1e-14, 0.0, 1e-6)
    x = np.zeros(s.n_cols)
    info = ctx.solve(x, mode=g.GSR_MIXED, damp=1e-6, inner_itn=10, max_outer=8, inner_tol=1e-30, atol=0.0,
                     btol=0.0, inner_fused=fused)
    assert info["itn"] == 10 * info["outer_itn"], info
    errs = block_errors(x, xo, s)
    assert max(errs.values()) <= 1e-9, (errs, info)
    ctx.close()
