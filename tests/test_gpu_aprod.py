"""aprod 1 / aprod 2 on the GPU against the CPU oracle, element by element.

Tolerance: |gpu - oracle| <= 1e-13 * (sum of |terms|) per element: both sides
compute in binary64 and differ only in summation order and FMA contraction.
Cases span many blocks and warps, ragged stars (including empty stars and
single-row stars), no global column, and attitude / instrumental widths that
select each accumulator placement (shared memory or global atomics).
"""
import numpy as np
import pytest
import torch

import gsrgen
import oracle
import paper_2308_00778_gb300 as g
from gpu_util import abs_system, context_for

pytestmark = pytest.mark.gpu

CASES = {
    "tiny": gsrgen.make_cfg(7, 20, 30, 12, 8),
    "ragged_noglob": gsrgen.make_cfg(21, 13, (1, 37), 9, 6, n_glob=0),
    "empty_stars": gsrgen.make_cfg(23, 50, (0, 4), 4, 6),
    "c1": gsrgen.workloads()["c1"].cfg,
    "ragged_many": gsrgen.make_cfg(31, 3000, (1, 300), 250, 40),
    "wide_att_global": gsrgen.make_cfg(33, 400, 100, 20000, 15000),   # accumulators too big for shared memory
    "wide_att_instr_smem": gsrgen.make_cfg(34, 400, 100, 6000, 2000),  # attitude global, instr shared
    "instr_32bit": gsrgen.make_cfg(35, 2000, 100, 100, 70000),  # n_instr > 65536: 32-bit instrumental planes
}


def _check(got, want, scale, tol=1e-13):
    err = np.abs(got - want)
    bound = tol * (scale + np.abs(want)) + 1e-300
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3g}"


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("fp32", [False, True])
def test_aprod_vs_oracle(name, fp32):
    cfg = CASES[name]
    h = gsrgen.generate(cfg, fp32=fp32)
    s = oracle.from_host_system(h)
    ctx = context_for(h, fp32=fp32)
    ctx.set_system(h.A32 if fp32 else h.A, h.knot, h.instr)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(s.n_cols)
    y0 = rng.standard_normal(s.n_rows)
    xd = torch.tensor(x, device="cuda")
    yd = torch.tensor(y0, device="cuda")
    ctx.aprod1(xd, yd)
    want = oracle.aprod1(s, x, y0.copy())
    scale = oracle.aprod1(abs_system(s), np.abs(x), np.abs(y0).copy())
    _check(yd.cpu().numpy(), want, scale)

    u = rng.standard_normal(s.n_rows)
    x0 = rng.standard_normal(s.n_cols)
    ud = torch.tensor(u, device="cuda")
    zd = torch.tensor(x0, device="cuda")
    ctx.aprod2(ud, zd)
    want2 = oracle.aprod2(s, u, x0.copy())
    scale2 = oracle.aprod2(abs_system(s), np.abs(u), np.abs(x0).copy())
    _check(zd.cpu().numpy(), want2, scale2)
    ctx.close()


def test_aprod2_repeat_runs_agree():
    """aprod 2 adds per-star segments and per-knot runs with atomic adds, so the
    order of additions (and the last bits) can change from run to run; repeated
    runs agree to 1e-13 of the sum of |terms| in every unknown."""
    h = gsrgen.generate(CASES["c1"])
    s = oracle.from_host_system(h)
    ctx = context_for(h)
    ctx.set_system(h.A, h.knot, h.instr)
    u = torch.randn(s.n_rows, dtype=torch.float64, device="cuda")
    outs = []
    for _ in range(3):
        z = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
        ctx.aprod2(u, z)
        outs.append(z.cpu().numpy())
    scale = oracle.aprod2(abs_system(s), np.abs(u.cpu().numpy()), np.zeros(s.n_cols))
    for o in outs[1:]:
        assert np.all(np.abs(o - outs[0]) <= 1e-13 * scale)
    ctx.close()


def test_device_soa_input_and_chunks():
    """Rows loaded from device SoA planes in two chunks equal the host AoS load."""
    cfg = CASES["ragged_many"]
    h = gsrgen.generate(cfg)
    s = oracle.from_host_system(h)
    ctx = context_for(h)
    n = s.n_rows
    stride = n + 5
    vals = torch.zeros(24 * stride, dtype=torch.float64, device="cuda")
    ins = torch.zeros(6 * stride, dtype=torch.int32, device="cuda")
    A = torch.tensor(h.A, device="cuda")
    I = torch.tensor(h.instr, device="cuda")
    for j in range(24):
        vals[j * stride:j * stride + n] = A[:, j]
    for j in range(6):
        ins[j * stride:j * stride + n] = I[:, j]
    knot = torch.tensor(h.knot, device="cuda")
    cut = n // 3
    ctx.set_rows(cut, n - cut, vals[cut:], knot[cut:], ins[cut:], layout=g.GSR_SOA, plane_stride=stride)
    with pytest.raises(g.GsrError) as e:
        ctx.aprod1(torch.zeros(s.n_cols, dtype=torch.float64, device="cuda"),
                   torch.zeros(n, dtype=torch.float64, device="cuda"))
    assert e.value.status == g.Status.ESTATE
    ctx.set_rows(0, cut, vals, knot, ins, layout=g.GSR_SOA, plane_stride=stride)
    x = np.random.default_rng(4).standard_normal(s.n_cols)
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.aprod1(torch.tensor(x, device="cuda"), y)
    want = oracle.aprod1(s, x, np.zeros(n))
    scale = oracle.aprod1(abs_system(s), np.abs(x), np.zeros(n))
    _check(y.cpu().numpy(), want, scale)
    ctx.close()


@pytest.mark.parametrize("where", ["host", "device"])
def test_validation_rejects_bad_rows(where):
    cfg = CASES["tiny"]
    h = gsrgen.generate(cfg)
    ctx = context_for(h)

    def put(A, knot, instr):
        if where == "device":
            A, knot, instr = (torch.tensor(a, device="cuda") for a in (A, knot, instr))
        ctx.set_system(A, knot, instr)

    bad = h.knot.copy()
    bad[17] = cfg.n_dfa - 3
    with pytest.raises(g.GsrError) as e:
        put(h.A, bad, h.instr)
    assert e.value.status == g.Status.EINVAL
    bad = h.knot.copy()
    bad[3] = -1
    with pytest.raises(g.GsrError) as e:
        put(h.A, bad, h.instr)
    assert e.value.status == g.Status.EINVAL
    badi = h.instr.copy()
    badi[5, 2] = cfg.n_instr
    with pytest.raises(g.GsrError) as e:
        put(h.A, h.knot, badi)
    assert e.value.status == g.Status.EINVAL
    badA = h.A.copy()
    badA[9, 11] = np.nan
    with pytest.raises(g.GsrError) as e:
        put(badA, h.knot, h.instr)
    assert e.value.status == g.Status.ENUMERIC
    # nothing was committed: aprod still refuses
    with pytest.raises(g.GsrError) as e:
        ctx.aprod1(torch.zeros(ctx.n_cols, dtype=torch.float64, device="cuda"),
                   torch.zeros(ctx.n_rows, dtype=torch.float64, device="cuda"))
    assert e.value.status == g.Status.ESTATE
    put(h.A, h.knot, h.instr)
    b = np.ones(ctx.n_rows)
    b[4] = np.inf
    with pytest.raises(g.GsrError) as e:
        ctx.set_rhs(b)
    assert e.value.status == g.Status.ENUMERIC
    with pytest.raises(g.GsrError) as e:
        ctx.solve(np.zeros(ctx.n_cols))
    assert e.value.status == g.Status.ESTATE
    # a good b, then a bad one: the bad one is not kept either
    ctx.set_rhs(np.ones(ctx.n_rows))
    with pytest.raises(g.GsrError) as e:
        ctx.set_rhs(b)
    assert e.value.status == g.Status.ENUMERIC
    with pytest.raises(g.GsrError) as e:
        ctx.solve(np.zeros(ctx.n_cols))
    assert e.value.status == g.Status.ESTATE
    ctx.close()


@pytest.mark.parametrize("fp32", [False, True])
def test_pinned_host_rows_convert_in_one_pass(fp32):
    """AoS rows in pinned host memory are converted straight from host memory
    (one pass that also validates): the result equals the device-input load,
    and on a bad index or value the rows of the call are not loaded."""
    cfg = CASES["ragged_many"]
    h = gsrgen.generate(cfg, fp32=fp32)
    s = oracle.from_host_system(h)
    A = torch.tensor(h.A32 if fp32 else h.A).pin_memory()
    knot = torch.tensor(h.knot).pin_memory()
    instr = torch.tensor(h.instr).pin_memory()
    ref = context_for(h, fp32=fp32)
    ref.set_system(A.cuda(), knot.cuda(), instr.cuda())
    ctx = context_for(h, fp32=fp32)
    ctx.set_system(A, knot, instr)
    u = torch.randn(s.n_rows, dtype=torch.float64, device="cuda")
    z1 = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
    z2 = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
    ref.aprod2(u, z1)
    ctx.aprod2(u, z2)
    scale = oracle.aprod2(abs_system(s), np.abs(u.cpu().numpy()), np.zeros(s.n_cols))
    assert np.all(np.abs(z1.cpu().numpy() - z2.cpu().numpy()) <= 1e-13 * scale)
    x = torch.randn(s.n_cols, dtype=torch.float64, device="cuda")
    y1 = torch.zeros(s.n_rows, dtype=torch.float64, device="cuda")
    y2 = torch.zeros(s.n_rows, dtype=torch.float64, device="cuda")
    ref.aprod1(x, y1)
    ctx.aprod1(x, y2)
    assert torch.equal(y1, y2)
    # rows 100.. of a second load carry a bad instrumental column: those rows are not loaded
    bad = instr.clone().pin_memory()
    bad[150, 3] = cfg.n_instr
    n2 = s.n_rows - 100
    with pytest.raises(g.GsrError) as e:
        ctx.set_rows(100, n2, A[100:], knot[100:], bad[100:])
    assert e.value.status == g.Status.EINVAL
    with pytest.raises(g.GsrError) as e:
        ctx.aprod1(x, y2)
    assert e.value.status == g.Status.ESTATE
    badA = A.clone().pin_memory()
    badA[7, 2] = float("nan")
    with pytest.raises(g.GsrError) as e:
        ctx.set_rows(0, s.n_rows, badA, knot, instr)
    assert e.value.status == g.Status.ENUMERIC
    ctx.set_rows(0, s.n_rows, A, knot, instr)
    y2.zero_()
    ctx.aprod1(x, y2)
    assert torch.equal(y1, y2)
    ref.close()
    ctx.close()


@pytest.mark.parametrize("name", ["c1", "wide_att_global", "ragged_many"])
def test_aprod2_binary64_instrumental_columns_of_spread_scale(name):
    """The binary64 star pass sums the instrumental products as int64 fixed point with one power-of-two
    scale per column (from the column's largest |coefficient|, the most contributions one block adds to
    it, and max |y| of the call). Columns whose coefficients are 2^-20, 1 and 2^20 times the others
    (by column index mod 3) must each keep binary64 accuracy: every entry within 1e-13 of its own sum
    of |terms|, against the oracle on the same values. c1 and ragged_many take blocks of 256 threads,
    wide_att_global (15,000 instrumental columns: 150 KB of sums and shifts) one block of 512 per SM.
    Also y with a single huge entry (the bound then far above the typical product) and y = 0."""
    cfg = CASES[name]
    h = gsrgen.generate(cfg)
    fac = 2.0 ** (20.0 * ((np.arange(cfg.n_instr) % 3) - 1.0))
    A = h.A.copy()
    a_ins = 5 + 12
    for j in range(cfg.n_ipr):
        A[:, a_ins + j] *= fac[h.instr[:, j]]
    s = oracle.from_host_system(h)
    s = oracle.System(s.star_ptr, A, s.knot, s.instr, s.n_dfa, s.n_instr, s.n_glob, s.n_astro, s.n_ipr)
    ctx = context_for(h)
    ctx.set_system(A, h.knot, h.instr)
    rng = np.random.default_rng(11)
    u_spike = rng.standard_normal(s.n_rows)
    u_spike[s.n_rows // 3] = 1e6
    for u in (rng.standard_normal(s.n_rows), u_spike, np.zeros(s.n_rows)):
        x0 = rng.standard_normal(s.n_cols)
        zd = torch.tensor(x0, device="cuda")
        ctx.aprod2(torch.tensor(u, device="cuda"), zd)
        want = oracle.aprod2(s, u, x0.copy())
        scale = oracle.aprod2(abs_system(s), np.abs(u), np.abs(x0).copy())
        _check(zd.cpu().numpy(), want, scale)
    ctx.close()
