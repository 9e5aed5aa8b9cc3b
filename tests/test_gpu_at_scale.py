"""Parity at the sizes of the mixed-precision configuration (2e8 rows: 1e6 stars x 200
observations, 30,000 knots per axis, 10,000 instrumental unknowns) and of the
combined-at-scale one (5e8 rows: 2e6 stars x 250, 60,000 knots per axis, 20,000
instrumental unknowns), with binary32 storage as both state, in the launch configuration
of the solver's kernels.

The oracle cannot run over the whole system at these sizes, so:
* aprod 1 (binary32) on every row of sampled stars, and the astrometric entries of
  aprod 2 (binary32) of those stars (only their own rows feed them), against the oracle
  run on a system made of those stars' rows (the generator's host twin draws them);
* the whole of both products through the adjoint identity <A x, u> = <x, A^T u> of the
  binary64-arithmetic aprods, to 1e-12 of <|A||x|, |u|>;
* the fused inner-iteration pass (both products from one read of each tile) the same
  way: its new u on the sampled stars' rows and their astrometric columns against the
  oracle, every entry of its A^T u against the binary64 aprod 2 of the same u;
* every entry of the binary32 aprod 2 against the binary64 one, within the binary32
  bounds: 2e3 u of |A|^T|u| as in the small-size tests, plus, for the attitude,
  instrumental and global columns, the longest run of terms one lane adds in binary32
  at these sizes, and 2^-20 of the column's bound max|a_j| max|u| per contribution for
  fixed-point columns.
The scales |A||x| and |A|^T|u| come from a second context that holds |A|.
"""
import numpy as np
import pytest
import torch

import gsrgen
import oracle
import paper_2308_00778_gb300 as g
from paper_2308_00778_gb300.data import new_context

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


def _load(cfg, dev):
    """Two binary32-stored contexts of cfg's rows, the second holding |A|; per-column counts and
    largest |a| of the attitude and instrumental columns (device tensors)."""
    sp = gsrgen.star_ptr(cfg)
    n = int(sp[-1])
    spd = torch.tensor(sp, device=dev)
    vals = torch.empty(24 * n, dtype=torch.float32, device=dev)
    knot = torch.empty(n, dtype=torch.int32, device=dev)
    ins = torch.empty(6 * n, dtype=torch.int32, device=dev)
    gsrgen.dev_rows(cfg, spd, sp, 0, cfg.n_stars, vals, n, knot, ins, round32=True)
    ctx = new_context(cfg, True, dev.index or 0)
    ctx.set_rows(0, n, vals, knot, ins, layout=g.GSR_SOA, plane_stride=n)
    vals.abs_()
    cabs = new_context(cfg, True, dev.index or 0)
    cabs.set_rows(0, n, vals, knot, ins, layout=g.GSR_SOA, plane_stride=n)
    torch.cuda.synchronize(dev)
    # column statistics for the fixed-point bound (counts over all rows bound any block's count)
    nd, ni = cfg.n_dfa, cfg.n_instr
    kcount = torch.bincount(knot.long(), minlength=nd)
    att_count = torch.zeros(3 * nd, dtype=torch.int64, device=dev)
    att_max = torch.zeros(3 * nd, dtype=torch.float32, device=dev)
    for ax in range(3):
        for j in range(4):
            att_count[ax * nd + j: ax * nd + nd] += kcount[: nd - j]
            col = knot.long() + (ax * nd + j)
            att_max.scatter_reduce_(0, col, vals[(5 + 4 * ax + j) * n:(6 + 4 * ax + j) * n], "amax")
    ins_l = ins.long()
    ins_count = torch.bincount(ins_l, minlength=ni)
    ins_max = torch.zeros(ni, dtype=torch.float32, device=dev)
    for j in range(6):
        ins_max.scatter_reduce_(0, ins_l[j * n:(j + 1) * n], vals[(17 + j) * n:(18 + j) * n], "amax")
    del vals, knot, ins, ins_l, col
    torch.cuda.empty_cache()
    count = torch.cat([att_count, ins_count]).double()
    cmax = torch.cat([att_max, ins_max]).double()
    return sp, ctx, cabs, count, cmax


def _star_system(cfg, sp, stars, x):
    """The oracle's system of the given stars' rows, and x restricted to it (astrometric unknowns
    of those stars, then every attitude, instrumental and global unknown)."""
    As, ks, iis, cnt = [], [], [], [0]
    for s in stars:
        A, kn, ic = gsrgen.rows(cfg, sp, int(s), int(s) + 1, fp32=True)
        As.append(A)
        ks.append(kn)
        iis.append(ic)
        cnt.append(cnt[-1] + len(kn))
    sub = oracle.System(np.array(cnt), np.concatenate(As), np.concatenate(ks), np.concatenate(iis), cfg.n_dfa,
                        cfg.n_instr, cfg.n_glob)
    a0 = 5 * cfg.n_stars
    xs = np.concatenate([x[5 * s:5 * s + 5] for s in stars] + [x[a0:]])
    return sub, xs


def _bytes_needed(cfg):
    """Peak device memory of the test: two binary32 contexts (116 B a row each), the generator's
    staging planes with the int64 index copy of the statistics (24 + 4 + 24 + 48 B a row), then the
    knot-ordered attitude copies and their temporaries (52 + 64 B a row per context) and row vectors."""
    n = int(gsrgen.star_ptr(cfg)[-1])
    return max(2 * 116 * n + 100 * n, 2 * 116 * n + 2 * 52 * n + 64 * n + 40 * n)


@pytest.mark.parametrize("name", ["c3", "c5"])
def test_aprods_at_scale(name):
    cfg = gsrgen.workloads()[name].cfg
    dev = torch.device("cuda", 0)
    torch.cuda.empty_cache()  # what earlier tests left cached is free for this one
    free, _ = torch.cuda.mem_get_info(dev)
    if free < 1.1 * _bytes_needed(cfg):
        pytest.skip(f"needs about {_bytes_needed(cfg) / 1e9:.0f} GB of device memory, {free / 1e9:.0f} GB free")
    sp, ctx, cabs, count, cmax = _load(cfg, dev)
    try:
        _check(cfg, dev, sp, ctx, cabs, count, cmax)
    finally:
        ctx.close()
        cabs.close()
        torch.cuda.empty_cache()


def _check(cfg, dev, sp, ctx, cabs, count, cmax):
    n, nc = ctx.n_rows, ctx.n_cols
    a0 = 5 * cfg.n_stars
    t0 = a0 + 3 * cfg.n_dfa
    rng = np.random.default_rng(11)
    x = rng.standard_normal(nc).astype(np.float32)
    gen = torch.Generator(device=dev)
    gen.manual_seed(12)
    u = torch.randn(n, dtype=torch.float32, device=dev, generator=gen)
    xd = torch.tensor(x, device=dev)

    # binary32 products
    y = torch.zeros(n, dtype=torch.float32, device=dev)
    ctx.aprod1_f32(xd, y)
    z = torch.zeros(nc, dtype=torch.float64, device=dev)
    ctx.aprod2_f32(u, z)

    # sampled stars against the oracle
    stars = np.unique(np.concatenate([[0, cfg.n_stars - 1], rng.choice(cfg.n_stars, 40, replace=False)]))
    sub, xs = _star_system(cfg, sp, stars, x.astype(np.float64))
    sabs = oracle.System(sub.star_ptr, np.abs(sub.A), sub.knot, sub.instr, sub.n_dfa, sub.n_instr, sub.n_glob)
    rows = np.concatenate([np.arange(sp[s], sp[s + 1]) for s in stars])
    rows_d = torch.tensor(rows, device=dev)
    want = oracle.aprod1(sub, xs, np.zeros(sub.n_rows))
    scale = oracle.aprod1(sabs, np.abs(xs), np.zeros(sub.n_rows))
    got = y[rows_d].double().cpu().numpy()
    assert np.all(np.abs(got - want) <= 25 * EPS32 * scale), np.max(np.abs(got - want) / scale)
    us = u[rows_d].double().cpu().numpy()
    want2 = oracle.aprod2(sub, us, np.zeros(sub.n_cols))[:5 * len(stars)]
    scale2 = oracle.aprod2(sabs, np.abs(us), np.zeros(sub.n_cols))[:5 * len(stars)]
    astro_cols = torch.tensor(np.concatenate([np.arange(5 * s, 5 * s + 5) for s in stars]), device=dev)
    got2 = z[astro_cols].cpu().numpy()
    assert np.all(np.abs(got2 - want2) <= 2e3 * EPS32 * scale2)

    # the whole vectors: adjoint identity of the binary64-arithmetic aprods
    x64 = xd.double()
    u64 = u.double()
    y64 = torch.zeros(n, dtype=torch.float64, device=dev)
    ctx.aprod1(x64, y64)
    z64 = torch.zeros(nc, dtype=torch.float64, device=dev)
    ctx.aprod2(u64, z64)
    s64 = torch.zeros(n, dtype=torch.float64, device=dev)
    cabs.aprod1(x64.abs(), s64)
    S = torch.dot(s64, u64.abs()).item()
    d = abs(torch.dot(y64, u64).item() - torch.dot(x64, z64).item())
    assert d <= 1e-12 * S, (d, S)
    del y64, s64

    # every entry of the binary32 aprod 2 against the binary64 one
    w64 = torch.zeros(nc, dtype=torch.float64, device=dev)
    cabs.aprod2(u64.abs(), w64)
    umax = u.abs().max().double().item()
    bound = 2e3 * EPS32 * w64 + 1e-13 * w64
    # attitude, instrumental and global sums: one lane adds at most the 4 rows of each tile of its
    # warp's range in binary32 before a reduction (ranges of at most max(ceil(tiles / (8 x SMs)), 8) tiles)
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    n_tiles = -(-n // 128)
    k_lane = 4 * max(-(-n_tiles // (8 * sm)), 8)
    bound[a0:] += k_lane * EPS32 * w64[a0:]
    bound[a0:t0 + cfg.n_instr] += count * 2.0 ** -20 * cmax * umax
    err = (z - z64).abs()
    assert bool(torch.all(err <= bound)), float(torch.max(err / bound.clamp_min(1e-300)))
    del z64, w64, err, bound

    # the fused inner-iteration pass (y <- A x + coef y, then z += A^T y with the new y from the same read
    # of each tile), the solver's dominant kernel on these shapes: the new y on the sampled stars' rows and
    # the astrometric entries of their columns against the oracle, every entry of z against the
    # binary64-arithmetic aprod 2 of the GPU's own new y, with the bounds above
    assert ctx.aprod2_plan()["passes"] == 3
    coef = -0.75
    y1 = u.clone()
    z1 = torch.zeros(nc, dtype=torch.float64, device=dev)
    ctx.aprod12_f32(xd, y1, z1, coef)
    want = oracle.aprod1(sub, xs, coef * us)
    scale = oracle.aprod1(sabs, np.abs(xs), np.abs(coef * us))
    y1s = y1[rows_d].double().cpu().numpy()
    assert np.all(np.abs(y1s - want) <= 25 * EPS32 * scale), np.max(np.abs(y1s - want) / scale)
    want2 = oracle.aprod2(sub, y1s, np.zeros(sub.n_cols))[:5 * len(stars)]
    scale2 = oracle.aprod2(sabs, np.abs(y1s), np.zeros(sub.n_cols))[:5 * len(stars)]
    got2 = z1[astro_cols].cpu().numpy()
    assert np.all(np.abs(got2 - want2) <= 2e3 * EPS32 * scale2)
    y164 = y1.double()
    z164 = torch.zeros(nc, dtype=torch.float64, device=dev)
    ctx.aprod2(y164, z164)
    w164 = torch.zeros(nc, dtype=torch.float64, device=dev)
    cabs.aprod2(y164.abs(), w164)
    bound1 = 2e3 * EPS32 * w164 + 1e-13 * w164
    bound1[a0:] += k_lane * EPS32 * w164[a0:]
    err1 = (z1 - z164).abs()
    assert bool(torch.all(err1 <= bound1)), float(torch.max(err1 / bound1.clamp_min(1e-300)))
