"""The form of the binary32 aprod 2 (gsr_aprod2_plan) against the statistics it rests on.

The fixed-point sums of the binary32 aprod 2 give column j b_j = min(30, 31 -
ceil(log2(k_j + 1))) bits, k_j being the largest number of contributions one
block of the pass's fixed partition (8 warps a block, each warp a contiguous
range of max(ceil(tiles / (16 x SM count)), 8) tiles of 128 rows) adds to column j;
they are used when every instrumental column gets >= 20 bits. One pass over
the tiles sums the attitude columns too, with one scale for all of them, when
their fewest bits minus ceil(log2(largest / smallest column max |a|)) stay >=
20 and their accumulators fit in shared memory (8 bytes per column, 100 KB);
the instrumental columns share one scale on the same condition. Otherwise the
standard row adds the attitude products by vector reductions into L2 window
accumulators (form 3). The expected plan is recomputed here from the rows on
the host.
"""
import math

import numpy as np
import pytest
import torch

import gsrgen
import paper_2308_00778_gb300 as g
from gpu_util import context_for

pytestmark = pytest.mark.gpu


def _bits(kmax):
    lg = np.ceil(np.log2(kmax.astype(np.float64) + 1.0))
    return np.minimum(31 - lg, 30).astype(np.int64)


def _loss(colmax):
    nz = colmax[colmax > 0].astype(np.float64)
    return 99 if nz.size == 0 else math.ceil(math.log2(nz.max() / nz.min()))


def expected_plan(A32, knot, instr, n_dfa, n_instr, sm_count):
    n = len(knot)
    T = 128
    n_tiles = -(-n // T)
    per = max(-(-n_tiles // (sm_count * 16)), 8)
    blk = np.arange(n, dtype=np.int64) // (8 * per * T)
    nb = int(blk.max()) + 1
    cnt_i = np.bincount((blk[:, None] * n_instr + instr).ravel(), minlength=nb * n_instr).reshape(nb, n_instr)
    min_ins = int(_bits(cnt_i.max(0)).min())
    if min_ins < 20:
        return {"passes": 3, "fx_bits": 0, "ins_group": 0}
    na = 3 * n_dfa
    cols = np.concatenate([ax * n_dfa + knot[:, None] + np.arange(4)[None, :] for ax in range(3)], axis=1)
    cnt_a = np.bincount((blk[:, None] * na + cols).ravel(), minlength=nb * na).reshape(nb, na)
    min_att = int(_bits(cnt_a.max(0)).min())
    am_i = np.zeros(n_instr, np.float32)
    np.maximum.at(am_i, instr.ravel(), np.abs(A32[:, 17:23]).ravel())
    am_a = np.zeros(na, np.float32)
    np.maximum.at(am_a, cols.ravel(), np.abs(A32[:, 5:17]).ravel())
    fits = 8 * (n_instr + na) <= 100 * 1024
    one = fits and min_att - _loss(am_a) >= 20
    grp = one and min_ins - _loss(am_i) >= 20
    return {"passes": 1 if one else 3, "fx_bits": min_ins, "ins_group": 1 if grp else 0}


def _c2_shape(n_stars):
    c = gsrgen.workloads()["c2"].cfg
    return gsrgen.make_cfg(c.seed, n_stars, (c.obs_min, c.obs_max), c.n_dfa, c.n_instr, c.n_glob, c.att_kind,
                           c.noise_sigma)


@pytest.mark.parametrize("name", ["c1", "c2_10k_stars"])
def test_plan_matches_the_statistics(name):
    """c1 and a 2e6-row system of the 2e7-row workload's shape (8,192 rows per block: edge knots
    appear in few rows of a block, which must not shrink the attitude group's smallest column
    bound, a global maximum) both take the one-pass form with one instrumental scale."""
    cfg = gsrgen.workloads()["c1"].cfg if name == "c1" else _c2_shape(10000)
    h = gsrgen.generate(cfg, fp32=True)
    ctx = context_for(h, fp32=True)
    ctx.set_system(h.A32, h.knot, h.instr)
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    want = expected_plan(h.A32, h.knot, h.instr, cfg.n_dfa, cfg.n_instr, sm)
    assert ctx.aprod2_plan() == want
    assert want["passes"] == 1 and want["ins_group"] == 1
    ctx.close()


def test_plan_follows_a_reload():
    """A reload whose rows all start at knot 0 (12 attitude columns take every row) leaves too few
    bits for the one-pass form, so the attitude products go to the window reductions; reloading the
    first rows brings the one-pass form back."""
    cfg = gsrgen.workloads()["c1"].cfg
    h = gsrgen.generate(cfg, fp32=True)
    ctx = context_for(h, fp32=True)
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    knot0 = np.zeros_like(h.knot)
    for kn, passes in ((h.knot, 1), (knot0, 3), (h.knot, 1)):
        ctx.set_system(h.A32, kn, h.instr)
        plan = ctx.aprod2_plan()
        assert plan == expected_plan(h.A32, kn, h.instr, cfg.n_dfa, cfg.n_instr, sm)
        assert plan["passes"] == passes
    ctx.close()


def test_plan_errors():
    cfg = gsrgen.workloads()["tiny"].cfg
    h = gsrgen.generate(cfg, fp32=False)
    ctx = context_for(h, fp32=False)
    ctx.set_system(h.A, h.knot, h.instr)
    assert g.gsr_aprod2_plan(ctx.h)[0] == g.Status.EINVAL  # binary64-stored context
    ctx.close()
    c32 = context_for(h, fp32=True)
    assert g.gsr_aprod2_plan(c32.h)[0] == g.Status.ESTATE  # rows not loaded
    c32.close()
