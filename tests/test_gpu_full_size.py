"""Parity at the benchmark's full size: the 2e7-row workload (100,000 stars x
200 observations, 3,000 knots per axis, 1,000 instrumental unknowns, sinusoid
attitude, coefficients rounded to binary32), in the launch configuration the
benchmark times. The oracle computes every output here (its aprods take about
a second on this size, its LSQR about a second per iteration).

Bars: binary64 aprods within 1e-13 of sum|terms| per output; binary32 aprods
within the binary32 bounds of the small-size tests; a fixed number of binary64
LSQR iterations within 1e-10 per block of the oracle's; the benchmark's
solvers within 1e-9 per block of the oracle's tightly converged solution."""
import numpy as np
import pytest
import torch

import gsrgen
import oracle
import paper_2308_00778_gb300 as g
from gpu_util import block_errors, context_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    w = gsrgen.workloads()["c2"]
    h = gsrgen.generate(w.cfg, fp32=True)  # h.A: the binary32-rounded values, widened
    s = oracle.from_host_system(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    ctx64 = context_for(h, fp32=False)
    ctx64.set_system(h.A, h.knot, h.instr, b)
    ctx32 = context_for(h, fp32=True)
    ctx32.set_system(h.A32, h.knot, h.instr, b)
    sabs = oracle.System(s.star_ptr, np.abs(s.A), s.knot, s.instr, s.n_dfa, s.n_instr, s.n_glob)
    yield w, h, s, b, ctx64, ctx32, sabs
    ctx64.close()
    ctx32.close()


def test_full_size_aprods_vs_oracle(full):
    w, h, s, b, ctx64, ctx32, sabs = full
    rng = np.random.default_rng(5)
    x = rng.standard_normal(s.n_cols)
    u = rng.standard_normal(s.n_rows)
    y = torch.zeros(s.n_rows, dtype=torch.float64, device="cuda")
    ctx64.aprod1(torch.tensor(x, device="cuda"), y)
    want = oracle.aprod1(s, x, np.zeros(s.n_rows))
    scale = oracle.aprod1(sabs, np.abs(x), np.zeros(s.n_rows))
    assert np.all(np.abs(y.cpu().numpy() - want) <= 1e-13 * scale)
    z = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
    ctx64.aprod2(torch.tensor(u, device="cuda"), z)
    want2 = oracle.aprod2(s, u, np.zeros(s.n_cols))
    scale2 = oracle.aprod2(sabs, np.abs(u), np.zeros(s.n_cols))
    assert np.all(np.abs(z.cpu().numpy() - want2) <= 1e-13 * scale2)
    # binary32 kernels on binary32-valued inputs
    eps = 2.0 ** -24
    x32 = x.astype(np.float32)
    u32 = u.astype(np.float32)
    y32 = torch.zeros(s.n_rows, dtype=torch.float32, device="cuda")
    ctx32.aprod1_f32(torch.tensor(x32, device="cuda"), y32)
    want = oracle.aprod1(s, x32.astype(np.float64), np.zeros(s.n_rows))
    scale = oracle.aprod1(sabs, np.abs(x32).astype(np.float64), np.zeros(s.n_rows))
    assert np.all(np.abs(y32.cpu().numpy() - want) <= 25 * eps * scale)
    z = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
    ctx32.aprod2_f32(torch.tensor(u32, device="cuda"), z)
    want2 = oracle.aprod2(s, u32.astype(np.float64), np.zeros(s.n_cols))
    scale2 = oracle.aprod2(sabs, np.abs(u32).astype(np.float64), np.zeros(s.n_cols))
    err = np.abs(z.cpu().numpy() - want2)
    a0, a1 = s.blocks()["instr"]
    assert np.all(err[:a0] <= 2e3 * eps * scale2[:a0])
    assert np.all(err[a1:] <= 2e3 * eps * scale2[a1:])
    # instrumental columns: fixed point, at most 2^-20 of the column's largest |a| max|u| per contribution
    ic = s.instr.reshape(-1, 6)
    amax = np.zeros(s.n_instr)
    np.maximum.at(amax, ic.ravel(), np.abs(s.A.reshape(-1, 24)[:, 17:23]).ravel())
    count = np.bincount(ic.ravel(), minlength=s.n_instr)
    bound = count * 2.0 ** -20 * amax * np.abs(u32).max() + 2.0 ** -23 * scale2[a0:a1]
    assert np.all(err[a0:a1] <= bound)


def test_full_size_lsqr_iterations_vs_oracle(full):
    """Five binary64 LSQR iterations (tolerances off) against the oracle's five."""
    w, h, s, b, ctx64, ctx32, sabs = full
    x = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
    ctx64.solve(x, itnlim=5, atol=0.0, btol=0.0, conlim=0.0, damp=w.damp)
    xo, _ = oracle.lsqr(s, b, 5, 0.0, 0.0, 0.0, w.damp)
    errs = block_errors(x.cpu().numpy(), xo, s)
    assert max(errs.values()) <= 1e-10, errs


def test_full_size_benchmark_solvers_vs_oracle(full):
    """The benchmark's solvers (binary64 from zero, mixed from zero and from the
    learned start) against the oracle's tightly converged solution."""
    w, h, s, b, ctx64, ctx32, sabs = full
    xs, info = oracle.lsqr(s, b, 60, 1e-15, 1e-15, 0.0, w.damp)
    cases = {
        "fp64_plain": (ctx64, dict(itnlim=16, atol=0.0, btol=0.0, conlim=0.0, damp=w.damp)),
        "mixed": (ctx32, dict(mode=g.GSR_MIXED, inner_itn=8, inner_itn_next=8, max_outer=2, refine_tol=-1.0,
                              inner_tol=1e-30, atol=0.0, btol=0.0, conlim=0.0, damp=w.damp)),
        "mixed_learned": (ctx32, dict(mode=g.GSR_MIXED, inner_itn=8, inner_itn_next=5, max_outer=2,
                                      refine_tol=-1.0, inner_tol=1e-30, atol=0.0, btol=0.0, conlim=0.0,
                                      damp=w.damp, warm=g.GSR_WARM_LEARNED, weights_path=g.WARM_WEIGHTS)),
    }
    for name, (ctx, kw) in cases.items():
        x = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
        ctx.solve(x, **kw)
        errs = block_errors(x.cpu().numpy(), xs, s)
        assert max(errs.values()) <= 1e-9, (name, errs)
