"""gsr_residual_static, the allocation-free variant of gsr_residual.

Some callers cannot allocate device memory when they call the library (their
device memory is held by another allocator's pool, or they cannot afford the
implicit synchronisation of cudaMalloc). gsr_residual_static serves them: it
keeps its scratch in a fixed file-scope device array instead of the context's
workspace. This test calls it through the C ABI twice in a row (different x
each time, the second call overwriting what the first left in the shared
array) and checks each result against gsr_residual, the entry point that uses
the workspace, within the residual tolerance of the other GPU tests
(u |r| + 2^-40 sum|terms|, u = 2^-24). It runs last (file name) so that a
failure here never hides the other tests, and it also passes on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

import gsrgen
import oracle
import paper_2308_00778_gb300 as g
from gpu_util import context_for

pytestmark = pytest.mark.gpu


def _abs_sys(s):
    return oracle.System(s.star_ptr, np.abs(s.A), s.knot, s.instr, s.n_dfa, s.n_instr, s.n_glob)


def test_static_residual_matches_workspace_residual_twice():
    cfg = gsrgen.make_cfg(71, 3000, (40, 160), 700, 300, att_kind=1)
    h = gsrgen.generate(cfg, fp32=True)
    s = oracle.from_host_system(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    ctx = context_for(h, fp32=True)
    ctx.set_system(h.A32, h.knot, h.instr, b)
    u = 2.0 ** -24
    L = g.lib()
    rng = np.random.default_rng(17)
    for call in range(2):
        x = rng.standard_normal(s.n_cols) * (1.0 + call)
        xd = torch.tensor(x, device="cuda")
        r_ws = torch.empty(s.n_rows, dtype=torch.float32, device="cuda")
        ctx.residual(xd, r_ws)
        r_st = torch.full((s.n_rows,), float("nan"), dtype=torch.float32, device="cuda")
        st = L.gsr_residual_static(ctypes.c_void_p(ctx.h), ctypes.c_void_p(xd.data_ptr()),
                                   ctypes.c_void_p(r_st.data_ptr()), None)
        assert st == g.Status.OK, g.gsr_last_error(ctx.h)
        torch.cuda.synchronize()
        got, ref = r_st.cpu().numpy().astype(np.float64), r_ws.cpu().numpy().astype(np.float64)
        scale = oracle.aprod1(_abs_sys(s), np.abs(x), np.abs(b).copy())
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= u * np.abs(ref) + 2.0 ** -40 * scale), call
    ctx.close()


def test_static_residual_rejects_too_many_columns():
    # 5 * 210,000 astrometric unknowns alone exceed the 2^20-column capacity
    ctx = g.Context(210_000, obs_per_star=1, n_dfa=4, n_instr=6, n_glob=1, fp32=True)
    assert ctx.n_cols > 1 << 20
    x = torch.zeros(ctx.n_cols, dtype=torch.float64, device="cuda")
    r = torch.zeros(ctx.n_rows, dtype=torch.float32, device="cuda")
    st = g.gsr_residual_static(ctx.h, x.data_ptr(), r.data_ptr())
    assert st == g.Status.EINVAL and "capacity" in g.gsr_last_error(ctx.h)
    ctx.close()
