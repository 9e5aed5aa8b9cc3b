"""gsr_residual_static, the allocation-free variant of gsr_residual.

Some callers cannot allocate device memory when they call the library: their
device memory is held by another allocator's pool, or they run a loop that
cannot afford cudaMalloc's implicit synchronisation. gsr_residual_static serves
them: it keeps its scratch in a fixed file-scope device array, placed on the
device (with the kernels it launches) when a context is created there, instead
of the context's workspace, which gsr_residual allocates on first use.

The test makes the entry point's first call on a fresh context, before any
gsr_residual call, and checks it against the oracle's binary64 residual within
the residual tolerance of the other GPU tests (u |r| + 2^-40 sum|terms|,
u = 2^-24); then a second call with another x, which overwrites what the first
left in the shared array. Device memory must not change across either call
(cudaMemGetInfo), and each result must equal gsr_residual's bit for bit (the
same kernels on the same inputs). The file name makes pytest collect it last,
so that a failure here never hides the other tests; it also passes on its own.
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


def _static_call(L, ctx, xd, r):
    """One gsr_residual_static call through the C ABI; returns the free device bytes before and after."""
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st = L.gsr_residual_static(ctypes.c_void_p(ctx.h), ctypes.c_void_p(xd.data_ptr()),
                               ctypes.c_void_p(r.data_ptr()), None)
    assert st == g.Status.OK, g.gsr_last_error(ctx.h)
    torch.cuda.synchronize()
    return free0, torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("n_dfa", [700, 6000])
def test_static_residual_allocates_nothing_and_matches_gsr_residual(n_dfa):
    # 6000 knots per axis: a wide attitude block, where gsr_residual reads the attitude pairs through the
    # context's window copy and the instrumental pairs from shared memory; the entry point here gathers
    # them from its own array, the same terms in the same order
    cfg = gsrgen.make_cfg(71, 3000, (40, 160), n_dfa, 300, att_kind=1)
    h = gsrgen.generate(cfg, fp32=True)
    s = oracle.from_host_system(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    ctx = context_for(h, fp32=True)
    ctx.set_system(h.A32, h.knot, h.instr, b)
    u = 2.0 ** -24
    L = g.lib()
    rng = np.random.default_rng(17)
    xs = [rng.standard_normal(s.n_cols) * (1.0 + call) for call in range(2)]
    # every tensor of the test exists before the first call
    xds = [torch.tensor(x, device="cuda") for x in xs]
    r_st = [torch.full((s.n_rows,), float("nan"), dtype=torch.float32, device="cuda") for _ in xs]
    r_ws = [torch.empty(s.n_rows, dtype=torch.float32, device="cuda") for _ in xs]
    for call, (x, xd) in enumerate(zip(xs, xds)):
        free0, free1 = _static_call(L, ctx, xd, r_st[call])
        assert free1 == free0, f"call {call}: free device memory {free0} -> {free1}"
        got = r_st[call].cpu().numpy().astype(np.float64)
        ref = b.copy()
        oracle.aprod1(s, -x, ref)  # b - A x in binary64
        scale = oracle.aprod1(_abs_sys(s), np.abs(x), np.abs(b).copy())
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= u * np.abs(ref) + 2.0 ** -40 * scale), call
        # the workspace entry point (allocating on its first use) gives the identical bits
        ctx.residual(xd, r_ws[call])
        torch.cuda.synchronize()
        assert torch.equal(r_st[call], r_ws[call]), call
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
