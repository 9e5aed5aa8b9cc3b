"""The warm start on the GPU: features and per-star solves against the oracle;
warm-started solves reach the same solution as cold solves."""
import numpy as np
import pytest
import torch

import gsrgen
import oracle
import paper_2308_00778_gb300 as g
from gpu_util import block_errors, context_for

pytestmark = pytest.mark.gpu


def _setup(cfg, fp32):
    h = gsrgen.generate(cfg, fp32=fp32)
    s = oracle.from_host_system(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    ctx = context_for(h, fp32=fp32)
    ctx.set_system(h.A32 if fp32 else h.A, h.knot, h.instr, b)
    return h, s, b, ctx


@pytest.mark.parametrize("fp32,wide", [(False, False), (True, False), (True, True)])
def test_features_vs_oracle(fp32, wide):
    # wide: 24,000 attitude columns, past the one-pass shared-memory form: the binary32 pass that sums
    # A^T b and the column norms adds the attitude products by vector reductions into L2 windows
    cfg = gsrgen.make_cfg(81, 2000, (50, 150), 8000 if wide else 400, 60, att_kind=1)
    h, s, b, ctx = _setup(cfg, fp32)
    f = torch.zeros((cfg.n_dfa, 6), dtype=torch.float32, device="cuda")
    scale = ctx.warm_features(f)
    fr, sr = oracle.jacobi_features(s, b)
    # binary32 storage: A^T b in binary32 products and partial sums
    tol = 2e-4 if fp32 else 1e-6
    assert scale == pytest.approx(sr, rel=tol)
    got = f.cpu().numpy().astype(np.float64)
    for c in range(6):
        assert np.linalg.norm(got[:, c] - fr[:, c]) <= tol * np.linalg.norm(fr[:, c]) + 1e-6, c
    ctx.close()


@pytest.mark.parametrize("fp32", [False, True])
def test_astro_solve_vs_oracle(fp32):
    cfg = gsrgen.make_cfg(82, 1500, (20, 120), 300, 40, att_kind=1)
    h, s, b, ctx = _setup(cfg, fp32)
    x0 = torch.zeros(s.n_cols, dtype=torch.float64, device="cuda")
    ctx.warm_start(x0)  # Jacobi attitude, per-star astrometric solve, zeros elsewhere
    got = x0.cpu().numpy()
    a0, a1 = s.blocks()["att"]
    # instrumental and global parts: their Jacobi estimates (A^T b)_j / |A_:,j|^2
    p = oracle.precond(s)
    jac = oracle.aprod2(s, b, np.zeros(s.n_cols)) * p * p
    tol = 2e-4 if fp32 else 1e-9
    assert np.linalg.norm(got[a1:] - jac[a1:]) <= tol * np.linalg.norm(jac[a1:])
    ref = np.zeros(s.n_cols)
    ref[a0:] = got[a0:]
    assert oracle.astro_solve(s, b, ref) == 0
    # binary64 storage: binary64 normal equations and Cholesky, so each star's 5 unknowns agree to
    # rounding (1e-12). Binary32 storage accumulates them in binary32 (the mixed solver's start, which
    # the refinement corrects): recursive summation of n <= 120 terms is good to n 2^-24 = 7e-6 of the
    # sum of |terms|, and the well-conditioned 5x5 systems (cond(G) ~ 10 with 20+ observations) keep
    # the solution within 1e-4.
    bar = 1e-4 if fp32 else 1e-12
    for st in range(cfg.n_stars):
        r, gg = ref[5 * st:5 * st + 5], got[5 * st:5 * st + 5]
        assert np.linalg.norm(gg - r) <= bar * np.linalg.norm(r) + bar * 1e-5, st
    ctx.close()


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_warm_started_solves_reach_the_cold_solution(mode, tmp_path):
    cfg = gsrgen.make_cfg(83, 4000, (100, 200), 500, 100, att_kind=1)
    h, s, b, ctx = _setup(cfg, fp32=True)
    kw = dict(damp=1e-6)
    if mode == "mixed":
        kw["mode"] = g.GSR_MIXED
    x_cold = np.zeros(s.n_cols)
    i_cold = ctx.solve(x_cold, itnlim=500, atol=1e-14, btol=1e-14, conlim=0.0, **kw)
    x_j = np.zeros(s.n_cols)
    i_j = ctx.solve(x_j, itnlim=500, atol=1e-14, btol=1e-14, conlim=0.0, warm=g.GSR_WARM_JACOBI, **kw)
    # a learned start with random (untrained) weights is still a valid start
    rng = np.random.default_rng(6)
    net = g.Net()
    net.set_params((rng.standard_normal(net.n_params) * 0.01).astype(np.float32))
    net.save(tmp_path / "w.bin")
    net.close()
    x_l = np.zeros(s.n_cols)
    i_l = ctx.solve(x_l, itnlim=500, atol=1e-14, btol=1e-14, conlim=0.0, warm=g.GSR_WARM_LEARNED,
                    weights_path=str(tmp_path / "w.bin"), **kw)
    for x, info in ((x_j, i_j), (x_l, i_l)):
        for k, e in block_errors(x, x_cold, s).items():
            assert e <= 1e-9, (mode, k, e, info)
        assert info["ms_warm"] > 0.0
    with pytest.raises(g.GsrError) as e:
        ctx.solve(np.zeros(s.n_cols), warm=g.GSR_WARM_LEARNED, weights_path=str(tmp_path / "missing.bin"))
    assert e.value.status == g.Status.EINVAL
    ctx.close()


def test_shipped_network_beats_jacobi_on_held_out_systems():
    """The trained network shipped with the package, on systems of its training
    shape drawn from seeds used neither in training nor in its evaluation: its
    attitude start is closer to the solution than the Jacobi estimate, and it
    needs no more LSQR iterations to 1e-9 than the Jacobi start, which needs
    fewer than the cold start."""
    import os

    from paper_2308_00778_gb300 import train

    assert os.path.exists(g.WARM_WEIGHTS)
    rows = train.evaluate(g.WARM_WEIGHTS, [400, 401], fp32=True)
    for r in rows:
        assert r["x0_err_learned_att"] < 0.6 * r["x0_err_jacobi_att"], r
        assert r["learned"] <= r["jacobi"] <= r["cold"], r
    assert sum(r["learned"] for r in rows) < sum(r["cold"] for r in rows)
