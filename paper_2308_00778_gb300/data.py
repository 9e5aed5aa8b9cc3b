"""Synthetic Gaia-shaped systems built directly in device memory.

The coefficients come from the seeded generator's device twin (gsrgen), are
loaded into a context through gsr_set_rows (SoA device input), and the
right-hand side b = A x_true + eps is assembled with the library's own
aprod 1 (binary64 arithmetic).
"""
from __future__ import annotations

import torch

import gsrgen

from . import gsr as g


def load_rows(ctx, cfg, round32: bool, device, stream=0):
    """Generate the rows of cfg on the device and load them into ctx (same shape)."""
    sp = gsrgen.star_ptr(cfg)
    n = int(sp[-1])
    spd = torch.tensor(sp, device=device)
    vdt = torch.float32 if ctx_fp32(ctx) else torch.float64
    vals = torch.empty(cfg.npar * n, dtype=vdt, device=device)
    knot = torch.empty(n, dtype=torch.int32, device=device)
    ins = torch.empty(max(cfg.n_ipr, 1) * n, dtype=torch.int32, device=device)
    gsrgen.dev_rows(cfg, spd, sp, 0, cfg.n_stars, vals, n, knot, ins, stream=stream, round32=round32)
    ctx.set_rows(0, n, vals, knot, ins, layout=g.GSR_SOA, plane_stride=n, stream=stream)
    return vals, knot, ins, sp


def ctx_fp32(ctx) -> bool:
    return getattr(ctx, "fp32", False)


def new_context(cfg, fp32_store: bool, device_index: int = 0):
    sp = gsrgen.star_ptr(cfg)
    obs = cfg.obs_min if cfg.obs_min == cfg.obs_max else 0
    ctx = g.Context(cfg.n_stars, obs_per_star=obs, star_ptr=None if obs else sp, n_dfa=cfg.n_dfa,
                    n_instr=cfg.n_instr, n_glob=cfg.n_glob, fp32=fp32_store, device=device_index,
                    n_astro=cfg.n_astro, n_ipr=cfg.n_ipr)
    ctx.fp32 = fp32_store
    return ctx


def set_rhs_from_truth(ctx, cfg, device, stream=0):
    """b = A x_true + eps with the context's aprod 1; returns (b, x_true) on the device."""
    xt = torch.empty(cfg.ncols(), dtype=torch.float64, device=device)
    gsrgen.dev_xtrue(cfg, xt, stream=stream)
    b = torch.empty(ctx.n_rows, dtype=torch.float64, device=device)
    gsrgen.dev_noise(cfg, b, stream=stream)
    ctx.aprod1(xt, b, stream=stream)
    ctx.set_rhs(b, stream=stream)
    return b, xt


def host_copies(cfg, vals, knot, ins, b, sp, chunk_rows: int = 1 << 25):
    """Pinned host copies of a generated system in the paper's row storage (A_d row-major, the
    instrumental columns row-major), transposed from the device planes chunk by chunk (so that no
    full-size transposed copy is made on the device)."""
    n = knot.numel()
    A = torch.empty((n, cfg.npar), dtype=vals.dtype, pin_memory=True)
    I = torch.empty((n, cfg.n_ipr), dtype=torch.int32, pin_memory=True)
    V = vals.view(cfg.npar, n)
    Iv = ins[:cfg.n_ipr * n].view(cfg.n_ipr, n)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        A[r0:r1].copy_(V[:, r0:r1].t().contiguous())
        if cfg.n_ipr:
            I[r0:r1].copy_(Iv[:, r0:r1].t().contiguous())
    kh = torch.empty(n, dtype=torch.int32, pin_memory=True)
    kh.copy_(knot)
    bh = torch.empty(n, dtype=torch.float64, pin_memory=True)
    bh.copy_(b)
    return {"A": A, "knot": kh, "instr": I, "b": bh, "star_ptr": sp}


def device_system(cfg, fp32_store: bool, round32: bool, device, stream=0, keep_host=False, ctx=None):
    """Build (or reload into ctx) the system of cfg. Returns (ctx, b, host copies or None)."""
    if ctx is None:
        ctx = new_context(cfg, fp32_store, device.index or 0)
    vals, knot, ins, sp = load_rows(ctx, cfg, round32, device, stream)
    b, _ = set_rhs_from_truth(ctx, cfg, device, stream)
    torch.cuda.synchronize(device)
    host = host_copies(cfg, vals, knot, ins, b, sp) if keep_host else None
    del vals, ins, knot
    torch.cuda.empty_cache()  # the staging planes: give them back for the library's own allocations
    return ctx, b, host
