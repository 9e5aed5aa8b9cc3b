"""Helpers shared by the GPU tests: build a context from a host system, compare with the oracle."""
import numpy as np

import gsrgen
import oracle
import paper_2308_00778_gb300 as g


def context_for(h, fp32=False, device=0, star_ptr_always=False):
    c = h.cfg
    obs = np.diff(h.star_ptr)
    uniform = (obs.min() == obs.max()) and obs.min() > 0 and not star_ptr_always
    sec = dict(n_astro=c.n_astro, n_ipr=c.n_ipr)
    if uniform:
        ctx = g.Context(c.n_stars, obs_per_star=int(obs[0]), n_dfa=c.n_dfa, n_instr=c.n_instr, n_glob=c.n_glob,
                        fp32=fp32, device=device, **sec)
    else:
        ctx = g.Context(c.n_stars, star_ptr=h.star_ptr, n_dfa=c.n_dfa, n_instr=c.n_instr, n_glob=c.n_glob,
                        fp32=fp32, device=device, **sec)
    return ctx


def abs_system(s):
    return oracle.System(s.star_ptr, np.abs(s.A), s.knot, s.instr, s.n_dfa, s.n_instr, s.n_glob, s.n_astro, s.n_ipr)


def block_errors(x, ref, s):
    """Relative error per block: |x_blk - ref_blk| / max(|ref_blk|, 1e-3)."""
    out = {}
    for name, (a, z) in s.blocks().items():
        if z > a:
            out[name] = float(np.linalg.norm(x[a:z] - ref[a:z]) / max(np.linalg.norm(ref[a:z]), 1e-3))
    return out
