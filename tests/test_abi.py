"""The C ABI library loads and exports every entry point declared in include/gsr.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header=None):
    """Function names declared in include/<header> (all headers when None)."""
    import glob

    files = [os.path.join(ROOT, "include", header)] if header else sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))
    names = set()
    for f in files:
        txt = re.sub(r"/\*.*?\*/", "", open(f).read(), flags=re.S)
        names |= set(re.findall(r"\b(gsr_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def libgsr():
    import paper_2308_00778_gb300.build as pb

    if not os.path.exists(pb.LIB):
        pb.build()
    return ctypes.CDLL(pb.LIB)


def test_every_declared_symbol_is_exported(libgsr):
    names = _declared()
    assert "gsr_lsqr_solve" in names and "gsr_aprod1" in names and "gsr_aprod2" in names
    missing = [n for n in names if not hasattr(libgsr, n)]
    assert not missing, missing


def test_no_internal_symbols_exported():
    import subprocess

    import paper_2308_00778_gb300.build as pb

    out = subprocess.run(["nm", "-D", "--defined-only", pb.LIB], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    ours = {n for n in exported if n.startswith("gsr")}
    assert ours == set(_declared()), sorted(ours ^ set(_declared()))


def test_errors_without_gpu_are_status_codes():
    """Calls fail with a status, never abort, when given bad arguments (CPU only: no device use)."""
    import paper_2308_00778_gb300 as g

    L = g.lib()
    h = ctypes.c_void_p()
    assert L.gsr_create(None, 1, 1, None, 4, 6, 1, 0, 0) == g.Status.EINVAL
    assert L.gsr_create(ctypes.byref(h), 0, 1, None, 4, 6, 1, 0, 0) == g.Status.EINVAL  # no stars
    assert L.gsr_create(ctypes.byref(h), 1, 1, None, 3, 6, 1, 0, 0) == g.Status.EINVAL  # n_dfa < 4
    assert L.gsr_create(ctypes.byref(h), 1, 1, None, 4, 5, 1, 0, 0) == g.Status.EINVAL  # n_instr < 6
    assert L.gsr_create(ctypes.byref(h), 1, 1, None, 4, 6, 2, 0, 0) == g.Status.EINVAL  # n_glob > 1
    assert L.gsr_create(ctypes.byref(h), 1, 1, None, 4, 6, 1, 7, 0) == g.Status.EINVAL  # precision
    assert L.gsr_create(ctypes.byref(h), 1, 0, None, 4, 6, 1, 0, 0) == g.Status.EINVAL  # no grouping
    assert h.value is None
    # section variants (Sec. 2): 0..5 astrometric, 0..6 instrumental per row (<= n_instr), 0..5 globals
    cs = L.gsr_create_sections
    assert cs(ctypes.byref(h), 1, 1, None, 6, 4, 6, 6, 1, 0, 0) == g.Status.EINVAL   # n_astro > 5
    assert cs(ctypes.byref(h), 1, 1, None, -1, 4, 6, 6, 1, 0, 0) == g.Status.EINVAL  # n_astro < 0
    assert cs(ctypes.byref(h), 1, 1, None, 5, 4, 6, 7, 1, 0, 0) == g.Status.EINVAL   # n_ipr > 6
    assert cs(ctypes.byref(h), 1, 1, None, 5, 4, 3, 4, 1, 0, 0) == g.Status.EINVAL   # n_instr < n_ipr
    assert cs(ctypes.byref(h), 1, 1, None, 5, 4, 6, 6, 6, 0, 0) == g.Status.EINVAL   # n_glob > GSR_MAX_GLOB
    assert cs(ctypes.byref(h), 1, 1, None, 5, 3, 6, 6, 1, 0, 0) == g.Status.EINVAL   # n_dfa < 4
    assert cs(None, 1, 1, None, 5, 4, 6, 6, 1, 0, 0) == g.Status.EINVAL
    assert h.value is None
    assert g.gsr_sections(0)[0] == g.Status.EINVAL
    assert g.gsr_aprod2_plan(0)[0] == g.Status.EINVAL
    assert g.gsr_aprod1(0, 0, 0) == g.Status.EINVAL
    assert g.gsr_lsqr_solve(0, g.gsr_default_params(), 0, 0, 0, g.SolveInfo()) == g.Status.EINVAL
    assert g.gsr_destroy(0) == g.Status.OK
    p = g.gsr_default_params()
    assert p.itnlim == 2000 and p.atol == 1e-12 and p.precond == 1 and p.mode == g.GSR_PLAIN


def test_shipped_weights_match_the_network(libgsr):
    """The trained warm-start network shipped with the package holds exactly the
    parameters of the library's network (header, count, finite values), in the
    layout the trainer writes (per layer W[cout][cin][5] then bias[cout])."""
    import json

    import numpy as np

    import paper_2308_00778_gb300 as g
    from paper_2308_00778_gb300 import train

    raw = open(g.WARM_WEIGHTS, "rb").read()
    assert raw[:8] == b"GSRNET01"
    cnt = int(np.frombuffer(raw[8:16], dtype=np.int64)[0])
    vals = np.frombuffer(raw[16:], dtype=np.float32)
    libgsr.gsr_net_num_params.restype = ctypes.c_int64
    n = libgsr.gsr_net_num_params()
    assert cnt == n == vals.size == train.init_params(0).size
    assert np.all(np.isfinite(vals))
    meta = json.load(open(g.WARM_WEIGHTS[:-4] + ".json"))
    assert meta["mean_iterations"]["learned"] < meta["mean_iterations"]["cold"]
