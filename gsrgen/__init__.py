"""Seeded synthetic Gaia-shaped systems, shared by the oracle and the GPU path.

This module only draws inputs: coefficients, attitude knots, instrumental
columns, the planted solution ``x_true`` and the noise ``eps``. It holds none of
the solver's arithmetic; ``b = A x_true + eps`` is assembled by each caller with
its own aprod 1. The generator itself is C (``gsrgen_core.h``), built twice:
``libgsrgen_host.so`` (gcc) and ``libgsrgen_dev.so`` (nvcc, device twin), with
bit-identical output.

Row model (paper Sec. 2): 24 coefficients per observation (5 astrometric,
3 axes x 4 attitude knots, 6 instrumental, 1 global), rows grouped by star,
observation times sorted within a star. Section variants (0..5 astrometric
and 0..6 instrumental coefficients per row, 0..5 globals) give compact rows of
n_astro + 12 + n_ipr + n_glob coefficients (``Cfg.npar``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
HOST_LIB = os.path.join(_HERE, "libgsrgen_host.so")
DEV_LIB = os.path.join(_HERE, "libgsrgen_dev.so")


class Cfg(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_stars", ctypes.c_int64),
        ("obs_min", ctypes.c_int32),
        ("obs_max", ctypes.c_int32),
        ("n_dfa", ctypes.c_int32),
        ("n_instr", ctypes.c_int32),
        ("n_glob", ctypes.c_int32),
        ("att_kind", ctypes.c_int32),
        ("noise_sigma", ctypes.c_double),
        ("n_astro", ctypes.c_int32),
        ("n_ipr", ctypes.c_int32),
    ]

    def ncols(self) -> int:
        return self.n_astro * self.n_stars + 3 * self.n_dfa + self.n_instr + self.n_glob

    @property
    def standard(self) -> bool:
        """The paper's standard sections (5 astrometric, 6 instrumental per row, at most 1 global)."""
        return self.n_astro == 5 and self.n_ipr == 6 and self.n_glob <= 1

    @property
    def npar(self) -> int:
        """Coefficients per generated row: 24 for the standard sections, else the compact row."""
        return 24 if self.standard else self.n_astro + 12 + self.n_ipr + self.n_glob

    def describe(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


def make_cfg(seed, n_stars, obs, n_dfa, n_instr, n_glob=1, att_kind=0, noise_sigma=1e-3, n_astro=5,
             n_ipr=6) -> Cfg:
    """obs is an int (fixed observations per star) or a (min, max) pair. n_astro (0..5), n_ipr (0..6,
    at most n_instr) and n_glob (0..5) choose the sections of a row."""
    lo, hi = (obs, obs) if isinstance(obs, int) else obs
    if not (0 <= n_astro <= 5 and 0 <= n_ipr <= min(6, n_instr) and 0 <= n_glob <= 5):
        raise ValueError("sections: n_astro in [0, 5], n_ipr in [0, min(6, n_instr)], n_glob in [0, 5]")
    return Cfg(seed, n_stars, lo, hi, n_dfa, n_instr, n_glob, att_kind, noise_sigma, n_astro, n_ipr)


@dataclass(frozen=True)
class Workload:
    """A named synthetic workload: generator settings plus the solve settings."""

    name: str
    cfg: Cfg
    fp32: bool        # values stored in binary32
    damp: float
    atol: float
    btol: float
    itnlim: int


def workloads() -> dict:
    """The synthetic stand-ins for the paper's (unavailable) DPCT systems.

    tiny : 20 stars x 30 obs, 12 knots, 8 instr, 1 global (600 x 145)
    c1   : 1,000 stars x 100 obs, 100 knots/axis, 60 instr, 1 global, seed 0
    c2   : 100k stars x 200 obs (2e7 rows), 3,000 knots/axis, 1,000 instr, sinusoid attitude, seed 1
    c2h  : c2 with half the stars (1e7 rows), for profiling captures
    c3   : 1M stars x 200 obs (2e8 rows), 30,000 knots/axis, 10,000 instr, FP32 values, seed 2
    c4   : 50k stars x 200 obs (1e7 rows), 2,000 knots/axis, 500 instr, sinusoid attitude (seed per system)
    c5   : 2M stars x 250 obs (5e8 rows), 60,000 knots/axis, 20,000 instr, sinusoid attitude, FP32 values, seed 5
    c2g5 : c2 with five global unknowns (the five-global systems of Sec. 4.2): 28 coefficients per row
    c2a2 : c2 with 2 astrometric and 3 instrumental coefficients per row and no global: 17 per row
    """
    return {
        "tiny": Workload("tiny", make_cfg(7, 20, 30, 12, 8), False, 1e-6, 1e-12, 1e-12, 400),
        "c1": Workload("c1", make_cfg(0, 1000, 100, 100, 60), False, 1e-6, 1e-12, 1e-12, 200),
        "c2": Workload("c2", make_cfg(1, 100_000, 200, 3000, 1000, att_kind=1), False, 1e-6, 1e-12, 1e-12, 2000),
        "c2h": Workload("c2h", make_cfg(1, 50_000, 200, 3000, 1000, att_kind=1), False, 1e-6, 1e-12, 1e-12, 2000),
        "c3": Workload("c3", make_cfg(2, 1_000_000, 200, 30000, 10000), True, 1e-6, 1e-12, 1e-12, 2000),
        "c4": Workload("c4", make_cfg(100, 50_000, 200, 2000, 500, att_kind=1), False, 1e-6, 1e-12, 1e-12, 2000),
        "c5": Workload("c5", make_cfg(5, 2_000_000, 250, 60000, 20000, att_kind=1), True, 1e-6, 1e-12, 1e-12, 2000),
        "c2g5": Workload("c2g5", make_cfg(1, 100_000, 200, 3000, 1000, n_glob=5, att_kind=1), False, 1e-6, 1e-12,
                         1e-12, 2000),
        "c2a2": Workload("c2a2", make_cfg(1, 100_000, 200, 3000, 1000, n_glob=0, att_kind=1, n_astro=2, n_ipr=3),
                         False, 1e-6, 1e-12, 1e-12, 2000),
    }


_host = None
_dev = None


def _load_host():
    global _host
    if _host is None:
        if not os.path.exists(HOST_LIB):
            from . import build as _b

            _b.build_host()
        lib = ctypes.CDLL(HOST_LIB)
        P = ctypes.c_void_p
        lib.gsrgen_host_ncols.restype = ctypes.c_int64
        lib.gsrgen_host_ncols.argtypes = [ctypes.POINTER(Cfg)]
        lib.gsrgen_host_star_ptr.restype = ctypes.c_int64
        lib.gsrgen_host_star_ptr.argtypes = [ctypes.POINTER(Cfg), P]
        lib.gsrgen_host_rows.restype = None
        lib.gsrgen_host_rows.argtypes = [ctypes.POINTER(Cfg), P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                         P, P, P, P]
        lib.gsrgen_host_xtrue.restype = None
        lib.gsrgen_host_xtrue.argtypes = [ctypes.POINTER(Cfg), ctypes.c_int64, ctypes.c_int64, P]
        lib.gsrgen_host_noise.restype = None
        lib.gsrgen_host_noise.argtypes = [ctypes.POINTER(Cfg), ctypes.c_int64, ctypes.c_int64, P]
        lib.gsrgen_host_normal_at.restype = ctypes.c_double
        lib.gsrgen_host_normal_at.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
        lib.gsrgen_host_ln.restype = ctypes.c_double
        lib.gsrgen_host_ln.argtypes = [ctypes.c_double]
        lib.gsrgen_host_cos_turn.restype = ctypes.c_double
        lib.gsrgen_host_cos_turn.argtypes = [ctypes.c_double]
        lib.gsrgen_host_bits.restype = ctypes.c_uint64
        lib.gsrgen_host_bits.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]
        _host = lib
    return _host


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def star_ptr(cfg: Cfg) -> np.ndarray:
    lib = _load_host()
    sp = np.empty(cfg.n_stars + 1, dtype=np.int64)
    lib.gsrgen_host_star_ptr(ctypes.byref(cfg), _ptr(sp))
    return sp


def rows(cfg: Cfg, sp: np.ndarray, s0: int, s1: int, fp32: bool = False, want32: bool = False):
    """Rows of stars [s0, s1): (A_d as float64 n x npar, knot, instr n x n_ipr[, A_d as float32]).

    With fp32 the float64 values are the binary32-rounded coefficients widened
    back (exactly what an FP32-stored system holds)."""
    lib = _load_host()
    n = int(sp[s1] - sp[s0])
    A = np.empty((n, cfg.npar), dtype=np.float64)
    A32 = np.empty((n, cfg.npar), dtype=np.float32) if want32 else None
    knot = np.empty(n, dtype=np.int32)
    instr = np.empty((n, cfg.n_ipr), dtype=np.int32)
    if n > 0:
        lib.gsrgen_host_rows(ctypes.byref(cfg), _ptr(sp), s0, s1, 1 if fp32 else 0, _ptr(A),
                             _ptr(A32) if want32 else None, _ptr(knot), _ptr(instr))
    if want32:
        return A, knot, instr, A32
    return A, knot, instr


def xtrue(cfg: Cfg, col0: int = 0, ncol: int | None = None) -> np.ndarray:
    lib = _load_host()
    if ncol is None:
        ncol = cfg.ncols() - col0
    x = np.empty(ncol, dtype=np.float64)
    if ncol > 0:
        lib.gsrgen_host_xtrue(ctypes.byref(cfg), col0, ncol, _ptr(x))
    return x


def noise(cfg: Cfg, row0: int, nrow: int) -> np.ndarray:
    lib = _load_host()
    e = np.empty(nrow, dtype=np.float64)
    if nrow > 0:
        lib.gsrgen_host_noise(ctypes.byref(cfg), row0, nrow, _ptr(e))
    return e


@dataclass
class HostSystem:
    """A whole synthetic system on the host (no right-hand side: see module doc)."""

    cfg: Cfg
    star_ptr: np.ndarray
    A: np.ndarray       # n x npar float64 (binary32-rounded values when fp32)
    knot: np.ndarray
    instr: np.ndarray
    x_true: np.ndarray
    eps: np.ndarray
    fp32: bool
    A32: np.ndarray | None = None

    @property
    def n_rows(self) -> int:
        return int(self.star_ptr[-1])

    @property
    def n_cols(self) -> int:
        return self.cfg.ncols()


def generate(cfg: Cfg, fp32: bool = False) -> HostSystem:
    sp = star_ptr(cfg)
    if fp32:
        A, knot, instr, A32 = rows(cfg, sp, 0, cfg.n_stars, fp32=True, want32=True)
    else:
        A, knot, instr = rows(cfg, sp, 0, cfg.n_stars)
        A32 = None
    return HostSystem(cfg, sp, A, knot, instr, xtrue(cfg), noise(cfg, 0, int(sp[-1])), fp32, A32)


# ---------------------------------------------------------------- device twin
def _load_dev():
    global _dev
    if _dev is None:
        if not os.path.exists(DEV_LIB):
            raise RuntimeError(f"device generator not built: {DEV_LIB} missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(DEV_LIB)
        P = ctypes.c_void_p
        lib.gsrgen_dev_rows.restype = ctypes.c_int
        lib.gsrgen_dev_rows.argtypes = [ctypes.POINTER(Cfg), P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                        P, P, ctypes.c_int64, P, P, P]
        lib.gsrgen_dev_xtrue.restype = ctypes.c_int
        lib.gsrgen_dev_xtrue.argtypes = [ctypes.POINTER(Cfg), ctypes.c_int64, ctypes.c_int64, P, P]
        lib.gsrgen_dev_noise.restype = ctypes.c_int
        lib.gsrgen_dev_noise.argtypes = [ctypes.POINTER(Cfg), ctypes.c_int64, ctypes.c_int64, P, P]
        _dev = lib
    return _dev


def dev_rows(cfg: Cfg, sp_dev, sp_host: np.ndarray, s0: int, s1: int, vals, plane_stride: int, knot, instr,
             stream: int = 0, round32: bool = False):
    """Fill device SoA planes (torch tensors) for stars [s0, s1). vals is float64 or float32."""
    import torch

    lib = _load_dev()
    v64 = vals.data_ptr() if vals.dtype == torch.float64 else None
    v32 = vals.data_ptr() if vals.dtype == torch.float32 else None
    rc = lib.gsrgen_dev_rows(ctypes.byref(cfg), sp_dev.data_ptr(), _ptr(sp_host), s0, s1, 1 if round32 else 0,
                             v64, v32, plane_stride, knot.data_ptr(), instr.data_ptr(), stream)
    if rc != 0:
        raise RuntimeError(f"gsrgen_dev_rows failed: cuda error {rc}")


def dev_xtrue(cfg: Cfg, x, col0: int = 0, stream: int = 0):
    rc = _load_dev().gsrgen_dev_xtrue(ctypes.byref(cfg), col0, x.numel(), x.data_ptr(), stream)
    if rc != 0:
        raise RuntimeError(f"gsrgen_dev_xtrue failed: cuda error {rc}")


def dev_noise(cfg: Cfg, eps, row0: int = 0, stream: int = 0):
    rc = _load_dev().gsrgen_dev_noise(ctypes.byref(cfg), row0, eps.numel(), eps.data_ptr(), stream)
    if rc != 0:
        raise RuntimeError(f"gsrgen_dev_noise failed: cuda error {rc}")
