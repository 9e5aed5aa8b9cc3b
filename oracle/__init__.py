"""Python face of the plain FP64 CPU oracle (liboracle.so, built from oracle/*.c).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference leg may import this package. It shares
no code with the GPU library and never loads it.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ORACLE_LIB lets the mutation tests load a deliberately broken copy of the oracle
LIB = os.environ.get("ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")


class _Sys(ctypes.Structure):
    _fields_ = [
        ("n_rows", ctypes.c_int64),
        ("n_stars", ctypes.c_int64),
        ("star_ptr", ctypes.c_void_p),
        ("n_dfa", ctypes.c_int32),
        ("n_instr", ctypes.c_int32),
        ("n_glob", ctypes.c_int32),
        ("A", ctypes.c_void_p),
        ("knot", ctypes.c_void_p),
        ("instr", ctypes.c_void_p),
    ]


class _Params(ctypes.Structure):
    _fields_ = [
        ("itnlim", ctypes.c_int32),
        ("atol", ctypes.c_double),
        ("btol", ctypes.c_double),
        ("conlim", ctypes.c_double),
        ("damp", ctypes.c_double),
        ("precond", ctypes.c_int32),
    ]


class _Info(ctypes.Structure):
    _fields_ = [
        ("istop", ctypes.c_int32),
        ("itn", ctypes.c_int32),
        ("anorm", ctypes.c_double),
        ("acond", ctypes.c_double),
        ("rnorm", ctypes.c_double),
        ("r1norm", ctypes.c_double),
        ("r2norm", ctypes.c_double),
        ("arnorm", ctypes.c_double),
        ("xnorm", ctypes.c_double),
        ("bnorm", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            from . import build as _b

            _b.build()
        lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        S = ctypes.POINTER(_Sys)
        lib.oracle_ncols.restype = ctypes.c_int64
        lib.oracle_ncols.argtypes = [S]
        lib.oracle_aprod1.restype = None
        lib.oracle_aprod1.argtypes = [S, P, P]
        lib.oracle_aprod2.restype = None
        lib.oracle_aprod2.argtypes = [S, P, P]
        lib.oracle_norm2.restype = ctypes.c_double
        lib.oracle_norm2.argtypes = [ctypes.c_int64, P]
        lib.oracle_precond.restype = None
        lib.oracle_precond.argtypes = [S, P]
        lib.oracle_scale_columns.restype = None
        lib.oracle_scale_columns.argtypes = [S, P, P]
        lib.oracle_lsqr.restype = ctypes.c_int
        lib.oracle_lsqr.argtypes = [S, P, ctypes.POINTER(_Params), P, P, ctypes.POINTER(_Info)]
        _extra_signatures(lib)
        _lib = lib
    return _lib


def _extra_signatures(lib):
    """Signatures of the warm-start reference routines (oracle_warm.c), when present."""
    P = ctypes.c_void_p
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    if hasattr(lib, "oracle_astro_solve"):
        lib.oracle_astro_solve.restype = ctypes.c_int
        lib.oracle_astro_solve.argtypes = [ctypes.POINTER(_Sys), P, P, f64, P]


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


@dataclass
class System:
    """A system in the paper's storage: A_d (n x 24), knot (M_i's attitude part), instr (I_c)."""

    star_ptr: np.ndarray
    A: np.ndarray
    knot: np.ndarray
    instr: np.ndarray
    n_dfa: int
    n_instr: int
    n_glob: int

    def __post_init__(self):
        self.star_ptr = np.ascontiguousarray(self.star_ptr, dtype=np.int64)
        self.A = np.ascontiguousarray(self.A, dtype=np.float64)
        self.knot = np.ascontiguousarray(self.knot, dtype=np.int32)
        self.instr = np.ascontiguousarray(self.instr, dtype=np.int32)
        self._s = _Sys(int(self.star_ptr[-1]), len(self.star_ptr) - 1, _p(self.star_ptr), self.n_dfa, self.n_instr,
                       self.n_glob, _p(self.A), _p(self.knot), _p(self.instr))

    @property
    def n_rows(self) -> int:
        return int(self.star_ptr[-1])

    @property
    def n_stars(self) -> int:
        return len(self.star_ptr) - 1

    @property
    def n_cols(self) -> int:
        return 5 * self.n_stars + 3 * self.n_dfa + self.n_instr + self.n_glob

    def blocks(self) -> dict:
        """Column ranges of the four sections of x (Sec. 2)."""
        a = 5 * self.n_stars
        t = a + 3 * self.n_dfa
        i = t + self.n_instr
        return {"astro": (0, a), "att": (a, t), "instr": (t, i), "glob": (i, i + self.n_glob)}


def from_host_system(hs) -> System:
    return System(hs.star_ptr, hs.A, hs.knot, hs.instr, hs.cfg.n_dfa, hs.cfg.n_instr, hs.cfg.n_glob)


def aprod1(s: System, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """y += A x (Eq. 2), in place; returns y."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert y.dtype == np.float64 and y.flags["C_CONTIGUOUS"] and y.shape == (s.n_rows,)
    _load().oracle_aprod1(ctypes.byref(s._s), _p(x), _p(y))
    return y


def aprod2(s: System, y: np.ndarray, x: np.ndarray) -> np.ndarray:
    """x += A^T y (Eq. 3), in place; returns x."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"] and x.shape == (s.n_cols,)
    _load().oracle_aprod2(ctypes.byref(s._s), _p(y), _p(x))
    return x


def norm2(a: np.ndarray) -> float:
    """Eq. 4 scaled 2-norm."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return _load().oracle_norm2(a.size, _p(a))


def precond(s: System) -> np.ndarray:
    p = np.empty(s.n_cols, dtype=np.float64)
    _load().oracle_precond(ctypes.byref(s._s), _p(p))
    return p


def rhs(s: System, x_true: np.ndarray, eps: np.ndarray) -> np.ndarray:
    """b = A x_true + eps, assembled with the oracle's aprod 1."""
    b = np.array(eps, dtype=np.float64, copy=True)
    return aprod1(s, x_true, b)


def lsqr(s: System, b: np.ndarray, itnlim: int, atol: float = 0.0, btol: float = 0.0, conlim: float = 0.0,
         damp: float = 0.0, precond: bool = True, want_var: bool = False):
    """Damped, column-preconditioned LSQR; returns (x, info dict[, var])."""
    lib = _load()
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(s.n_cols, dtype=np.float64)
    var = np.empty(s.n_cols, dtype=np.float64) if want_var else None
    prm = _Params(int(itnlim), atol, btol, conlim, damp, 1 if precond else 0)
    info = _Info()
    rc = lib.oracle_lsqr(ctypes.byref(s._s), _p(b), ctypes.byref(prm), _p(x), _p(var) if want_var else None,
                         ctypes.byref(info))
    if rc != 0:
        raise MemoryError("oracle_lsqr: allocation failed")
    if want_var:
        return x, info.as_dict(), var
    return x, info.as_dict()
