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
        ("n_astro", ctypes.c_int32),
        ("n_ipr", ctypes.c_int32),
        ("npar", ctypes.c_int32),
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
        lib.oracle_lsqr_omp.restype = ctypes.c_int
        lib.oracle_lsqr_omp.argtypes = [S, P, ctypes.POINTER(_Params), P, P, ctypes.POINTER(_Info), ctypes.c_int32]
        lib.oracle_omp_threads.restype = ctypes.c_int32
        lib.oracle_omp_threads.argtypes = []
        for f in (lib.oracle_aprod1_omp, lib.oracle_aprod2_omp):
            f.restype = None
            f.argtypes = [S, P, P]
        _extra_signatures(lib)
        _lib = lib
    return _lib


def _extra_signatures(lib):
    """Signatures of the warm-start reference routines (warm.c)."""
    P = ctypes.c_void_p
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.oracle_bf16.restype = f64
    lib.oracle_bf16.argtypes = [f64]
    lib.oracle_conv_fwd.restype = None
    lib.oracle_conv_fwd.argtypes = [P, i64, i64, i32, P, P, i32, i32, i32, P]
    lib.oracle_conv_bwd.restype = None
    lib.oracle_conv_bwd.argtypes = [P, P, i64, i64, i32, P, i32, i32, P, P, P]
    lib.oracle_mse.restype = f64
    lib.oracle_mse.argtypes = [P, P, i64, P]
    lib.oracle_adam.restype = None
    lib.oracle_adam.argtypes = [P, P, P, P, i64, f64, f64, f64, f64, i32]
    lib.oracle_astro_solve.restype = i64
    lib.oracle_astro_solve.argtypes = [ctypes.POINTER(_Sys), P, P]


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


@dataclass
class System:
    """A system in the paper's storage: A_d (n x npar), knot (M_i's attitude part), instr (I_c, n x n_ipr).

    Sections (Sec. 2): n_astro astrometric (0..5), 12 attitude, n_ipr instrumental (0..6) and n_glob
    global (0..5) coefficients per row. The standard sections (5, 6, n_glob <= 1) use the paper's
    24-slot row; other choices the compact row of n_astro + 12 + n_ipr + n_glob."""

    star_ptr: np.ndarray
    A: np.ndarray
    knot: np.ndarray
    instr: np.ndarray
    n_dfa: int
    n_instr: int
    n_glob: int
    n_astro: int = 5
    n_ipr: int = 6

    def __post_init__(self):
        self.star_ptr = np.ascontiguousarray(self.star_ptr, dtype=np.int64)
        self.A = np.ascontiguousarray(self.A, dtype=np.float64)
        self.knot = np.ascontiguousarray(self.knot, dtype=np.int32)
        self.instr = np.ascontiguousarray(self.instr, dtype=np.int32).reshape(len(self.knot), self.n_ipr)
        std = self.n_astro == 5 and self.n_ipr == 6 and self.n_glob <= 1
        self.npar = 24 if std else self.n_astro + 12 + self.n_ipr + self.n_glob
        assert self.A.shape == (len(self.knot), self.npar), (self.A.shape, self.npar)
        self._s = _Sys(int(self.star_ptr[-1]), len(self.star_ptr) - 1, _p(self.star_ptr), self.n_dfa, self.n_instr,
                       self.n_glob, _p(self.A), _p(self.knot), _p(self.instr), self.n_astro, self.n_ipr, self.npar)

    @property
    def n_rows(self) -> int:
        return int(self.star_ptr[-1])

    @property
    def n_stars(self) -> int:
        return len(self.star_ptr) - 1

    @property
    def n_cols(self) -> int:
        return self.n_astro * self.n_stars + 3 * self.n_dfa + self.n_instr + self.n_glob

    def blocks(self) -> dict:
        """Column ranges of the four sections of x (Sec. 2)."""
        a = self.n_astro * self.n_stars
        t = a + 3 * self.n_dfa
        i = t + self.n_instr
        return {"astro": (0, a), "att": (a, t), "instr": (t, i), "glob": (i, i + self.n_glob)}


def from_host_system(hs) -> System:
    c = hs.cfg
    return System(hs.star_ptr, hs.A, hs.knot, hs.instr, c.n_dfa, c.n_instr, c.n_glob, c.n_astro, c.n_ipr)


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


def lsqr_omp(s: System, b: np.ndarray, itnlim: int, atol: float = 0.0, btol: float = 0.0, conlim: float = 0.0,
             damp: float = 0.0, precond: bool = True, threads: int = 0):
    """The same LSQR with its loops split over the host cores (oracle_omp.c; threads 0 = all);
    returns (x, info dict)."""
    lib = _load()
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(s.n_cols, dtype=np.float64)
    prm = _Params(int(itnlim), atol, btol, conlim, damp, 1 if precond else 0)
    info = _Info()
    rc = lib.oracle_lsqr_omp(ctypes.byref(s._s), _p(b), ctypes.byref(prm), _p(x), None, ctypes.byref(info),
                             int(threads))
    if rc != 0:
        raise MemoryError("oracle_lsqr_omp: allocation failed")
    return x, info.as_dict()


def omp_threads() -> int:
    """Threads the all-cores LSQR uses (1 when the oracle was built without OpenMP)."""
    return int(_load().oracle_omp_threads())


def aprod1_omp(s: System, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert y.dtype == np.float64 and y.flags["C_CONTIGUOUS"] and y.shape == (s.n_rows,)
    _load().oracle_aprod1_omp(ctypes.byref(s._s), _p(x), _p(y))
    return y


def aprod2_omp(s: System, y: np.ndarray, x: np.ndarray) -> np.ndarray:
    y = np.ascontiguousarray(y, dtype=np.float64)
    assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"] and x.shape == (s.n_cols,)
    _load().oracle_aprod2_omp(ctypes.byref(s._s), _p(y), _p(x))
    return x


# ---------------------------------------------------------------- warm start (warm.c)
def bf16(v: float) -> float:
    """binary32 -> bfloat16 -> float, round to nearest even."""
    return _load().oracle_bf16(float(v))


def conv_fwd(inp: np.ndarray, W: np.ndarray, bias: np.ndarray, relu: bool, mirrored: bool = False) -> np.ndarray:
    """One conv1d layer (kernel 5, zero padding 2). inp [nb, L, cin], W [cout, cin, 5], bias [cout]."""
    inp = np.ascontiguousarray(inp, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    bias = np.ascontiguousarray(bias, dtype=np.float64)
    nb, L, cin = inp.shape
    cout = W.shape[0]
    out = np.empty((nb, L, cout))
    _load().oracle_conv_fwd(_p(inp), nb, L, cin, _p(W), _p(bias), cout, int(relu), int(mirrored), _p(out))
    return out


def conv_bwd(inp: np.ndarray, dout: np.ndarray, W: np.ndarray, mirrored: bool = False, want_din: bool = True):
    """Gradients of one layer given dout (w.r.t. the pre-activation output): (din, dW, dbias)."""
    inp = np.ascontiguousarray(inp, dtype=np.float64)
    dout = np.ascontiguousarray(dout, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    nb, L, cin = inp.shape
    cout = W.shape[0]
    din = np.empty_like(inp) if want_din else None
    dW = np.zeros_like(W)
    db = np.zeros(cout)
    _load().oracle_conv_bwd(_p(inp), _p(dout), nb, L, cin, _p(W), cout, int(mirrored), _p(din) if want_din else None,
                            _p(dW), _p(db))
    return din, dW, db


def mse(y: np.ndarray, t: np.ndarray):
    y = np.ascontiguousarray(y, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    g = np.empty_like(y)
    loss = _load().oracle_mse(_p(y), _p(t), y.size, _p(g))
    return loss, g


def adam(w, m, v, g, lr, b1=0.9, b2=0.999, eps=1e-8, step=1):
    """In-place Adam step on float64 arrays."""
    for a in (w, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    g = np.ascontiguousarray(g, dtype=np.float64)
    _load().oracle_adam(_p(w), _p(m), _p(v), _p(g), w.size, lr, b1, b2, eps, int(step))


def astro_solve(s: System, b: np.ndarray, x: np.ndarray) -> int:
    """Per-star n_astro x n_astro astrometric solve given the other parts of x (in place). Returns failed stars."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"]
    return int(_load().oracle_astro_solve(ctypes.byref(s._s), _p(b), _p(x)))


# The network: 6 conv1d layers, 64 channels, kernel 5: 6 -> 64 -> 64 -> 64 -> 64 -> 64 -> 3,
# ReLU after the first five. Parameters are a list of (W [cout, cin, 5], bias [cout]).
NET_CHANNELS = [6, 64, 64, 64, 64, 64, 3]


def net_forward(params, x: np.ndarray, mirrored: bool = False):
    """x [nb, L, 6] -> (y [nb, L, 3], activations: the input of every layer)."""
    acts = [np.ascontiguousarray(x, dtype=np.float64)]
    h = acts[0]
    for i, (W, bias) in enumerate(params):
        last = i == len(params) - 1
        h = conv_fwd(h, W, bias, relu=not last, mirrored=mirrored)
        if not last:
            acts.append(h)
    return h, acts


def net_backward(params, acts, dy: np.ndarray, mirrored: bool = False):
    """Gradients of all parameters given dLoss/dy; acts from net_forward."""
    grads = [None] * len(params)
    d = np.ascontiguousarray(dy, dtype=np.float64)
    for i in range(len(params) - 1, -1, -1):
        W, _ = params[i]
        din, dW, db = conv_bwd(acts[i], d, W, mirrored=mirrored, want_din=i > 0)
        grads[i] = (dW, db)
        if i > 0:
            d = din * (acts[i] > 0.0)  # ReLU of the previous layer
    return grads


def jacobi_features(s: System, b: np.ndarray):
    """Attitude features of the warm start: per knot and axis the Jacobi estimate
    (A^T b)_j / |A_:,j|^2, scaled by its root mean square, and the centred log of
    |A_:,j|^2. Returns (features [n_dfa, 6], scale)."""
    z = aprod2(s, b, np.zeros(s.n_cols))
    p = precond(s)
    a0, a1 = s.blocks()["att"]
    colsq = 1.0 / (p[a0:a1] ** 2)
    jac = z[a0:a1] / colsq
    scale = float(np.sqrt(np.mean(jac ** 2))) or 1.0
    lg = np.log(colsq)
    lg = lg - lg.mean()
    f = np.empty((s.n_dfa, 6))
    for ax in range(3):
        f[:, ax] = jac[ax * s.n_dfa:(ax + 1) * s.n_dfa] / scale
        f[:, 3 + ax] = lg[ax * s.n_dfa:(ax + 1) * s.n_dfa]
    return f, scale
