"""ctypes binding of libgsr (include/gsr.h), same names as the C entry points.

Each ``gsr_*`` function forwards its arguments to the C function of the same
name and returns the integer status; ``Context`` is a small convenience
wrapper that raises ``GsrError`` on a non-zero status. Pointers are plain
integers: ``tensor.data_ptr()``, ``ndarray.ctypes.data`` or 0 for NULL; a
stream is ``torch.cuda.Stream.cuda_stream`` (0 = legacy default stream).
The library must have been built (``__graft_entry__.build()``); importing
this module without it raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import enum
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libgsr.so")

GSR_FP64, GSR_FP32 = 0, 1
GSR_HOST, GSR_DEVICE = 0, 1
GSR_AOS, GSR_SOA = 0, 1
GSR_PLAIN, GSR_MIXED = 0, 1
GSR_WARM_NONE, GSR_WARM_JACOBI, GSR_WARM_LEARNED = 0, 1, 2


class Status(enum.IntEnum):
    OK = 0
    EINVAL = 1
    ENOMEM = 2
    ECUDA = 3
    ESTATE = 4
    ENUMERIC = 5
    ETIMEOUT = 6


class SolveParams(ctypes.Structure):
    _fields_ = [
        ("itnlim", ctypes.c_int32),
        ("atol", ctypes.c_double),
        ("btol", ctypes.c_double),
        ("conlim", ctypes.c_double),
        ("damp", ctypes.c_double),
        ("precond", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("warm", ctypes.c_int32),
        ("weights_path", ctypes.c_char_p),
        ("timeout_s", ctypes.c_double),
        ("graph_k", ctypes.c_int32),
        ("where", ctypes.c_int32),
        ("inner_itn", ctypes.c_int32),
        ("inner_tol", ctypes.c_double),
        ("refine_tol", ctypes.c_double),
        ("max_outer", ctypes.c_int32),
        ("inner_itn_next", ctypes.c_int32),
        ("refine_grad", ctypes.c_int32),
        ("inner_fused", ctypes.c_int32),
        ("inner_close", ctypes.c_int32),
    ]


class SolveInfo(ctypes.Structure):
    _fields_ = [
        ("istop", ctypes.c_int32),
        ("itn", ctypes.c_int32),
        ("outer_itn", ctypes.c_int32),
        ("r1norm", ctypes.c_double),
        ("r2norm", ctypes.c_double),
        ("anorm", ctypes.c_double),
        ("acond", ctypes.c_double),
        ("arnorm", ctypes.c_double),
        ("xnorm", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("ms_warm", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """Load libgsr.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise RuntimeError(f"libgsr.so not built ({library_path}); run __graft_entry__.build()")
        L = ctypes.CDLL(library_path)
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "gsr_create": (I32, [ctypes.POINTER(P), I64, I32, P, I32, I32, I32, I32, I32]),
            "gsr_create_sections": (I32, [ctypes.POINTER(P), I64, I32, P, I32, I32, I32, I32, I32, I32, I32]),
            "gsr_sections": (I32, [P, P, P, P, P]),
            "gsr_destroy": (I32, [P]),
            "gsr_last_error": (ctypes.c_char_p, [P]),
            "gsr_dims": (I32, [P, P, P]),
            "gsr_set_rows": (I32, [P, I64, I64, P, I32, I32, I64, P, P, I32, P]),
            "gsr_set_rhs": (I32, [P, P, I32, P]),
            "gsr_set_system": (I32, [P, P, I32, P, P, P, I32, P]),
            "gsr_aprod1": (I32, [P, P, P, P]),
            "gsr_aprod2": (I32, [P, P, P, P]),
            "gsr_aprod1_f32": (I32, [P, P, P, P]),
            "gsr_aprod2_f32": (I32, [P, P, P, P]),
            "gsr_aprod2_plan": (I32, [P, P, P, P, P]),
            "gsr_aprod12_f32": (I32, [P, P, P, P, ctypes.c_float, P]),
            "gsr_residual": (I32, [P, P, P, P]),
            "gsr_residual_static": (I32, [P, P, P, P]),
            "gsr_default_params": (None, [ctypes.POINTER(SolveParams)]),
            "gsr_fp64_fma_rate": (I32, [I32, P]),
            "gsr_tc_wait_check": (I32, [I32, ctypes.c_double, P, P]),
            "gsr_net_num_params": (I64, []),
            "gsr_net_create": (I32, [ctypes.POINTER(P), I32]),
            "gsr_net_destroy": (I32, [P]),
            "gsr_net_last_error": (ctypes.c_char_p, [P]),
            "gsr_net_set_params": (I32, [P, P, I64]),
            "gsr_net_get_params": (I32, [P, P, I64]),
            "gsr_net_save": (I32, [P, ctypes.c_char_p]),
            "gsr_net_load": (I32, [P, ctypes.c_char_p]),
            "gsr_net_forward": (I32, [P, P, I64, I64, P, P]),
            "gsr_net_train_step": (I32, [P, P, P, I64, I64, ctypes.c_float, P, P]),
            "gsr_net_gradients": (I32, [P, P, P, I64, I64, P, I64, P, P]),
            "gsr_net_layer_forward": (I32, [P, I32, P, I64, I64, P, P]),
            "gsr_net_layer_backward": (I32, [P, I32, P, P, I64, I64, P, P, P, P]),
            "gsr_net_apply_gradients": (I32, [P, P, I64, ctypes.c_float, P]),
            "gsr_warm_features": (I32, [P, P, P, P]),
            "gsr_warm_start": (I32, [P, P, P, P]),
            "gsr_lsqr_solve": (I32, [P, ctypes.POINTER(SolveParams), P, P, P, ctypes.POINTER(SolveInfo), P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# ---------------------------------------------------------------- same-name functions
def gsr_create(n_stars, obs_per_star, star_ptr, n_dfa, n_instr, n_glob, value_precision, device):
    """Returns (status, ctx handle). star_ptr: host pointer (int) or 0."""
    h = ctypes.c_void_p()
    st = lib().gsr_create(ctypes.byref(h), n_stars, obs_per_star, star_ptr or None, n_dfa, n_instr, n_glob,
                          value_precision, device)
    return st, h.value


def gsr_create_sections(n_stars, obs_per_star, star_ptr, n_astro, n_dfa, n_instr, n_ipr, n_glob, value_precision,
                        device):
    """Returns (status, ctx handle). star_ptr: host pointer (int) or 0."""
    h = ctypes.c_void_p()
    st = lib().gsr_create_sections(ctypes.byref(h), n_stars, obs_per_star, star_ptr or None, n_astro, n_dfa, n_instr,
                                   n_ipr, n_glob, value_precision, device)
    return st, h.value


def gsr_sections(ctx):
    """Returns (status, n_astro, n_ipr, n_glob, row_width)."""
    v = [ctypes.c_int32() for _ in range(4)]
    st = lib().gsr_sections(ctx, *[ctypes.byref(q) for q in v])
    return (st, *[q.value for q in v])


def gsr_aprod2_plan(ctx, stream=0):
    """Returns (status, passes, fx_bits, ins_group)."""
    v = [ctypes.c_int32() for _ in range(3)]
    st = lib().gsr_aprod2_plan(ctx, stream, *[ctypes.byref(q) for q in v])
    return (st, *[q.value for q in v])


def gsr_destroy(ctx):
    return lib().gsr_destroy(ctx)


def gsr_last_error(ctx) -> str:
    r = lib().gsr_last_error(ctx)
    return r.decode() if r else ""


def gsr_dims(ctx):
    nr, nc = ctypes.c_int64(), ctypes.c_int64()
    st = lib().gsr_dims(ctx, ctypes.byref(nr), ctypes.byref(nc))
    return st, nr.value, nc.value


def gsr_set_rows(ctx, row0, nrows, values, values_fp32, layout, plane_stride, att_knot, instr_col, where, stream=0):
    return lib().gsr_set_rows(ctx, row0, nrows, values or None, values_fp32, layout, plane_stride, att_knot or None,
                              instr_col or None, where, stream or None)


def gsr_set_rhs(ctx, b, where, stream=0):
    return lib().gsr_set_rhs(ctx, b or None, where, stream or None)


def gsr_set_system(ctx, values, values_fp32, att_knot, instr_col, b, where, stream=0):
    return lib().gsr_set_system(ctx, values or None, values_fp32, att_knot or None, instr_col or None, b or None,
                                where, stream or None)


def gsr_aprod1(ctx, x, y, stream=0):
    return lib().gsr_aprod1(ctx, x or None, y or None, stream or None)


def gsr_aprod2(ctx, y, x, stream=0):
    return lib().gsr_aprod2(ctx, y or None, x or None, stream or None)


def gsr_aprod1_f32(ctx, x, y, stream=0):
    return lib().gsr_aprod1_f32(ctx, x or None, y or None, stream or None)


def gsr_aprod2_f32(ctx, y, x, stream=0):
    return lib().gsr_aprod2_f32(ctx, y or None, x or None, stream or None)


def gsr_aprod12_f32(ctx, x, y, z, coef, stream=0):
    return lib().gsr_aprod12_f32(ctx, x or None, y or None, z or None, coef, stream or None)


def gsr_residual(ctx, x, r, stream=0):
    return lib().gsr_residual(ctx, x or None, r or None, stream or None)


def gsr_residual_static(ctx, x, r, stream=0):
    return lib().gsr_residual_static(ctx, x or None, r or None, stream or None)


def gsr_default_params() -> SolveParams:
    p = SolveParams()
    lib().gsr_default_params(ctypes.byref(p))
    return p


def gsr_lsqr_solve(ctx, params: SolveParams, x0, x_out, se_out, info: SolveInfo, stream=0):
    return lib().gsr_lsqr_solve(ctx, ctypes.byref(params), x0 or None, x_out or None, se_out or None,
                                ctypes.byref(info), stream or None)


def gsr_net_num_params() -> int:
    return lib().gsr_net_num_params()


def gsr_net_create(device=0):
    h = ctypes.c_void_p()
    st = lib().gsr_net_create(ctypes.byref(h), device)
    return st, h.value


def gsr_net_destroy(net):
    return lib().gsr_net_destroy(net)


def gsr_net_last_error(net) -> str:
    r = lib().gsr_net_last_error(net)
    return r.decode() if r else ""


def gsr_net_set_params(net, params, count):
    return lib().gsr_net_set_params(net, params or None, count)


def gsr_net_get_params(net, params, count):
    return lib().gsr_net_get_params(net, params or None, count)


def gsr_net_save(net, path: str):
    return lib().gsr_net_save(net, path.encode())


def gsr_net_load(net, path: str):
    return lib().gsr_net_load(net, path.encode())


def gsr_net_forward(net, x, batch, length, out, stream=0):
    return lib().gsr_net_forward(net, x or None, batch, length, out or None, stream or None)


def gsr_net_train_step(net, x, target, batch, length, lr, loss_ptr, stream=0):
    return lib().gsr_net_train_step(net, x or None, target or None, batch, length, lr, loss_ptr or None,
                                    stream or None)


def gsr_net_gradients(net, x, target, batch, length, grads, count, loss_ptr, stream=0):
    return lib().gsr_net_gradients(net, x or None, target or None, batch, length, grads or None, count,
                                   loss_ptr or None, stream or None)


def gsr_net_layer_forward(net, layer, x, batch, length, out, stream=0):
    return lib().gsr_net_layer_forward(net, layer, x or None, batch, length, out or None, stream or None)


def gsr_net_layer_backward(net, layer, x, dout, batch, length, din, dW, db, stream=0):
    return lib().gsr_net_layer_backward(net, layer, x or None, dout or None, batch, length, din or None, dW or None,
                                        db or None, stream or None)


def gsr_net_apply_gradients(net, grads, count, lr, stream=0):
    return lib().gsr_net_apply_gradients(net, grads or None, count, lr, stream or None)


def gsr_warm_features(ctx, feats, scale_ptr, stream=0):
    return lib().gsr_warm_features(ctx, feats or None, scale_ptr or None, stream or None)


def gsr_warm_start(ctx, net, x0, stream=0):
    return lib().gsr_warm_start(ctx, net or None, x0 or None, stream or None)


def gsr_fp64_fma_rate(device, tflops_ptr):
    return lib().gsr_fp64_fma_rate(device, tflops_ptr or None)


def gsr_tc_wait_check(device, limit_ms, timed_out_ptr, waited_ms_ptr):
    return lib().gsr_tc_wait_check(device, limit_ms, timed_out_ptr or None, waited_ms_ptr or None)


def tc_wait_check(device=0, limit_ms=20.0):
    """(timed_out, waited_ms) of the tensor-core kernels' bounded wait run out on purpose."""
    t, w = ctypes.c_int32(), ctypes.c_double()
    st = gsr_tc_wait_check(device, limit_ms, ctypes.addressof(t), ctypes.addressof(w))
    if st != 0:
        raise GsrError(st, "gsr_tc_wait_check failed")
    return t.value, w.value


def dfma_probe_tflops(device=0) -> float:
    """The device's binary64 FMA rate in TFLOP/s (the ceiling of the binary64 aprods)."""
    v = ctypes.c_double()
    st = gsr_fp64_fma_rate(device, ctypes.addressof(v))
    if st != 0:
        raise GsrError(st, "gsr_fp64_fma_rate failed")
    return v.value


# ---------------------------------------------------------------- convenience wrapper
class GsrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{Status(status).name}: {msg}")
        self.status = Status(status)


def _ptr(a) -> int:
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _where(a) -> int:
    return GSR_DEVICE if hasattr(a, "is_cuda") and a.is_cuda else GSR_HOST


class Net:
    """Owns one gsr_net (the warm start's conv1d network)."""

    def __init__(self, device=0):
        st, h = gsr_net_create(device)
        if st != 0:
            raise GsrError(st, "gsr_net_create failed")
        self.h = h
        self.n_params = gsr_net_num_params()

    def _check(self, st):
        if st != 0:
            raise GsrError(st, gsr_net_last_error(self.h))

    def close(self):
        if getattr(self, "h", None):
            gsr_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        import numpy as np

        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(gsr_net_set_params(self.h, p.ctypes.data, p.size))

    def get_params(self):
        import numpy as np

        p = np.empty(self.n_params, dtype=np.float32)
        self._check(gsr_net_get_params(self.h, p.ctypes.data, p.size))
        return p

    def save(self, path):
        self._check(gsr_net_save(self.h, str(path)))

    def load(self, path):
        self._check(gsr_net_load(self.h, str(path)))

    def forward(self, x, out, stream=0):
        """x: CUDA float32 [batch, len, 6]; out: CUDA float32 [batch, len, 3]."""
        b, n, _ = x.shape
        self._check(gsr_net_forward(self.h, x.data_ptr(), b, n, out.data_ptr(), stream))

    def train_step(self, x, target, lr, stream=0):
        b, n, _ = x.shape
        loss = ctypes.c_double()
        self._check(gsr_net_train_step(self.h, x.data_ptr(), target.data_ptr(), b, n, lr, ctypes.addressof(loss),
                                       stream))
        return loss.value

    def gradients(self, x, target, stream=0):
        import numpy as np

        b, n, _ = x.shape
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(gsr_net_gradients(self.h, x.data_ptr(), target.data_ptr(), b, n, g.ctypes.data, g.size,
                                      ctypes.addressof(loss), stream))
        return g, loss.value

    def layer_forward(self, layer, x, out, stream=0):
        """One layer before its ReLU: x CUDA float32 [batch, len, cin], out [batch, len, cout]."""
        b, n, _ = x.shape
        self._check(gsr_net_layer_forward(self.h, layer, x.data_ptr(), b, n, out.data_ptr(), stream))

    def layer_backward(self, layer, x, dout, din, dW, db, stream=0):
        """Gradients of one layer given dout (w.r.t. its output before the ReLU); din may be None."""
        b, n, _ = x.shape
        self._check(gsr_net_layer_backward(self.h, layer, x.data_ptr(), dout.data_ptr(), b, n,
                                           din.data_ptr() if din is not None else 0, dW.data_ptr(), db.data_ptr(),
                                           stream))

    def apply_gradients(self, grads, lr, stream=0):
        """One Adam step with the given gradients (host float32, parameter layout)."""
        import numpy as np

        g = np.ascontiguousarray(grads, dtype=np.float32)
        self._check(gsr_net_apply_gradients(self.h, g.ctypes.data, g.size, lr, stream))


class Context:
    """Owns one gsr_ctx. Arrays may be numpy arrays (host) or torch tensors (host or CUDA).

    The paper's standard sections (n_astro = 5, n_ipr = 6, n_glob 0 or 1) create the context with
    gsr_create (rows of 24 coefficients); any other choice with gsr_create_sections (compact rows of
    n_astro + 12 + n_ipr + n_glob coefficients and n_ipr instrumental columns)."""

    def __init__(self, n_stars, obs_per_star=0, star_ptr=None, n_dfa=4, n_instr=6, n_glob=1, fp32=False, device=0,
                 n_astro=5, n_ipr=6):
        import numpy as np

        self._sp = None if star_ptr is None else np.ascontiguousarray(star_ptr, dtype=np.int64)
        prec = GSR_FP32 if fp32 else GSR_FP64
        if n_astro == 5 and n_ipr == 6 and n_glob in (0, 1):
            st, h = gsr_create(n_stars, obs_per_star, _ptr(self._sp), n_dfa, n_instr, n_glob, prec, device)
        else:
            st, h = gsr_create_sections(n_stars, obs_per_star, _ptr(self._sp), n_astro, n_dfa, n_instr, n_ipr,
                                        n_glob, prec, device)
        if st != 0:
            raise GsrError(st, "gsr_create failed")
        self.h = h
        _, self.n_rows, self.n_cols = gsr_dims(h)
        _, self.n_astro, self.n_ipr, self.n_glob, self.row_width = gsr_sections(h)

    def _check(self, st):
        if st != 0:
            raise GsrError(st, gsr_last_error(self.h))

    def close(self):
        if getattr(self, "h", None):
            gsr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_system(self, A, knot, instr, b=None, stream=0):
        fp32 = 1 if str(A.dtype).endswith("float32") else 0
        self._check(gsr_set_system(self.h, _ptr(A), fp32, _ptr(knot), _ptr(instr), _ptr(b), _where(A), stream))

    def set_rows(self, row0, nrows, vals, knot, instr, layout=GSR_AOS, plane_stride=0, stream=0):
        fp32 = 1 if str(vals.dtype).endswith("float32") else 0
        self._check(gsr_set_rows(self.h, row0, nrows, _ptr(vals), fp32, layout, plane_stride, _ptr(knot),
                                 _ptr(instr), _where(vals), stream))

    def set_rhs(self, b, stream=0):
        self._check(gsr_set_rhs(self.h, _ptr(b), _where(b), stream))

    def aprod1(self, x, y, stream=0):
        self._check(gsr_aprod1(self.h, _ptr(x), _ptr(y), stream))

    def aprod2(self, y, x, stream=0):
        self._check(gsr_aprod2(self.h, _ptr(y), _ptr(x), stream))

    def aprod1_f32(self, x, y, stream=0):
        self._check(gsr_aprod1_f32(self.h, _ptr(x), _ptr(y), stream))

    def aprod2_f32(self, y, x, stream=0):
        self._check(gsr_aprod2_f32(self.h, _ptr(y), _ptr(x), stream))

    def aprod12_f32(self, x, y, z, coef=1.0, stream=0):
        """y <- A x + coef y, then z += A^T y with the new y (binary32; z binary64)."""
        self._check(gsr_aprod12_f32(self.h, _ptr(x), _ptr(y), _ptr(z), coef, stream))

    def aprod2_plan(self, stream=0):
        """The binary32 aprod 2's form on the loaded rows: {"passes", "fx_bits", "ins_group"}."""
        st, passes, bits, grp = gsr_aprod2_plan(self.h, stream)
        self._check(st)
        return {"passes": passes, "fx_bits": bits, "ins_group": grp}

    def residual(self, x, r, stream=0):
        self._check(gsr_residual(self.h, _ptr(x), _ptr(r), stream))

    def warm_features(self, feats, stream=0):
        """feats: CUDA float32 [n_dfa, 6]; returns the scale."""
        sc = ctypes.c_double()
        self._check(gsr_warm_features(self.h, feats.data_ptr(), ctypes.addressof(sc), stream))
        return sc.value

    def warm_start(self, x0, net=None, stream=0):
        """x0: CUDA float64 [n_cols] receives the start vector."""
        self._check(gsr_warm_start(self.h, net.h if net is not None else 0, x0.data_ptr(), stream))

    def solve(self, x_out, x0=None, se_out=None, stream=0, **kw):
        p = gsr_default_params()
        fields = {f for f, _ in SolveParams._fields_}
        for k, v in kw.items():
            if k not in fields:
                raise TypeError(f"unknown solve parameter {k!r}")
            if k == "weights_path" and isinstance(v, str):
                v = v.encode()
            setattr(p, k, v)
        p.where = _where(x_out)
        info = SolveInfo()
        st = gsr_lsqr_solve(self.h, p, _ptr(x0), _ptr(x_out), _ptr(se_out), info, stream)
        if st != 0:
            raise GsrError(st, gsr_last_error(self.h) + f" (info: {info.as_dict()})")
        return info.as_dict()
