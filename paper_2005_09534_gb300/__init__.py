"""Python binding of libpolfed.so, the GB300 POLFED hot path (C ABI in include/polfed.h).

Argument marshalling only: every step runs in the CUDA library.  Device
buffers are passed as raw device pointers (anything with ``data_ptr()``, such
as torch CUDA tensors, or a plain integer address); host arrays are numpy.
The library must have been built (``paper_2005_09534_gb300.build.build()``);
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int32, c_int64, c_size_t, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpolfed.so")

POLFED_OK = 0
POLFED_EINVAL = -1
POLFED_ENOMEM = -2
POLFED_ECUDA = -3
POLFED_EBOUNDS = -4
POLFED_ENOCONV = -5
POLFED_ETIMEOUT = -6

F64, F32, DF64 = 0, 1, 2

EXPORTED = ["polfed_opts_default", "polfed_basis_build", "polfed_h_apply", "polfed_cheb_filter",
            "polfed_cheb_filter_static",
            "polfed_ctx_create", "polfed_ctx_destroy", "polfed_ctx_set_stream", "polfed_block_lanczos",
            "polfed_eigs", "polfed_last_error"]


class PolfedError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"polfed error {code}: {msg}")
        self.code = code


class CModel(ctypes.Structure):
    _fields_ = [("L", c_int32), ("periodic", c_int32), ("J1", c_double), ("J2", c_double),
                ("Delta", c_double), ("h", POINTER(c_double))]


class COpts(ctypes.Structure):
    _fields_ = [("p", c_double), ("k_margin", c_double), ("tol_conv", c_double), ("tol_resid", c_double),
                ("cols_factor", c_double), ("precision", c_int32), ("bounds_steps", c_int32),
                ("verbose", c_int32), ("reserved", c_int32), ("seed", c_uint64)]


class CStats(ctypes.Structure):
    _fields_ = [("K", c_int32), ("m", c_int32), ("n_b", c_int32), ("n_conv", c_int32),
                ("n_ritz_checks", c_int32), ("status", c_int32), ("n_refine", c_int32), ("refine_K", c_int32),
                ("dim", c_int64), ("matvec_cols", c_int64),
                ("E_min", c_double), ("E_max", c_double), ("e_lo", c_double), ("e_hi", c_double),
                ("sigma", c_double), ("target", c_double), ("rho_sigma", c_double), ("max_resid", c_double),
                ("t_bounds", c_double), ("t_filter", c_double), ("t_reorth", c_double), ("t_qr", c_double),
                ("t_teig", c_double), ("t_ritz", c_double), ("t_total", c_double),
                ("n_launches", c_int64), ("n_step_launches", c_int64), ("step_gpu_s", c_double),
                ("step_alg_bytes", c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load libpolfed.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not built; run paper_2005_09534_gb300.build.build()")
    lib = ctypes.CDLL(path)
    lib.polfed_last_error.restype = ctypes.c_char_p
    lib.polfed_opts_default.argtypes = [POINTER(COpts)]
    lib.polfed_opts_default.restype = None
    lib.polfed_basis_build.argtypes = [c_int32, c_int32, c_void_p, POINTER(c_int64), c_void_p]
    lib.polfed_h_apply.argtypes = [POINTER(CModel), c_void_p, c_int64, c_double, c_double, c_void_p, c_void_p,
                                   c_int32, c_int32, c_void_p]
    lib.polfed_cheb_filter.argtypes = [POINTER(CModel), c_void_p, c_int64, c_double, c_double, c_double, c_int32,
                                       POINTER(c_double), c_void_p, c_void_p, c_int32, c_int32, c_void_p]
    lib.polfed_cheb_filter_static.argtypes = lib.polfed_cheb_filter.argtypes
    lib.polfed_ctx_create.argtypes = [c_int32, c_size_t, POINTER(c_void_p)]
    lib.polfed_ctx_destroy.argtypes = [c_void_p]
    lib.polfed_ctx_destroy.restype = None
    lib.polfed_ctx_set_stream.argtypes = [c_void_p, c_void_p]
    lib.polfed_block_lanczos.argtypes = [c_void_p, POINTER(CModel), c_double, c_double, c_double, c_int32, c_int32,
                                         c_int32, c_void_p, POINTER(c_double), POINTER(c_double), POINTER(c_int32)]
    lib.polfed_eigs.argtypes = [c_void_p, POINTER(CModel), c_double, c_int32, c_int32, c_int32, POINTER(COpts),
                                POINTER(c_double), c_void_p, POINTER(c_double), POINTER(CStats)]
    for name in EXPORTED:
        getattr(lib, name)
    _lib = lib
    return lib


def last_error() -> str:
    return load().polfed_last_error().decode()


def _check(rc, allow=()):
    if rc != POLFED_OK and rc not in allow:
        raise PolfedError(rc, last_error())
    return rc


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Model:
    """Eq. (1) parameters; keeps the host field array alive while in use."""

    def __init__(self, L, J1, J2, Delta, h, periodic=True):
        self.h = np.ascontiguousarray(np.asarray(h, dtype=np.float64))
        assert self.h.shape == (int(L),)
        self.c = CModel(int(L), 1 if periodic else 0, float(J1), float(J2), float(Delta),
                        self.h.ctypes.data_as(POINTER(c_double)))

    @classmethod
    def of(cls, m):
        if isinstance(m, Model):
            return m
        return cls(m.L, m.J1, m.J2, m.Delta, m.h, m.periodic)


def opts_default() -> COpts:
    o = COpts()
    load().polfed_opts_default(byref(o))
    return o


def basis_build(L, n_up, d_states=None, stream=None) -> int:
    dim = c_int64(0)
    _check(load().polfed_basis_build(int(L), int(n_up), _ptr(d_states), byref(dim), _stream(stream)))
    return dim.value


def h_apply(model, d_states, dim, e_lo, e_hi, X, Y, n_b, dtype, stream=None):
    m = Model.of(model)
    return _check(load().polfed_h_apply(byref(m.c), _ptr(d_states), int(dim), float(e_lo), float(e_hi), _ptr(X),
                                        _ptr(Y), int(n_b), int(dtype), _stream(stream)))


def cheb_filter(model, d_states, dim, e_lo, e_hi, sigma, K, X, Y, n_b, dtype, coeffs=None, stream=None,
                allow_bounds_error=False):
    m = Model.of(model)
    cptr = None
    if coeffs is not None:
        coeffs = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
        assert coeffs.shape == (int(K) + 1,)
        cptr = coeffs.ctypes.data_as(POINTER(c_double))
    rc = load().polfed_cheb_filter(byref(m.c), _ptr(d_states), int(dim), float(e_lo), float(e_hi), float(sigma),
                                   int(K), cptr, _ptr(X), _ptr(Y), int(n_b), int(dtype), _stream(stream))
    return _check(rc, allow=(POLFED_EBOUNDS,) if allow_bounds_error else ())


def cheb_filter_static(model, d_states, dim, e_lo, e_hi, sigma, K, X, Y, n_b, dtype, coeffs=None, stream=None):
    """polfed_cheb_filter_static: the filter without any device allocation (fixed
    32 MiB device array shared by all calls; L <= 18)."""
    m = Model.of(model)
    cptr = None
    if coeffs is not None:
        coeffs = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
        assert coeffs.shape == (int(K) + 1,)
        cptr = coeffs.ctypes.data_as(POINTER(c_double))
    rc = load().polfed_cheb_filter_static(byref(m.c), _ptr(d_states), int(dim), float(e_lo), float(e_hi),
                                          float(sigma), int(K), cptr, _ptr(X), _ptr(Y), int(n_b), int(dtype),
                                          _stream(stream))
    return _check(rc)


class Ctx:
    """polfed_ctx: device, stream, cuSOLVER handle and workspace."""

    def __init__(self, device=0, workspace_bytes=0):
        self.lib = load()
        h = c_void_p()
        _check(self.lib.polfed_ctx_create(int(device), int(workspace_bytes), byref(h)))
        self.h = h

    def close(self):
        if self.h:
            self.lib.polfed_ctx_destroy(self.h)
            self.h = c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _check(self.lib.polfed_ctx_set_stream(self.h, _stream(stream)))


def ctx_create(device=0, workspace_bytes=0) -> Ctx:
    return Ctx(device, workspace_bytes)


def block_lanczos(ctx, model, e_lo, e_hi, sigma, K, n_b, N_ev, d_evecs=None, allow_noconv=False):
    m = Model.of(model)
    evals = np.zeros(N_ev)
    resid = np.zeros(N_ev)
    n_conv = c_int32(0)
    rc = load().polfed_block_lanczos(ctx.h, byref(m.c), float(e_lo), float(e_hi), float(sigma), int(K), int(n_b),
                                     int(N_ev), _ptr(d_evecs), evals.ctypes.data_as(POINTER(c_double)),
                                     resid.ctypes.data_as(POINTER(c_double)), byref(n_conv))
    _check(rc, allow=(POLFED_ENOCONV,) if allow_noconv else ())
    n = n_conv.value
    return evals[:n], resid[:n], rc


def eigs(ctx, model, eps_target, N_ev, K=0, n_b=64, opts=None, d_evecs=None, allow_noconv=False):
    """polfed_eigs: returns (evals, resid, stats dict, status)."""
    m = Model.of(model)
    o = opts if opts is not None else opts_default()
    evals = np.zeros(N_ev)
    resid = np.zeros(N_ev)
    st = CStats()
    rc = load().polfed_eigs(ctx.h, byref(m.c), float(eps_target), int(N_ev), int(K), int(n_b), byref(o),
                            evals.ctypes.data_as(POINTER(c_double)), _ptr(d_evecs),
                            resid.ctypes.data_as(POINTER(c_double)), byref(st))
    _check(rc, allow=(POLFED_ENOCONV,) if allow_noconv else ())
    return evals, resid, st.as_dict(), rc
