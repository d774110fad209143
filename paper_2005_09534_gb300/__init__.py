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
from ctypes import POINTER, byref, c_double, c_float, c_int32, c_int64, c_size_t, c_uint64, c_void_p

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

DOS_MOMENTS, DOS_GAMMA, DOS_KPM, DOS_HINT = 0, 1, 2, 3

PHASE_START, PHASE_BLOCK, PHASE_REFINE, PHASE_END = 0, 1, 2, 3

# void (*)(void* user, int32_t phase, int32_t index)
PROGRESS_FN = ctypes.CFUNCTYPE(None, c_void_p, c_int32, c_int32)

EXPORTED = ["polfed_opts_default", "polfed_basis_build", "polfed_h_apply", "polfed_cheb_filter",
            "polfed_cheb_filter_cols", "polfed_cheb_filter_static",
            "polfed_ctx_create", "polfed_ctx_destroy", "polfed_ctx_set_stream", "polfed_ctx_set_progress",
            "polfed_get_counters", "polfed_ctx_history", "polfed_block_lanczos",
            "polfed_eigs", "polfed_spectral_bounds", "polfed_kpm_moments", "polfed_kpm_count",
            "polfed_spectral_labels", "polfed_mlp_create", "polfed_mlp_destroy", "polfed_mlp_num_params",
            "polfed_mlp_set_params", "polfed_mlp_get_params", "polfed_mlp_set_scaling", "polfed_mlp_forward",
            "polfed_mlp_grad", "polfed_mlp_train_step", "polfed_mlp_features", "polfed_mlp_targets",
            "polfed_mlp_predict", "polfed_cheb_filter_batched", "polfed_eigs_batched", "polfed_gap_ratio",
            "polfed_entanglement_entropy", "polfed_set_wait_limit", "polfed_last_error"]


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
                ("verbose", c_int32), ("dos_rule", c_int32), ("seed", c_uint64), ("rho_hint", c_double),
                ("emin_hint", c_double), ("emax_hint", c_double), ("kpm_moments", c_int32),
                ("kpm_vectors", c_int32), ("tol_refine", c_double)]


class CStats(ctypes.Structure):
    _fields_ = [("K", c_int32), ("m", c_int32), ("n_b", c_int32), ("n_conv", c_int32),
                ("n_ritz_checks", c_int32), ("status", c_int32), ("n_refine", c_int32), ("refine_K", c_int32),
                ("dim", c_int64), ("matvec_cols", c_int64),
                ("E_min", c_double), ("E_max", c_double), ("e_lo", c_double), ("e_hi", c_double),
                ("sigma", c_double), ("target", c_double), ("rho_sigma", c_double), ("max_resid", c_double),
                ("t_bounds", c_double), ("t_filter", c_double), ("t_reorth", c_double), ("t_qr", c_double),
                ("t_teig", c_double), ("t_ritz", c_double), ("t_total", c_double),
                ("n_launches", c_int64), ("n_step_launches", c_int64), ("step_gpu_s", c_double),
                ("step_alg_bytes", c_double), ("dos_rule", c_int32), ("bounds_from_hint", c_int32),
                ("n_restarts", c_int32), ("fallback_df64", c_int32), ("kind_launches", c_int64 * 3),
                ("kind_gpu_s", c_double * 3), ("kind_alg_bytes", c_double * 3)]

    def as_dict(self):
        d = {}
        for f, _ in self._fields_:
            v = getattr(self, f)
            d[f] = list(v) if f.startswith("kind_") else v
        return d


class CCounters(ctypes.Structure):
    _fields_ = [("launches", c_int64), ("step_launches", c_int64), ("step_gpu_s", c_double),
                ("step_alg_bytes", c_double), ("kind_launches", c_int64 * 3), ("kind_gpu_s", c_double * 3),
                ("kind_alg_bytes", c_double * 3)]

    def as_dict(self):
        return {f: (list(getattr(self, f)) if f.startswith("kind_") else getattr(self, f)) for f, _ in self._fields_}


class CConvPoint(ctypes.Structure):
    _fields_ = [("step", c_int32), ("cols", c_int32), ("n_conv", c_int32), ("n_acc", c_int32),
                ("attempt", c_int32), ("reserved", c_int32), ("theta_nev", c_double), ("max_res_top", c_double)]


class CBatchInfo(ctypes.Structure):
    _fields_ = [("n_b", c_int32), ("ctas_per_sm", c_int32), ("rounds", c_int32), ("workers", c_int32),
                ("n_width16", c_int32), ("n_width32", c_int32), ("n_width64", c_int32), ("reserved", c_int32),
                ("t_total", c_double), ("t_tune", c_double), ("filter_gpu_s", c_double),
                ("filter_alg_bytes", c_double), ("tune_step_s", c_double * 6), ("n_launches", c_int64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "tune_step_s"}
        d["tune_step_s"] = [[self.tune_step_s[2 * w + c] for c in range(2)] for w in range(3)]
        return d


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
    lib.polfed_cheb_filter_cols.argtypes = [POINTER(CModel), c_void_p, c_int64, c_double, c_double, c_int32,
                                            POINTER(c_double), c_void_p, c_void_p, c_int32, c_void_p]
    lib.polfed_ctx_create.argtypes = [c_int32, c_size_t, POINTER(c_void_p)]
    lib.polfed_ctx_destroy.argtypes = [c_void_p]
    lib.polfed_ctx_destroy.restype = None
    lib.polfed_ctx_set_stream.argtypes = [c_void_p, c_void_p]
    lib.polfed_ctx_set_progress.argtypes = [c_void_p, PROGRESS_FN, c_void_p]
    lib.polfed_get_counters.argtypes = [POINTER(CCounters)]
    lib.polfed_ctx_history.argtypes = [c_void_p, POINTER(CConvPoint), c_int32, POINTER(c_int32)]
    lib.polfed_block_lanczos.argtypes = [c_void_p, POINTER(CModel), c_double, c_double, c_double, c_int32, c_int32,
                                         c_int32, c_void_p, POINTER(c_double), POINTER(c_double), POINTER(c_int32)]
    lib.polfed_eigs.argtypes = [c_void_p, POINTER(CModel), c_double, c_int32, c_int32, c_int32, POINTER(COpts),
                                POINTER(c_double), c_void_p, POINTER(c_double), POINTER(CStats)]
    lib.polfed_spectral_bounds.argtypes = [c_void_p, POINTER(CModel), POINTER(c_double)]
    lib.polfed_kpm_moments.argtypes = [POINTER(CModel), c_void_p, c_int64, c_double, c_double, c_int32, c_void_p,
                                       c_int32, c_int32, POINTER(c_double), c_void_p]
    lib.polfed_kpm_count.argtypes = [POINTER(c_double), c_int32, c_double, c_double, POINTER(c_double)]
    lib.polfed_spectral_labels.argtypes = [c_void_p, POINTER(CModel), c_double, c_int32, c_int32, POINTER(c_double)]
    lib.polfed_mlp_create.argtypes = [c_int32, c_int32, c_int32, c_uint64, POINTER(c_void_p)]
    lib.polfed_mlp_destroy.argtypes = [c_void_p]
    lib.polfed_mlp_destroy.restype = None
    lib.polfed_mlp_num_params.argtypes = [c_void_p]
    lib.polfed_mlp_set_params.argtypes = [c_void_p, POINTER(c_float)]
    lib.polfed_mlp_get_params.argtypes = [c_void_p, POINTER(c_float)]
    lib.polfed_mlp_set_scaling.argtypes = [c_void_p] + [POINTER(c_float)] * 4
    lib.polfed_mlp_forward.argtypes = [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]
    lib.polfed_mlp_grad.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, POINTER(c_float), c_void_p]
    lib.polfed_mlp_train_step.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, c_float, POINTER(c_float), c_void_p]
    lib.polfed_mlp_features.argtypes = [POINTER(CModel), c_double, POINTER(c_float)]
    lib.polfed_mlp_targets.argtypes = [c_int32, POINTER(c_double), POINTER(c_float)]
    lib.polfed_mlp_predict.argtypes = [c_void_p, POINTER(CModel), c_double, POINTER(c_double)]
    lib.polfed_cheb_filter_batched.argtypes = [c_int32, POINTER(CModel), POINTER(c_double), POINTER(c_double),
                                               POINTER(c_double), POINTER(c_int32), POINTER(c_void_p),
                                               POINTER(c_void_p), c_int32, c_int32, c_int32, c_void_p]
    lib.polfed_eigs_batched.argtypes = [c_int32, c_int32, POINTER(CModel), POINTER(c_double), POINTER(c_int32),
                                        POINTER(c_int32), c_int32, POINTER(COpts), c_int32, POINTER(c_double),
                                        POINTER(c_double), POINTER(c_void_p), POINTER(CStats), POINTER(c_int32),
                                        POINTER(CBatchInfo)]
    lib.polfed_set_wait_limit.argtypes = [ctypes.c_uint32]
    lib.polfed_gap_ratio.argtypes = [c_void_p, c_int32, POINTER(c_double), c_void_p, c_void_p]
    lib.polfed_entanglement_entropy.argtypes = [c_void_p, c_int32, c_void_p, c_void_p, c_int64, c_int32, c_int32,
                                                POINTER(c_double)]
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


def cheb_filter_cols(model, d_states, dim, e_lo, e_hi, coeffs, X, Y, n_b, stream=None):
    """polfed_cheb_filter_cols: FP32 filter, column j through its own series coeffs[j] (n_b x (K + 1))."""
    m = Model.of(model)
    coeffs = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    assert coeffs.ndim == 2 and coeffs.shape[0] == int(n_b)
    K = coeffs.shape[1] - 1
    return _check(load().polfed_cheb_filter_cols(byref(m.c), _ptr(d_states), int(dim), float(e_lo), float(e_hi),
                                                 int(K), coeffs.ctypes.data_as(POINTER(c_double)), _ptr(X), _ptr(Y),
                                                 int(n_b), _stream(stream)))


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

    def set_progress(self, fn):
        """polfed_ctx_set_progress: fn(phase, index) at every phase boundary (None removes it).
        The ctypes thunk is kept on the context so that it outlives the calls."""
        if fn is None:
            self._progress = None
            _check(self.lib.polfed_ctx_set_progress(self.h, PROGRESS_FN(), None))
            return
        self._progress = PROGRESS_FN(lambda user, phase, index: fn(int(phase), int(index)))
        _check(self.lib.polfed_ctx_set_progress(self.h, self._progress, None))


def history(ctx) -> list:
    """polfed_ctx_history: the convergence checks of the last call on ctx, as dicts."""
    n = c_int32(0)
    _check(load().polfed_ctx_history(ctx.h, None, 0, byref(n)))
    arr = (CConvPoint * max(1, n.value))()
    _check(load().polfed_ctx_history(ctx.h, arr, n.value, byref(n)))
    return [{f: getattr(arr[i], f) for f, _ in CConvPoint._fields_ if f != "reserved"} for i in range(n.value)]


def get_counters() -> dict:
    """polfed_get_counters: this thread's launch and step-kernel counters (monotone)."""
    c = CCounters()
    _check(load().polfed_get_counters(byref(c)))
    return c.as_dict()


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


def _dptr(a):
    return a.ctypes.data_as(POINTER(c_double))


def _fptr(a):
    return a.ctypes.data_as(POINTER(c_float))


def spectral_bounds(ctx, model):
    """polfed_spectral_bounds: (E_min, E_max, err)."""
    m = Model.of(model)
    out = np.zeros(3)
    _check(load().polfed_spectral_bounds(ctx.h, byref(m.c), _dptr(out)))
    return float(out[0]), float(out[1]), float(out[2])


def kpm_moments(model, d_states, dim, e_lo, e_hi, n_mom, R_block, R, dtype, stream=None):
    """polfed_kpm_moments: numpy array of n_mom moments."""
    m = Model.of(model)
    mu = np.zeros(int(n_mom))
    _check(load().polfed_kpm_moments(byref(m.c), _ptr(d_states), int(dim), float(e_lo), float(e_hi), int(n_mom),
                                     _ptr(R_block), int(R), int(dtype), _dptr(mu), _stream(stream)))
    return mu


def kpm_count(mu, x_a, x_b) -> float:
    mu = np.ascontiguousarray(np.asarray(mu, dtype=np.float64))
    f = c_double(0.0)
    _check(load().polfed_kpm_count(_dptr(mu), int(mu.size), float(x_a), float(x_b), byref(f)))
    return f.value


def spectral_labels(ctx, model, eps_target=0.5, n_mom=256, R=16):
    """polfed_spectral_labels: (E_min, E_max, rho_eps)."""
    m = Model.of(model)
    out = np.zeros(3)
    _check(load().polfed_spectral_labels(ctx.h, byref(m.c), float(eps_target), int(n_mom), int(R), _dptr(out)))
    return float(out[0]), float(out[1]), float(out[2])


def mlp_features(model, W):
    m = Model.of(model)
    x = np.zeros(m.c.L + 1, dtype=np.float32)
    _check(load().polfed_mlp_features(byref(m.c), float(W), _fptr(x)))
    return x


def mlp_targets(L, labels):
    lab = np.ascontiguousarray(np.asarray(labels, dtype=np.float64))
    y = np.zeros(3, dtype=np.float32)
    _check(load().polfed_mlp_targets(int(L), _dptr(lab), _fptr(y)))
    return y


class MLP:
    """polfed_mlp: the learned spectral predictor (device-resident FP32 network)."""

    def __init__(self, d_in, hidden=128, d_out=3, seed=0):
        self.lib = load()
        h = c_void_p()
        _check(self.lib.polfed_mlp_create(int(d_in), int(hidden), int(d_out), int(seed), byref(h)))
        self.h = h
        self.d_in, self.hidden, self.d_out = int(d_in), int(hidden), int(d_out)

    def close(self):
        if self.h:
            self.lib.polfed_mlp_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self) -> int:
        return int(self.lib.polfed_mlp_num_params(self.h))

    def get_params(self):
        p = np.zeros(self.num_params, dtype=np.float32)
        _check(self.lib.polfed_mlp_get_params(self.h, _fptr(p)))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        assert p.size == self.num_params
        _check(self.lib.polfed_mlp_set_params(self.h, _fptr(p)))

    def set_scaling(self, x_mean, x_std, y_mean, y_std):
        a = [np.ascontiguousarray(np.asarray(v, dtype=np.float32)) for v in (x_mean, x_std, y_mean, y_std)]
        _check(self.lib.polfed_mlp_set_scaling(self.h, *[_fptr(v) for v in a]))

    def forward(self, d_x, B, d_y, stream=None):
        _check(self.lib.polfed_mlp_forward(self.h, _ptr(d_x), int(B), _ptr(d_y), _stream(stream)))

    def grad(self, d_x, d_t, B, d_grad=None, stream=None) -> float:
        loss = c_float(0.0)
        _check(self.lib.polfed_mlp_grad(self.h, _ptr(d_x), _ptr(d_t), int(B), _ptr(d_grad), byref(loss),
                                        _stream(stream)))
        return loss.value

    def train_step(self, d_x, d_t, B, lr, stream=None) -> float:
        loss = c_float(0.0)
        _check(self.lib.polfed_mlp_train_step(self.h, _ptr(d_x), _ptr(d_t), int(B), float(lr), byref(loss),
                                              _stream(stream)))
        return loss.value

    def predict(self, model, W):
        """(E_min, E_max, rho_eps) for one realization."""
        m = Model.of(model)
        out = np.zeros(3)
        _check(self.lib.polfed_mlp_predict(self.h, byref(m.c), float(W), _dptr(out)))
        return float(out[0]), float(out[1]), float(out[2])


def _models_array(models):
    ms = [Model.of(m) for m in models]
    arr = (CModel * len(ms))(*[m.c for m in ms])
    return ms, arr


def cheb_filter_batched(models, e_lo, e_hi, sigma, K, Xs, Ys, n_b, dtype, ctas_per_sm=0, stream=None):
    """polfed_cheb_filter_batched: all realizations' filters in one cooperative launch."""
    n = len(models)
    keep, arr = _models_array(models)
    lo = np.ascontiguousarray(e_lo, dtype=np.float64)
    hi = np.ascontiguousarray(e_hi, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    kk = np.ascontiguousarray(K, dtype=np.int32)
    xp = (c_void_p * n)(*[_ptr(x) for x in Xs])
    yp = (c_void_p * n)(*[_ptr(y) for y in Ys])
    return _check(load().polfed_cheb_filter_batched(n, arr, _dptr(lo), _dptr(hi), _dptr(sg),
                                                    kk.ctypes.data_as(POINTER(c_int32)), xp, yp, int(n_b),
                                                    int(dtype), int(ctas_per_sm), _stream(stream)))


def eigs_batched(models, eps_target, N_ev, K=None, n_b=0, opts=None, max_workers=0, d_evecs=None, device=0,
                 allow_fail=False):
    """polfed_eigs_batched: returns (list of evals, list of resid, list of stats dicts, statuses, info dict, rc)."""
    n = len(models)
    keep, arr = _models_array(models)
    eps = np.ascontiguousarray(np.broadcast_to(np.asarray(eps_target, dtype=np.float64), (n,)))
    nev = np.ascontiguousarray(np.broadcast_to(np.asarray(N_ev, dtype=np.int32), (n,)))
    kk = None if K is None else np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.int32), (n,)))
    tot = int(nev.sum())
    ev = np.zeros(tot)
    rs = np.zeros(tot)
    st = (CStats * n)()
    status = np.zeros(n, dtype=np.int32)
    info = CBatchInfo()
    o = opts if opts is not None else opts_default()
    vp = None if d_evecs is None else (c_void_p * n)(*[_ptr(v) for v in d_evecs])
    rc = load().polfed_eigs_batched(int(device), n, arr, _dptr(eps), nev.ctypes.data_as(POINTER(c_int32)),
                                    None if kk is None else kk.ctypes.data_as(POINTER(c_int32)), int(n_b), byref(o),
                                    int(max_workers), _dptr(ev), _dptr(rs), vp, st,
                                    status.ctypes.data_as(POINTER(c_int32)), byref(info))
    if not allow_fail:
        _check(rc)
    offs = np.concatenate([[0], np.cumsum(nev)])
    evs = [ev[offs[i]:offs[i + 1]] for i in range(n)]
    res = [rs[offs[i]:offs[i + 1]] for i in range(n)]
    return evs, res, [s.as_dict() for s in st], status, info.as_dict(), rc


def gap_ratio(d_evals, n, d_r=None, stream=None) -> float:
    """polfed_gap_ratio: mean gap ratio of n ascending eigenvalues on the device."""
    r = c_double(0.0)
    _check(load().polfed_gap_ratio(_ptr(d_evals), int(n), byref(r), _ptr(d_r), _stream(stream)))
    return r.value


def entanglement_entropy(ctx, L, d_states, d_vecs, ld, n_vec, per_cut=False):
    """polfed_entanglement_entropy: numpy array of n_vec cut-averaged entropies, or
    n_vec x L per-cut entropies with per_cut."""
    out = np.zeros(int(n_vec) * (int(L) if per_cut else 1))
    _check(load().polfed_entanglement_entropy(ctx.h, int(L), _ptr(d_states), _ptr(d_vecs), int(ld), int(n_vec),
                                              1 if per_cut else 0, _dptr(out)))
    return out.reshape(int(n_vec), int(L)) if per_cut else out


def set_wait_limit(polls: int):
    """polfed_set_wait_limit: cap every bounded device wait at `polls` iterations (0 = defaults); tests only."""
    _check(load().polfed_set_wait_limit(int(polls)))
