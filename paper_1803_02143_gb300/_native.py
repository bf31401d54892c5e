"""ctypes binding of libsldg (``include/sldg.h``): argument marshalling only.

Every function here has the name of the C entry point it wraps and raises
``SldgError`` on a non-zero status.  No arithmetic of the method happens in
Python: every step runs in the CUDA kernels of ``libsldg.so``.  If the
library is missing the import fails loudly; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libsldg.so")

SLDG_OK = 0
SLDG_ERR_BAD_CONFIG = -1
SLDG_ERR_BAD_PTR = -2
SLDG_ERR_OOM = -3
SLDG_ERR_CUDA = -4
SLDG_ERR_NONFINITE = -5
SLDG_ERR_UNSUPPORTED = -6
SLDG_ERR_STATE = -7
SLDG_ERR_ARG = -8

SLDG_FP64 = 0
SLDG_FP32 = 1
SLDG_FLAG_NATIVE_FP64 = 1
SLDG_FLAG_NO_XFUSION = 2
SLDG_FLAG_ORDER4 = 4
SLDG_FLAG_MERGE_DRIFTS = 8
SLDG_FLAG_SPLINE = 16
SLDG_VBC_ZERO_INFLOW = 0
SLDG_VBC_PERIODIC = 1
SLDG_INIT_LANDAU = 0
SLDG_INIT_TWO_STREAM = 1
SLDG_INIT_TWO_STREAM_PAPER = 2

KIND_NAMES = ("x1", "x2", "v1", "v2", "rho", "poisson", "vmat", "other", "adj_x", "adj_v", "x12")
SLDG_NUM_KINDS = len(KIND_NAMES)


class sldg_config(ctypes.Structure):
    _fields_ = [
        ("degree", ctypes.c_int),
        ("ncell", ctypes.c_int * 4),
        ("lo", ctypes.c_double * 4),
        ("hi", ctypes.c_double * 4),
        ("dt", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("vbc", ctypes.c_int),
        ("poisson_kmax", ctypes.c_int),
        ("flags", ctypes.c_int),
    ]


class sldg_diag(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double),
        ("step", ctypes.c_longlong),
        ("mass", ctypes.c_double),
        ("l1", ctypes.c_double),
        ("l2sq", ctypes.c_double),
        ("kinetic", ctypes.c_double),
        ("electric", ctypes.c_double),
        ("total", ctypes.c_double),
    ]


class SldgError(RuntimeError):
    def __init__(self, fn, code):
        self.code = code
        super().__init__(f"{fn}: {sldg_strerror(code)} ({code})")


_lib = None
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_LLP = ctypes.POINTER(ctypes.c_longlong)

# name -> (restype, argtypes); the full C ABI of include/sldg.h
SIGNATURES = {
    "sldg_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sldg_abi_version": (ctypes.c_int, []),
    "sldg_init": (ctypes.c_int, [ctypes.POINTER(sldg_config), _VP, _VP, ctypes.POINTER(_VP)]),
    "sldg_destroy": (None, [_VP]),
    "sldg_numel": (ctypes.c_longlong, [_VP]),
    "sldg_bind": (ctypes.c_int, [_VP, _VP]),
    "sldg_set_initial": (ctypes.c_int, [_VP, ctypes.c_int, _DP, ctypes.c_int]),
    "sldg_get_f": (ctypes.c_int, [_VP, _VP, ctypes.c_int]),
    "sldg_set_f": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_double, ctypes.c_longlong]),
    "sldg_step": (ctypes.c_int, [_VP, ctypes.c_int, _DP]),
    "sldg_step_host_batches": (ctypes.c_int, [_VP, _VP, ctypes.c_longlong, ctypes.c_int, _DP]),
    "sldg_sweep": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_double]),
    "sldg_drift": (ctypes.c_int, [_VP, ctypes.c_double]),
    "sldg_compute_fields": (ctypes.c_int, [_VP]),
    "sldg_set_field": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int]),
    "sldg_fields": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int]),
    "sldg_diagnostics": (ctypes.c_int, [_VP, ctypes.POINTER(sldg_diag)]),
    "sldg_sweep_adjoint": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_double, _VP, _VP, _VP]),
    "sldg_record": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _DP]),
    "sldg_objective": (ctypes.c_int, [_VP, _DP, ctypes.c_int, _DP]),
    "sldg_backward": (ctypes.c_int, [_VP, _DP, ctypes.c_int, _VP, _DP]),
    "sldg_set_slot_limit": (ctypes.c_int, [_VP, ctypes.c_int]),
    "sldg_backward_stats": (ctypes.c_int, [_VP, _LLP, ctypes.POINTER(ctypes.c_int)]),
    "sldg_initial_param_grad": (ctypes.c_int, [_VP, ctypes.c_int, _DP, ctypes.c_int, _VP, _DP]),
    "sldg_rho_noalloc": (ctypes.c_int, [ctypes.POINTER(sldg_config), _VP, _VP, _VP]),
    "sldg_launch_count": (ctypes.c_longlong, [_VP]),
    "sldg_x_pass_shape": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "sldg_timing": (ctypes.c_int, [_VP, ctypes.c_int]),
    "sldg_timing_read": (ctypes.c_int, [_VP, _DP, _LLP]),
}


def load(path: str = LIBPATH):
    """Load libsldg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_1803_02143_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(fn, rc):
    if rc != SLDG_OK:
        raise SldgError(fn, rc)


def _dptr(a):
    """ctypes double* for a host float64 numpy array or None."""
    if a is None:
        return None
    return a.ctypes.data_as(_DP)


def sldg_strerror(code: int) -> str:
    return load().sldg_strerror(code).decode()


def sldg_abi_version() -> int:
    return load().sldg_abi_version()


def sldg_init(cfg: sldg_config, f_ptr: int, stream_ptr: int):
    out = _VP()
    _check("sldg_init", load().sldg_init(ctypes.byref(cfg), _VP(f_ptr), _VP(stream_ptr),
                                         ctypes.byref(out)))
    return out


def sldg_destroy(ctx) -> None:
    load().sldg_destroy(ctx)


def sldg_numel(ctx) -> int:
    return load().sldg_numel(ctx)


def sldg_bind(ctx, f_ptr: int) -> None:
    _check("sldg_bind", load().sldg_bind(ctx, _VP(f_ptr)))


def sldg_set_initial(ctx, kind: int, params) -> None:
    import numpy as np

    p = np.ascontiguousarray(params, dtype=np.float64)
    _check("sldg_set_initial", load().sldg_set_initial(ctx, int(kind), _dptr(p), int(p.size)))


def sldg_get_f(ctx, dst_ptr: int, on_device: bool) -> None:
    _check("sldg_get_f", load().sldg_get_f(ctx, _VP(dst_ptr), int(on_device)))


def sldg_set_f(ctx, src_ptr: int, on_device: bool, t: float = 0.0, step: int = 0) -> None:
    _check("sldg_set_f", load().sldg_set_f(ctx, _VP(src_ptr), int(on_device), float(t), int(step)))


def sldg_step(ctx, nsteps: int, W_history=None) -> None:
    _check("sldg_step", load().sldg_step(ctx, int(nsteps), _dptr(W_history)))


def sldg_sweep(ctx, dim: int, frac: float) -> None:
    _check("sldg_sweep", load().sldg_sweep(ctx, int(dim), float(frac)))


def sldg_drift(ctx, frac: float) -> None:
    _check("sldg_drift", load().sldg_drift(ctx, float(frac)))


def sldg_compute_fields(ctx) -> None:
    _check("sldg_compute_fields", load().sldg_compute_fields(ctx))


def sldg_set_field(ctx, E1_ptr: int, E2_ptr: int, on_device: bool) -> None:
    _check("sldg_set_field", load().sldg_set_field(ctx, _VP(E1_ptr), _VP(E2_ptr), int(on_device)))


def sldg_fields(ctx, rho_ptr, E1_ptr, E2_ptr, on_device: bool) -> None:
    _check("sldg_fields", load().sldg_fields(ctx, _VP(rho_ptr), _VP(E1_ptr), _VP(E2_ptr),
                                             int(on_device)))


def sldg_diagnostics(ctx) -> sldg_diag:
    d = sldg_diag()
    _check("sldg_diagnostics", load().sldg_diagnostics(ctx, ctypes.byref(d)))
    return d


def sldg_sweep_adjoint(ctx, dim: int, frac: float, lam_ptr: int, g_ptr=None, Ebar_ptr=None) -> None:
    _check("sldg_sweep_adjoint", load().sldg_sweep_adjoint(ctx, int(dim), float(frac), _VP(lam_ptr),
                                                           _VP(g_ptr), _VP(Ebar_ptr)))


def sldg_step_host_batches(ctx, host_ptr: int, stride_bytes: int, nbatch: int, W_out) -> None:
    _check("sldg_step_host_batches",
           load().sldg_step_host_batches(ctx, _VP(host_ptr), int(stride_bytes), int(nbatch),
                                         _dptr(W_out)))


def sldg_record(ctx, nsteps: int, ckpt_every: int, W_history=None) -> None:
    _check("sldg_record", load().sldg_record(ctx, int(nsteps), int(ckpt_every), _dptr(W_history)))


def sldg_objective(ctx, cW=None) -> float:
    J = ctypes.c_double(0.0)
    n = 0 if cW is None else int(cW.size)
    _check("sldg_objective", load().sldg_objective(ctx, _dptr(cW), n, ctypes.byref(J)))
    return J.value


def sldg_backward(ctx, cW, grad_ptr: int) -> float:
    J = ctypes.c_double(0.0)
    n = 0 if cW is None else int(cW.size)
    _check("sldg_backward", load().sldg_backward(ctx, _dptr(cW), n, _VP(grad_ptr), ctypes.byref(J)))
    return J.value


def sldg_set_slot_limit(ctx, max_slots: int) -> None:
    _check("sldg_set_slot_limit", load().sldg_set_slot_limit(ctx, int(max_slots)))


def sldg_backward_stats(ctx):
    n = ctypes.c_longlong(0)
    k = ctypes.c_int(0)
    _check("sldg_backward_stats", load().sldg_backward_stats(ctx, ctypes.byref(n), ctypes.byref(k)))
    return n.value, k.value


def sldg_initial_param_grad(ctx, kind: int, params, grad_ptr: int) -> float:
    import numpy as np

    p = np.ascontiguousarray(params, dtype=np.float64)
    out = ctypes.c_double(0.0)
    _check("sldg_initial_param_grad",
           load().sldg_initial_param_grad(ctx, int(kind), _dptr(p), int(p.size), _VP(grad_ptr),
                                          ctypes.byref(out)))
    return out.value


def sldg_rho_noalloc(cfg: sldg_config, f_ptr: int, rho_ptr: int, stream_ptr: int) -> None:
    _check("sldg_rho_noalloc", load().sldg_rho_noalloc(ctypes.byref(cfg), _VP(f_ptr), _VP(rho_ptr),
                                                       _VP(stream_ptr)))


def sldg_launch_count(ctx) -> int:
    return load().sldg_launch_count(ctx)


def sldg_x_pass_shape(ctx):
    cs = ctypes.c_int(0)
    lanes = ctypes.c_int(0)
    _check("sldg_x_pass_shape", load().sldg_x_pass_shape(ctx, ctypes.byref(cs), ctypes.byref(lanes)))
    return cs.value, lanes.value


def sldg_timing(ctx, enable: bool) -> None:
    _check("sldg_timing", load().sldg_timing(ctx, int(enable)))


def sldg_timing_read(ctx):
    ms = (ctypes.c_double * SLDG_NUM_KINDS)()
    cnt = (ctypes.c_longlong * SLDG_NUM_KINDS)()
    _check("sldg_timing_read", load().sldg_timing_read(ctx, ms, cnt))
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KIND_NAMES)}
