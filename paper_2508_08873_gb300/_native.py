"""ctypes binding of liblrp.so (include/lrp.h): argument marshalling only.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA); they
must be float64 and C-contiguous.  Every computation runs in the CUDA library;
if the library cannot be loaded this module raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

LRP_OK, LRP_EINVAL, LRP_ENOMEM, LRP_ENOTCONV, LRP_EBREAKDOWN, LRP_ETIMEOUT, LRP_ECUDA, LRP_EBUSY = range(8)
PREC_F64, PREC_MIXED = 0, 1

_lib = None
_lock = threading.Lock()
_exiting = False


def _mark_exit():
    global _exiting
    _exiting = True


import atexit  # noqa: E402
atexit.register(_mark_exit)


def exiting() -> bool:
    """True once the interpreter shuts down: handles are then left to the
    process exit instead of being freed through a half-finalised runtime."""
    return _exiting


class LrpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("lrp status %d (%s): %s" % (status, _status_string(status), msg))
        self.status = status


class SolveStats(ctypes.Structure):
    _fields_ = [("k_done", ctypes.c_int), ("fine_evals", ctypes.c_int),
                ("converged", ctypes.c_int), ("final_bound", ctypes.c_double),
                ("scale", ctypes.c_double), ("device_ms", ctypes.c_double)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("k_done", ctypes.c_int), ("status", ctypes.c_int),
                ("final_bound", ctypes.c_double), ("scale", ctypes.c_double),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_ulonglong), ("ticks", ctypes.c_ulonglong),
                ("queued", ctypes.c_size_t), ("active", ctypes.c_int), ("slots", ctypes.c_int),
                ("error", ctypes.c_int), ("busy_ms", ctypes.c_double)]


LRP_PENDING = 8
LRP_BUILD_INDEPENDENT_ADJOINT = 1   # flags of lrp_build_coarse_ex
STEPPERS = {"be": 0, "sdirk2": 1, "sdirk2l": 2}   # lrp_stepper

# (name, restype, argtypes)
_P, _I, _D, _S, _U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_uint64
_PP = ctypes.POINTER(ctypes.c_void_p)
_PI = ctypes.POINTER(ctypes.c_int)
_PD = ctypes.POINTER(ctypes.c_double)
SIGNATURES = [
    ("lrp_create", _I, [_PP, _I, _S]),
    ("lrp_destroy", None, [_P]),
    ("lrp_set_stream", _I, [_P, _P]),
    ("lrp_get_stream", _P, [_P]),
    ("lrp_synchronize", _I, [_P]),
    ("lrp_status_string", ctypes.c_char_p, [_I]),
    ("lrp_last_error", ctypes.c_char_p, [_P]),
    ("lrp_bytes_in_use", _S, [_P]),
    ("lrp_launch_count", ctypes.c_long, [_P]),
    ("lrp_set_param", _I, [_P, ctypes.c_char_p, _I]),
    ("lrp_get_param", _I, [_P, ctypes.c_char_p, _PI]),
    ("lrp_set_kernel_timing", _I, [_P, _I]),
    ("lrp_kernel_time", _I, [_P, ctypes.c_char_p, _PI, _PD]),
    ("lrp_reset_kernel_time", _I, [_P]),
    ("lrp_operator_tridiag", _I, [_P, _I, _P, _P, _P, _PP]),
    ("lrp_operator_tridiag_td", _I, [_P, _I, _I, _P, _P, _P, _PP]),
    ("lrp_operator_stencil5", _I, [_P, _I, _I, _P, _P, _P, _P, _P, _PP]),
    ("lrp_operator_stencil5_td", _I, [_P, _I, _I, _I, _P, _P, _P, _P, _P, _PP]),
    ("lrp_operator_tridiag_td_sdirk", _I, [_P, _I, _I, _I, _P, _P, _P, _PP]),
    ("lrp_operator_stencil5_td_sdirk", _I, [_P, _I, _I, _I, _I, _P, _P, _P, _P, _P, _PP]),
    ("lrp_operator_free", None, [_P]),
    ("lrp_operator_size", _I, [_P]),
    ("lrp_operator_krylov_iterations", ctypes.c_ulonglong, [_P]),
    ("lrp_operator_set_krylov", _I, [_P, _D, _D, _I]),
    ("lrp_propagate", _I, [_P, _P, _D, _I, _I, _I, _P, _P, _I, _P, _P, _I]),
    ("lrp_propagate_noalloc", _I, [_I, _P, _I, _P, _P, _P, _D, _I, _I, _I, _P, _P, _I, _P, _P, _I]),
    ("lrp_gaussian", _I, [_P, _U64, _I, _I, _I, _I, _P]),
    ("lrp_build_coarse", _I, [_P, _P, _D, _I, _I, _I, _I, _U64, _I, _PP]),
    ("lrp_build_coarse_ex", _I, [_P, _P, _D, _I, _I, _I, _I, _U64, _I, _I, _PP]),
    ("lrp_coarse_free", None, [_P]),
    ("lrp_coarse_info", _I, [_P, _P, _P, _P, _P, _P, _P]),
    ("lrp_coarse_orth_method", _I, [_P, _P, _P]),
    ("lrp_coarse_factors", _I, [_P, _I, _P, _P, _P]),
    ("lrp_coarse_export", _I, [_P, _P, _P, ctypes.POINTER(ctypes.c_uint64), _P, _P, _P, _P, _P, _P, _P]),
    ("lrp_coarse_import", _I, [_P, _P, _P, _P, _U64, _P, _P, _P, _P, _P, _P, _P, _PP]),
    ("lrp_parareal_solve", _I, [_P, _P, _P, _I, _P, _P, _I, _D, _P, _P, _PI,
                                ctypes.POINTER(SolveStats)]),
    ("lrp_fine_solution", _I, [_P, _P, _D, _I, _I, _P, _I, _P, _P, _P]),
    ("lrp_operator_set_stepper", _I, [_P, _I]),
    ("lrp_parareal_solve_classical", _I, [_P, _P, _D, _I, _I, _P, _I, _P, _P, _I, _D, _P, _P, _PI,
                                          ctypes.POINTER(SolveStats)]),
    ("lrp_build_coarse_batch", _I, [_P, _I, _P, _D, _I, _I, _I, _I, _U64, _I, _P]),
    ("lrp_parareal_solve_batch", _I, [_P, _I, _P, _P, _I, _D, _P, _P]),
    ("lrp_server_create", _I, [_P, _I, _I, _S, _PP]),
    ("lrp_server_destroy", None, [_P]),
    ("lrp_server_submit", _I, [_P, _P, _P, _I, _P, _P, _I, _D, ctypes.POINTER(ctypes.c_uint64)]),
    ("lrp_server_poll", _I, [_P, ctypes.c_uint64, _P, ctypes.POINTER(RequestInfo)]),
    ("lrp_server_wait", _I, [_P, ctypes.c_uint64, _D, _P, ctypes.POINTER(RequestInfo)]),
    ("lrp_server_stats_get", _I, [_P, ctypes.POINTER(ServerStats)]),
    ("lrp_server_set_latency_target", _I, [_P, _P, ctypes.c_double]),
    ("lrp_server_estimate", _I, [_P, _P, ctypes.POINTER(ctypes.c_double)]),
]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblrp.so (building it with nvcc when missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("liblrp.so is not built; run paper_2508_08873_gb300/build.py")
            L = ctypes.CDLL(_build.LIB)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _status_string(s: int) -> str:
    try:
        return load(False).lrp_status_string(s).decode()
    except Exception:
        return "?"


def ptr(a) -> Optional[int]:
    """Raw address of a float64 C-contiguous numpy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous float64 numpy array")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 torch tensor")
        return a.data_ptr()
    raise TypeError("unsupported array type %r" % type(a))


def check(status: int, ctx=None, ok=(LRP_OK,)):
    if status not in ok:
        msg = ""
        if ctx is not None:
            msg = (load(False).lrp_last_error(ctx) or b"").decode()
        raise LrpError(status, msg)
    return status
