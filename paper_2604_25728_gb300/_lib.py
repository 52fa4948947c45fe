"""ctypes declarations of the C ABI in include/sqngd.h.

Loading fails loudly when libsqngd.so is missing or cannot be built: there is
no CPU or PyTorch fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_int32, c_int64, c_double, c_float = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_float
c_void_p = ctypes.c_void_p
P_double = ctypes.POINTER(c_double)
P_float = ctypes.POINTER(c_float)

AF_OK, AF_ERR_INVALID_ARG, AF_ERR_CUDA, AF_ERR_NONFINITE, AF_ERR_TIMEOUT, AF_ERR_OOM, AF_ERR_UNIMPLEMENTED = range(7)
STATUS_NAMES = ["AF_OK", "AF_ERR_INVALID_ARG", "AF_ERR_CUDA", "AF_ERR_NONFINITE", "AF_ERR_TIMEOUT",
                "AF_ERR_OOM", "AF_ERR_UNIMPLEMENTED"]
AF_PATH_AUTO, AF_PATH_FFT, AF_PATH_DFT, AF_PATH_SPLIT_BF16 = range(4)
AF_TERMS_FIXED = 8


class AfConfig(ctypes.Structure):
    _fields_ = [
        ("M", c_int32), ("N", c_int32), ("B", c_int32), ("L", c_int32),
        ("nu", P_double),
        ("k_lo", c_int32), ("k_hi", c_int32),
        ("weights", P_float),
        ("eps", c_double), ("snrl_db", c_double),
        ("r_n", c_int32), ("c", c_double),
        ("pnorm", c_double),
        ("path", c_int32),
        ("n_h", c_int32), ("n_x", c_int32),
        ("lr_h", c_double), ("lr_x", c_double),
        ("beta1", c_double), ("beta2", c_double), ("adam_eps", c_double),
        ("matched", c_int32),
        ("train_rho", c_int32), ("lr_rho", c_double),
    ]


class AfState(ctypes.Structure):
    _fields_ = [
        ("u_dev", c_void_p), ("h_dev", c_void_p),
        ("m_u_dev", c_void_p), ("v_u_dev", c_void_p),
        ("m_h_dev", c_void_p), ("v_h_dev", c_void_p),
        ("best_q_dev", c_void_p), ("best_h_dev", c_void_p),
        ("best_dev", c_void_p),
        ("t_h", c_int64), ("t_x", c_int64), ("outer", c_int64),
    ]


class AfStop(ctypes.Structure):
    _fields_ = [("best_wpsl", c_double), ("best_outer", c_int64), ("stopped", c_int32)]


class WsConfig(ctypes.Structure):
    _fields_ = [("M", c_int32), ("N", c_int32), ("B", c_int32), ("cond", c_double * 5)]


# name -> (restype, argtypes); every symbol include/sqngd.h and include/warmstart.h declare
SIGNATURES = {
    "af_init": (c_int32, [ctypes.POINTER(AfConfig), c_void_p, ctypes.POINTER(c_void_p)]),
    "af_destroy": (c_int32, [c_void_p]),
    "af_last_error": (ctypes.c_char_p, [c_void_p]),
    "af_path_of": (c_int32, [c_void_p]),
    "af_sync": (c_int32, [c_void_p]),
    "af_set_thresholds": (c_int32, [c_void_p, P_float]),
    "af_ambiguity": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "af_forward": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "af_loss_grad_xh": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "af_loss_grad": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "quantize": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "soft_quantize": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "af_project": (c_int32, [c_void_p, c_void_p]),
    "af_loss_grad_rho": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "af_get_thresholds": (c_int32, [c_void_p, P_float]),
    "af_project_thresholds": (c_int32, [c_void_p, c_void_p]),
    "sqngd_init": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sqngd_step": (c_int32, [c_void_p, ctypes.POINTER(AfState), c_int32, P_double]),
    "sqngd_run": (c_int32, [c_void_p, ctypes.POINTER(AfState), c_int64, c_int32, ctypes.POINTER(AfStop),
                            P_double, ctypes.POINTER(c_int64)]),
    "af_get_rho_state": (c_int32, [c_void_p, P_float, P_float, P_float, ctypes.POINTER(c_int32)]),
    "af_set_rho_state": (c_int32, [c_void_p, P_float, P_float, P_float, c_int32]),
    "af_eval_hard": (c_int32, [c_void_p, c_void_p, c_void_p, P_double]),
    "af_loss_terms_noalloc": (c_int32, [c_int32, c_int32, c_int32, c_double, c_int32, c_int32, c_double, c_double,
                                        c_void_p, c_void_p, c_void_p, c_void_p]),
    "rn_param_count": (c_int64, [c_int32]),
    "rn_create": (c_int32, [c_int32, c_void_p, ctypes.POINTER(c_void_p)]),
    "rn_destroy": (c_int32, [c_void_p]),
    "rn_last_error": (ctypes.c_char_p, [c_void_p]),
    "rn_set_params": (c_int32, [c_void_p, P_float]),
    "rn_get_params": (c_int32, [c_void_p, P_float]),
    "rn_set_adam": (c_int32, [c_void_p, P_float, P_float]),
    "rn_get_adam": (c_int32, [c_void_p, P_float, P_float]),
    "rn_forward": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "rn_train_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_float, c_int64, c_void_p]),
    "sqngd_attach_generator": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "ws_param_count": (c_int64, []),
    "ws_create": (c_int32, [c_int32, c_int32, c_void_p, ctypes.POINTER(c_void_p)]),
    "ws_destroy": (c_int32, [c_void_p]),
    "ws_last_error": (ctypes.c_char_p, [c_void_p]),
    "ws_set_params": (c_int32, [c_void_p, P_float]),
    "ws_get_params": (c_int32, [c_void_p, P_float]),
    "ws_forward": (c_int32, [c_void_p, ctypes.POINTER(WsConfig), c_int32, c_void_p, c_void_p, c_void_p]),
    "ws_loss_grad": (c_int32, [c_void_p, ctypes.POINTER(WsConfig), c_int32, c_void_p, c_void_p, P_double,
                               P_float]),
    "ws_train_step": (c_int32, [c_void_p, ctypes.POINTER(WsConfig), c_int32, c_void_p, c_void_p, c_float,
                                P_double]),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load libsqngd.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_needed:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"{_build.LIB} is missing: build the sm_103a library first")
            lib = ctypes.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class AfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


def check(status: int, ctx_handle=None):
    if status != AF_OK:
        msg = load().af_last_error(ctx_handle)
        raise AfError(status, msg.decode() if msg else "")
