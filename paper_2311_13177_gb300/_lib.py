"""ctypes view of libprop.so (declarations mirror include/prop.h).

Loading fails loudly when the library has not been built: there is no
fallback implementation of any step.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB

c_int, c_float, c_double, c_void_p, c_size_t = (ctypes.c_int, ctypes.c_float, ctypes.c_double,
                                                ctypes.c_void_p, ctypes.c_size_t)

PROP_OK = 0
PROP_NUM_STAGES = 12
STAGE_NAMES = ["fft_fwd_rows", "fft_fwd_cols", "interp", "spread", "fft_adj_cols", "fft_adj_rows",
               "tv_adam", "other", "rows_update", "kplanes_render", "kplanes_vjp", "kplanes_adam"]
STATUS_NAMES = {0: "PROP_OK", 1: "PROP_ERR_INVALID_ARG", 2: "PROP_ERR_OOM", 3: "PROP_ERR_CUDA",
                4: "PROP_ERR_TIMEOUT", 5: "PROP_ERR_BUSY", 6: "PROP_ERR_NOT_READY",
                7: "PROP_ERR_CANCELLED", 8: "PROP_ERR_UNIMPLEMENTED"}


class PlanDesc(ctypes.Structure):
    _fields_ = [("n", c_int), ("nf", c_int), ("delta", ctypes.POINTER(c_double)),
                ("nblades", c_int), ("theta", ctypes.POINTER(c_double)), ("lines", c_int),
                ("readout", c_int), ("nframes", c_int), ("blade_frame", ctypes.POINTER(c_int)),
                ("kb_width", c_int), ("bin_chunk", c_int), ("row_kernel", c_int),
                ("device", c_int)]


class ReconParamsC(ctypes.Structure):
    _fields_ = [("iters", c_int), ("lr", c_float), ("beta1", c_float), ("beta2", c_float),
                ("eps", c_float), ("tv_xy", c_float), ("tv_t", c_float), ("tv_eps", c_float)]


class ProjParamsC(ctypes.Structure):
    _fields_ = [("iters", c_int), ("lr", c_float), ("beta1", c_float), ("beta2", c_float), ("eps", c_float),
                ("w_kspace", c_float), ("w_image", c_float), ("tv_xy", c_float), ("tv_f", c_float),
                ("tv_t", c_float), ("l1", c_float), ("tv_eps", c_float)]


# name -> (restype, argtypes); every symbol include/prop.h declares.
SIGNATURES = {
    "prop_plan_create": (c_int, [ctypes.POINTER(PlanDesc), ctypes.POINTER(c_void_p)]),
    "prop_plan_destroy": (c_int, [c_void_p]),
    "prop_plan_workspace_bytes": (c_int, [c_void_p, ctypes.POINTER(c_size_t)]),
    "prop_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "prop_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "prop_reconstruct": (c_int, [c_void_p, c_void_p, ctypes.POINTER(ReconParamsC), c_void_p,
                                 ctypes.POINTER(c_double), c_void_p]),
    "prop_reconstruct_batch": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(c_void_p),
                                       ctypes.POINTER(ReconParamsC), ctypes.POINTER(c_void_p),
                                       ctypes.POINTER(ctypes.POINTER(c_double)), c_void_p]),
    "prop_recon_step": (c_int, [c_void_p, c_void_p, ctypes.POINTER(ReconParamsC), c_int, c_void_p, c_void_p,
                                c_void_p, c_void_p]),
    "prop_shard_forward": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "prop_shard_update": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(ReconParamsC), c_int, c_void_p,
                                  c_void_p, c_void_p, c_void_p]),
    "prop_reconstruct_host": (c_int, [c_void_p, c_void_p, ctypes.POINTER(ReconParamsC), c_void_p,
                                      ctypes.POINTER(c_double), c_void_p]),
    "prop_loss_grad": (c_int, [c_void_p, c_void_p, ctypes.POINTER(ReconParamsC), c_void_p, c_void_p,
                               ctypes.POINTER(c_double), c_void_p]),
    "prop_render": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "prop_psnr": (c_int, [c_void_p, c_void_p, c_void_p, c_int, ctypes.POINTER(c_double), c_void_p]),
    "prop_plan_estimate_bytes": (c_int, [ctypes.POINTER(PlanDesc), c_int, ctypes.POINTER(c_size_t)]),
    "prop_serve_create": (c_int, [c_size_t, c_int, c_int, ctypes.POINTER(c_void_p)]),
    "prop_serve_submit": (c_int, [c_void_p, ctypes.POINTER(PlanDesc), ctypes.POINTER(ReconParamsC), c_void_p,
                                  c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "prop_serve_poll": (c_int, [c_void_p, ctypes.c_uint64, ctypes.POINTER(c_int)]),
    "prop_serve_wait": (c_int, [c_void_p, ctypes.c_uint64, c_int, c_void_p, ctypes.POINTER(c_double),
                                ctypes.POINTER(c_double)]),
    "prop_serve_cancel": (c_int, [c_void_p, ctypes.c_uint64]),
    "prop_serve_stats": (c_int, [c_void_p, c_void_p]),
    "prop_serve_destroy": (c_int, [c_void_p]),
    "prop_tv_grad_static": (c_int, [c_void_p, c_int, c_int, c_int, c_float, c_float, c_float, c_void_p,
                                    c_void_p, c_void_p]),
    "prop_profile_enable": (c_int, [c_void_p, c_int]),
    "prop_profile_read": (c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "prop_fp32_fma_peak": (c_int, [c_int, ctypes.POINTER(c_double)]),
    "prop_proj_forward": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "prop_proj_adjoint": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "prop_proj_reconstruct": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(ProjParamsC), c_void_p,
                                      ctypes.POINTER(c_double), c_void_p]),
    "prop_proj_baseline": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "prop_kplanes_param_count": (c_int, [c_void_p, c_int, c_int, ctypes.POINTER(c_size_t)]),
    "prop_kplanes_render": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "prop_kplanes_vjp": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "prop_kplanes_reconstruct": (c_int, [c_void_p, c_void_p, ctypes.POINTER(ReconParamsC), c_int, c_int, c_void_p,
                                         ctypes.POINTER(c_double), c_void_p]),
    "prop_check_bounded_wait": (c_int, [c_int, ctypes.c_longlong, ctypes.POINTER(c_int), ctypes.POINTER(c_double)]),
    "prop_last_error": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


class PropError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def lib() -> ctypes.CDLL:
    """The loaded libprop.so (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(f"{LIB} is not built; run paper_2311_13177_gb300.build.build()")
            L = ctypes.CDLL(LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != PROP_OK:
        raise PropError(status, where, lib().prop_last_error().decode(errors="replace"))


class ServeStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("cancelled", ctypes.c_longlong), ("pending", ctypes.c_longlong),
                ("running", ctypes.c_longlong), ("reserved_bytes", c_size_t),
                ("arena_bytes_in_use", c_size_t), ("arena_peak_bytes", c_size_t),
                ("budget_bytes", c_size_t)]
