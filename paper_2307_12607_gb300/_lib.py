"""ctypes loader for libexw.so (the C ABI declared in include/exw.h).

The library is looked up in this package's ``_build/`` directory (built by ``paper_2307_12607_gb300.build``).  There
is no fallback: if it is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libexw.so")

_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I = ctypes.c_int
U = ctypes.c_uint
SZ = ctypes.c_size_t

# C prototypes: name -> (restype, argtypes)
PROTOTYPES = {
    "exw_status_string": (ctypes.c_char_p, [I]),
    "exw_version": (I, []),
    "exw_workspace_bytes": (SZ, [I, I, I, I, I, I]),
    "exw_motion_bounds": (I, [P, P, I, I, P, P, P, SZ, P]),
    "exw_splat_motion": (I, [P, P, I, I, I, I, P, P]),
    "exw_warp": (I, [P, I, P, P, P, I, I, I, I, P, P, P]),
    "exw_fill_holes": (I, [P, I, P, I, I, P, SZ, P]),
    "exw_fill_holes_static": (I, [P, I, P, I, I, P]),
    "exw_extrapolate": (I, [P, I, I, U, P, P, SZ, P]),
    "exw_extrapolate_host": (I, [P, P, I, I, U, P, P, I, P, SZ, P]),
    "exw_mv_variance": (I, [P, I, I, P, P, SZ, P]),
    "exw_carry_motion": (I, [P, P, P, P, I, I, P, P, P]),
    "exw_color_mse": (I, [P, P, I, I, I, P, P, SZ, P]),
    "exw_psnr": (I, [P, P, I, I, I, P, P, SZ, P]),
    "exw_warp_recursive": (I, [P, I, P, P, I, I, I, U, P, P, SZ, P]),
    "exw_ssim": (I, [P, P, I, I, I, P, P, SZ, P]),
    "exw_warp_backward": (I, [P, P, I, P, P, P, I, I, I, I, P, P, P, SZ, P]),
    "exw_l2_loss_grad": (I, [P, P, I, P, I, I, P, P, P]),
    "exw_warp_l2_grad": (I, [P, I, I, P, P, SZ, P]),
    "exw_device_status": (I, [P, P]),
    "exw_tuner_create": (P, []),
    "exw_tuner_destroy": (None, [P]),
    "exw_tuner_fix": (I, [P, I, I, I]),
    "exw_tuner_report": (SZ, [P, ctypes.c_char_p, SZ]),
    "exw_batched_workspace_bytes": (SZ, [P, I, I]),
    "exw_extrapolate_batched": (I, [P, I, I, U, P, SZ, P, P]),
    "exw_timing_enable": (None, [I]),
    "exw_timing_query": (I, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I)]),
    "exw_timing_names": (SZ, [ctypes.c_char_p, SZ]),
    "exw_launch_count": (ctypes.c_uint64, []),
}


class ExwFrame(ctypes.Structure):
    _fields_ = [("color", P), ("depth", P), ("mv", P), ("W", I), ("H", I), ("cdt", I)]


class ExwFrameOut(ctypes.Structure):
    _fields_ = [("color", P), ("mask", P)]


class ExwTrainFrame(ctypes.Structure):
    _fields_ = [("src", ExwFrame), ("target", P * 3), ("grad_color", P), ("grad_mv", P)]


class ExwStreamDesc(ctypes.Structure):
    _fields_ = [("src", ExwFrame), ("out", ExwFrameOut * 3)]


def load(path: str | None = None):
    """Load (once) and return the ctypes handle of libexw.so."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libexw.so not found at {p}: build it with "
                                   "`python -m paper_2307_12607_gb300.build` (the CUDA path has no fallback)")
            lib = ctypes.CDLL(p)
            for name, (res, args) in PROTOTYPES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib
