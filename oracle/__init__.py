"""Python face of the FP64 CPU oracle (``exw_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package; the product path never does.  It shares no code with the CUDA library.

The C file is compiled with gcc on first use (or by ``build()``) into ``oracle/_build/``.  Each wrapper converts
its inputs to the exact types the C code reads (float32 depth/motion, float64 colour -- an FP16 or FP32 colour is
read as its exact value) and returns numpy arrays.  The definitions, and the passages of the paper they follow,
are documented at each C function.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "exw_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libexw_oracle.so")
_lock = threading.Lock()
_lib = None

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
MASK_EMPTY = 1
MASK_CRACK = 2


def compile_source(src: str, out: str) -> str:
    """Compile an oracle C source into the shared library ``out`` (plain C, FP64, no FMA contraction so x86 and Arm
    give the same bits)."""
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``exw_oracle.c`` into ``oracle/_build/`` unless the library is up to date."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # EXW_ORACLE_LIB names another compiled copy to load instead: the mutation test runs the pins against
            # deliberately broken copies of the oracle this way
            lib = ctypes.CDLL(os.environ.get("EXW_ORACLE_LIB") or build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.oracle_target_offset.argtypes = [ctypes.c_float, I, I, ctypes.POINTER(ctypes.c_longlong)]
            lib.oracle_target_offset.restype = I
            lib.oracle_splat.argtypes = [P, P, I, I, I, I, P]
            lib.oracle_mask.argtypes = [P, I, I, P]
            lib.oracle_warp.argtypes = [P, P, P, P, I, I, I, I, P, P]
            lib.oracle_weight_sum.argtypes = [P, P, I, I, I, I, I]
            lib.oracle_weight_sum.restype = ctypes.c_double
            lib.oracle_fill_holes.argtypes = [P, P, I, I]
            lib.oracle_warp_backward.argtypes = [P, P, P, P, P, I, I, I, I, P, P]
            lib.oracle_motion_bounds.argtypes = [P, P, I, I, I, P, P]
            lib.oracle_mv_variance.argtypes = [P, I, I, P]
            lib.oracle_mv_variance.restype = None
            lib.oracle_color_mse.argtypes = [P, P, I, I]
            lib.oracle_color_mse.restype = ctypes.c_double
            lib.oracle_carry_motion.argtypes = [P, P, P, P, I, I, P, P]
            lib.oracle_carry_motion.restype = None
            lib.oracle_ssim.argtypes = [P, P, I, I]
            lib.oracle_ssim.restype = ctypes.c_double
            for f in (lib.oracle_splat, lib.oracle_mask, lib.oracle_warp, lib.oracle_fill_holes,
                      lib.oracle_warp_backward, lib.oracle_motion_bounds):
                f.restype = None
            _lib = lib
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(depth):
    H, W = depth.shape
    return int(W), int(H)


def target_offset(mv: float, k: int, denom: int = 4):
    """floor(1/2 + k*mv/denom) for one float32 ``mv``; None when it cannot land in any frame."""
    out = ctypes.c_longlong(0)
    ok = _load().oracle_target_offset(ctypes.c_float(np.float32(mv)), int(k), int(denom), ctypes.byref(out))
    return int(out.value) if ok else None


def splat(depth, mv, k: int, denom: int = 4):
    """Forward z-buffered splat: uint64 keys [H][W] (EMPTY where nothing lands)."""
    depth, mv = _f32(depth), _f32(mv)
    W, H = _dims(depth)
    keys = np.empty((H, W), np.uint64)
    _load().oracle_splat(_ptr(depth), _ptr(mv), W, H, int(k), int(denom), _ptr(keys))
    return keys


def mask_from_keys(keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    H, W = keys.shape
    mask = np.empty((H, W), np.uint8)
    _load().oracle_mask(_ptr(keys), W, H, _ptr(mask))
    return mask


def warp(color, depth, mv, keys, k: int, denom: int = 4):
    """Backward bilinear gather with hole mask: (out float64 [3][H][W], mask uint8 [H][W])."""
    color, depth, mv = _f64(color), _f32(depth), _f32(mv)
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    W, H = _dims(depth)
    out = np.empty((3, H, W), np.float64)
    mask = np.empty((H, W), np.uint8)
    _load().oracle_warp(_ptr(color), _ptr(depth), _ptr(mv), _ptr(keys), W, H, int(k), int(denom), _ptr(out),
                        _ptr(mask))
    return out, mask


def weight_sum(mv, keys, q: int, k: int, denom: int = 4) -> float:
    mv = _f32(mv)
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    H, W = keys.shape
    return _load().oracle_weight_sum(_ptr(mv), _ptr(keys), W, H, int(k), int(denom), int(q))


def fill_holes(color, mask):
    """Pull-push fill of the pixels with mask != 0: float64 [3][H][W]."""
    out = np.array(color, dtype=np.float64, order="C", copy=True)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    H, W = mask.shape
    _load().oracle_fill_holes(_ptr(out), _ptr(mask), W, H)
    return out


def warp_backward(grad_out, color, depth, mv, keys, k: int, denom: int = 4, grad_color=None, grad_mv=None):
    """Adjoint of ``warp`` w.r.t. colour and motion, accumulated into (and returned as) float64 arrays."""
    grad_out, color, depth, mv = _f64(grad_out), _f64(color), _f32(depth), _f32(mv)
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    W, H = _dims(depth)
    gc = np.zeros((3, H, W), np.float64) if grad_color is None else _f64(grad_color).copy()
    gm = np.zeros((2, H, W), np.float64) if grad_mv is None else _f64(grad_mv).copy()
    _load().oracle_warp_backward(_ptr(grad_out), _ptr(color), _ptr(depth), _ptr(mv), _ptr(keys), W, H, int(k),
                                 int(denom), _ptr(gc), _ptr(gm))
    return gc, gm


def motion_bounds(depth, mv, block: int = 8):
    """Per-tile and whole-frame [min mvx, max mvx, min mvy, max mvy] over splattable pixels."""
    depth, mv = _f32(depth), _f32(mv)
    W, H = _dims(depth)
    nbx, nby = (W + block - 1) // block, (H + block - 1) // block
    tiles = np.empty((nby, nbx, 4), np.float32)
    frame = np.empty(4, np.float32)
    _load().oracle_motion_bounds(_ptr(depth), _ptr(mv), W, H, int(block), _ptr(tiles), _ptr(frame))
    return tiles, frame


def halo(frame_bounds, k: int, denom: int = 4) -> int:
    """Largest |target offset| of fraction k over a frame, from its motion bounds (monotone in mv)."""
    if not np.isfinite(frame_bounds[0]):
        return 0
    return max(abs(target_offset(float(v), k, denom)) for v in frame_bounds)


def extrapolate(color, depth, mv, nfrac: int = 3, storage=np.float32, fill: bool = True):
    """P_1..P_nfrac at t + k/4 (Sec. IV-B): splat, warp, round the warped colour once to the storage type, fill.
    Returns a list of (colour float64 [3][H][W], mask uint8 [H][W], keys uint64 [H][W])."""
    res = []
    for k in range(1, nfrac + 1):
        keys = splat(depth, mv, k, 4)
        out, mask = warp(color, depth, mv, keys, k, 4)
        if fill:
            stored = out.astype(storage).astype(np.float64)
            out = fill_holes(stored, mask)
        res.append((out, mask, keys))
    return res


def l2_loss_grad(out, target, mask):
    """L = sum over non-hole pixels and channels of (out - target)^2 and dL/d out (zero on holes)."""
    out = _f64(out)
    target = _f64(target)
    valid = (np.asarray(mask) == 0)[None, :, :]
    diff = np.where(valid, out - target, 0.0)
    return float(np.sum(diff * diff)), 2.0 * diff


def mv_variance(mv):
    """(count, Var_x, Var_y) of the finite motion vectors of a [2][H][W] field (Sec. IV-C Eq. 1, see the C code)."""
    mv = _f32(mv)
    H, W = mv.shape[1], mv.shape[2]
    out = np.zeros(3, np.float64)
    _load().oracle_mv_variance(_ptr(mv), W, H, _ptr(out))
    return float(out[0]), float(out[1]), float(out[2])


def color_mse(a, b):
    """Mean squared difference of two [3][H][W] colour images in FP64 (Sec. IV-C Eq. 3's MSE)."""
    a = _f64(a)
    b = _f64(b)
    return float(_load().oracle_color_mse(_ptr(a), _ptr(b), a.shape[2], a.shape[1]))


def psnr(a, b) -> float:
    """PSNR = 10 log10(255^2 / MSE) of colours in [0, 1] scaled by 255 (Sec. IV-C Eq. 3); inf for equal images."""
    mse = color_mse(a, b)
    return float("inf") if mse == 0.0 else 10.0 * np.log10(1.0 / mse)


def ssim(a, b) -> float:
    """Mean SSIM of two [3][H][W] colour images in [0, 1] (11 x 11 Gaussian window, sigma 1.5, valid positions;
    Sec. IV-C Eq. 3, see the C code).  NaN when W or H is below 11."""
    a = _f64(a)
    b = _f64(b)
    return float(_load().oracle_ssim(_ptr(a), _ptr(b), a.shape[2], a.shape[1]))


def carry_motion(keys, mask, depth, mv):
    """Depth [H][W] and motion [2][H][W] of a warped frame for warping it again (Table V, S5/S6; see the C code)."""
    keys = np.ascontiguousarray(keys).view(np.uint64)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    depth = _f32(depth)
    mv = _f32(mv)
    H, W = depth.shape
    d_out = np.empty((H, W), np.float32)
    mv_out = np.empty((2, H, W), np.float32)
    _load().oracle_carry_motion(_ptr(keys), _ptr(mask), _ptr(depth), _ptr(mv), W, H, _ptr(d_out), _ptr(mv_out))
    return d_out, mv_out


def warp_recursive(color, depth, mv, steps: int, fill: bool = True):
    """Decision path S6 (Table V): P_1 = W(F), P_{i+1} = W(P_i), each a quarter step (k = 1 of 4) of the motion each
    pixel carries (carry_motion); FP64 colour, filled after each warp when ``fill``.  Returns [(colour, mask)]."""
    c = _f64(color)
    d, m = _f32(depth), _f32(mv)
    outs = []
    for _ in range(steps):
        keys = splat(d, m, 1, 4)
        out, mask = warp(c, d, m, keys, 1, 4)
        if fill:
            out = fill_holes(out, mask)
        outs.append((out, mask))
        d, m = carry_motion(keys, mask, d, m)
        c = out
    return outs
