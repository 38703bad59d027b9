"""Python binding of libexw: the C entry points under the same names, marshalling torch CUDA tensors to pointers.

Every function checks devices, dtypes, shapes and contiguity, allocates outputs the caller did not pass (torch is
the device-memory allocator; the library itself never allocates), passes the current torch CUDA stream and raises
``ExwError`` on a non-zero status.  All arithmetic runs in the CUDA kernels of libexw.so; nothing here computes.

Layouts (see include/exw.h): colour [3][H][W] float32/float16, depth [H][W] float32, motion [2][H][W] float32
(plane 0 = x), keys [H][W] (uint64 bit patterns held in an int64 tensor), mask [H][W] uint8.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib

F32, F16 = 0, 1
OP_MOTION_BOUNDS, OP_FILL_HOLES, OP_EXTRAPOLATE, OP_WARP_BACKWARD = 0, 1, 2, 3
FLAG_NO_FILL = 1
FLAG_NO_TMA = 2
MASK_EMPTY, MASK_CRACK = 1, 2
KEY_EMPTY = -1  # all-ones uint64 as int64
MAX_FRAC = 3


class ExwError(RuntimeError):
    def __init__(self, status: int, text: str):
        super().__init__(f"libexw status {status}: {text}")
        self.status = status


def lib():
    return _lib.load()


def _check(status: int):
    if status != 0:
        raise ExwError(status, lib().exw_status_string(status).decode())


def _cdt(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float16:
        return F16
    raise TypeError(f"colour must be float32 or float16, got {t.dtype}")


def _dev(t: torch.Tensor, name: str, dtype=None, shape=None) -> int:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (libexw runs on the GPU only)")
    if t.device.index != torch.cuda.current_device():  # the kernels launch on the current device
        raise ValueError(f"{name} is on {t.device}, not on the current device cuda:{torch.cuda.current_device()} "
                         "(select it with torch.cuda.device)")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream(stream, device) -> int:
    if stream is None:
        return torch.cuda.current_stream(device).cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _hw(depth: torch.Tensor):
    if depth.dim() != 2:
        raise ValueError("depth must be [H][W]")
    return int(depth.shape[1]), int(depth.shape[0])


def exw_status_string(status: int) -> str:
    return lib().exw_status_string(int(status)).decode()


def exw_version() -> int:
    return int(lib().exw_version())


def exw_workspace_bytes(op: int, W: int, H: int, cdt: int = F32, nframes: int = 1, nfrac: int = 1) -> int:
    return int(lib().exw_workspace_bytes(op, W, H, cdt, nframes, nfrac))


def workspace(nbytes: int, device) -> torch.Tensor:
    """Device workspace of at least ``nbytes`` (torch allocates it; contents need no initialisation)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def exw_motion_bounds(depth, mv, tile_bounds=None, frame_bounds=None, ws=None, stream=None):
    """Stage (a0).  Returns (tile_bounds [ceil(H/8)][ceil(W/8)][4], frame_bounds [4]) float32."""
    W, H = _hw(depth)
    dev = depth.device
    if tile_bounds is None:
        tile_bounds = torch.empty(((H + 7) // 8, (W + 7) // 8, 4), dtype=torch.float32, device=dev)
    if frame_bounds is None:
        frame_bounds = torch.empty(4, dtype=torch.float32, device=dev)
    need = exw_workspace_bytes(OP_MOTION_BOUNDS, W, H)
    if ws is None:
        ws = workspace(need, dev)
    _check(lib().exw_motion_bounds(_dev(depth, "depth", torch.float32), _dev(mv, "mv", torch.float32, (2, H, W)),
                                   W, H, _dev(tile_bounds, "tile_bounds", torch.float32),
                                   _dev(frame_bounds, "frame_bounds", torch.float32), ws.data_ptr(), ws.numel(),
                                   _stream(stream, dev)))
    return tile_bounds, frame_bounds


def exw_splat_motion(depth, mv, k: int, denom: int = 4, keys=None, stream=None):
    """Stage (a).  Returns keys [H][W] (int64 tensor holding the uint64 keys)."""
    W, H = _hw(depth)
    if keys is None:
        keys = torch.empty((H, W), dtype=torch.int64, device=depth.device)
    _check(lib().exw_splat_motion(_dev(depth, "depth", torch.float32), _dev(mv, "mv", torch.float32, (2, H, W)), W,
                                  H, int(k), int(denom), _dev(keys, "keys", torch.int64, (H, W)),
                                  _stream(stream, depth.device)))
    return keys


def exw_warp(color, depth, mv, keys, k: int, denom: int = 4, out=None, mask=None, stream=None):
    """Stage (b).  Returns (out colour [3][H][W] in the colour dtype, mask [H][W] uint8)."""
    W, H = _hw(depth)
    if out is None:
        out = torch.empty((3, H, W), dtype=color.dtype, device=color.device)
    if mask is None:
        mask = torch.empty((H, W), dtype=torch.uint8, device=color.device)
    _check(lib().exw_warp(_dev(color, "color", None, (3, H, W)), _cdt(color), _dev(depth, "depth", torch.float32),
                          _dev(mv, "mv", torch.float32, (2, H, W)), _dev(keys, "keys", torch.int64, (H, W)), W, H,
                          int(k), int(denom), _dev(out, "out", color.dtype, (3, H, W)),
                          _dev(mask, "mask", torch.uint8, (H, W)), _stream(stream, color.device)))
    return out, mask


def exw_fill_holes(color, mask, ws=None, stream=None):
    """Stage (c), in place on ``color``.  Returns ``color``."""
    H, W = int(mask.shape[0]), int(mask.shape[1])
    need = exw_workspace_bytes(OP_FILL_HOLES, W, H, _cdt(color))
    if ws is None:
        ws = workspace(need, color.device)
    _check(lib().exw_fill_holes(_dev(color, "color", None, (3, H, W)), _cdt(color),
                                _dev(mask, "mask", torch.uint8, (H, W)), W, H, ws.data_ptr(), ws.numel(),
                                _stream(stream, color.device)))
    return color


def exw_fill_holes_static(color, mask, stream=None):
    """Stage (c) in place, with the library's built-in scratch array instead of a workspace (for callers that
    cannot allocate device memory; frames up to 16384 fill tiles of 32 x 32).  Calls that may overlap on the GPU
    share that array and must be serialised by the caller.  Returns ``color``."""
    H, W = int(mask.shape[0]), int(mask.shape[1])
    _check(lib().exw_fill_holes_static(_dev(color, "color", None, (3, H, W)), _cdt(color),
                                       _dev(mask, "mask", torch.uint8, (H, W)), W, H, _stream(stream, color.device)))
    return color


def exw_extrapolate(color, depth, mv, nfrac: int = 3, fill: bool = True, out=None, mask=None, ws=None, stream=None,
                    tma: bool = True):
    """Stages (a0)+(a)+(b)+(c) for one frame ([3][H][W] colour) or a sequence ([F][3][H][W]).

    Returns (out [F][nfrac][3][H][W], mask [F][nfrac][H][W]) -- without the F axis for a single frame.
    ``tma=False`` sets EXW_FLAG_NO_TMA (global-memory source reads; identical results)."""
    single = color.dim() == 3
    if single:
        color, depth, mv = color.unsqueeze(0), depth.unsqueeze(0), mv.unsqueeze(0)
    F, _, H, W = (int(s) for s in color.shape)
    dev = color.device
    cdt = _cdt(color)
    if out is None:
        out = torch.empty((F, nfrac, 3, H, W), dtype=color.dtype, device=dev)
    if mask is None:
        mask = torch.empty((F, nfrac, H, W), dtype=torch.uint8, device=dev)
    _dev(color, "color", None, (F, 3, H, W))
    _dev(depth, "depth", torch.float32, (F, H, W))
    _dev(mv, "mv", torch.float32, (F, 2, H, W))
    _dev(out, "out", color.dtype, (F, nfrac, 3, H, W))
    _dev(mask, "mask", torch.uint8, (F, nfrac, H, W))
    need = exw_workspace_bytes(OP_EXTRAPOLATE, W, H, cdt, F, nfrac)
    if ws is None:
        ws = workspace(need, dev)
    frames = (_lib.ExwFrame * F)()
    outs = (_lib.ExwFrameOut * (F * nfrac))()
    for f in range(F):
        frames[f] = _lib.ExwFrame(color[f].data_ptr(), depth[f].data_ptr(), mv[f].data_ptr(), W, H, cdt)
        for j in range(nfrac):
            outs[f * nfrac + j] = _lib.ExwFrameOut(out[f, j].data_ptr(), mask[f, j].data_ptr())
    flags = (0 if fill else FLAG_NO_FILL) | (0 if tma else FLAG_NO_TMA)
    _check(lib().exw_extrapolate(ctypes.cast(frames, ctypes.c_void_p), F, int(nfrac), flags,
                                 ctypes.cast(outs, ctypes.c_void_p), ws.data_ptr(), ws.numel(),
                                 _stream(stream, dev)))
    if single:
        return out[0], mask[0]
    return out, mask


def exw_extrapolate_host(color, depth, mv, nfrac: int = 3, fill: bool = True, out=None, mask=None, dev_in=None,
                         dev_out=None, ws=None, chunk: int = 8, stream=None, tma: bool = True, direct: bool = False):
    """exw_extrapolate for a sequence in HOST memory ([F][3][H][W] colour, [F][H][W] depth, [F][2][H][W] motion;
    page-locked for the copies to overlap): the copies in, the work and the copies out run chunk by chunk on
    three streams inside the call.  Returns host (out [F][nfrac][3][H][W], mask [F][nfrac][H][W]) once the
    caller's stream has been synchronised.  dev_in = (colour, depth, motion) and dev_out = (out, mask): device
    staging tensors of the same shapes (allocated here when None).  direct=True: the engine writes the outputs
    straight into the (page-locked) host tensors; dev_out is not used."""
    F, _, H, W = (int(v) for v in color.shape)
    cdt = _cdt(color)
    dev = torch.device("cuda", torch.cuda.current_device())
    if out is None:
        out = torch.empty((F, nfrac, 3, H, W), dtype=color.dtype).pin_memory()
    if mask is None:
        mask = torch.empty((F, nfrac, H, W), dtype=torch.uint8).pin_memory()
    for t, name in ((color, "color"), (depth, "depth"), (mv, "mv"), (out, "out"), (mask, "mask")):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name}: a contiguous host tensor is expected")
    if dev_in is None:
        dev_in = (torch.empty_like(color, device=dev), torch.empty_like(depth, device=dev),
                  torch.empty_like(mv, device=dev))
    if dev_out is None and not direct:
        dev_out = (torch.empty_like(out, device=dev), torch.empty_like(mask, device=dev))
    dc, dd, dm = dev_in
    do, dk = dev_out if not direct else (out, mask)
    _dev(dc, "dev color", color.dtype, (F, 3, H, W))
    _dev(dd, "dev depth", torch.float32, (F, H, W))
    _dev(dm, "dev mv", torch.float32, (F, 2, H, W))
    if not direct:
        _dev(do, "dev out", color.dtype, (F, nfrac, 3, H, W))
        _dev(dk, "dev mask", torch.uint8, (F, nfrac, H, W))
    need = exw_workspace_bytes(OP_EXTRAPOLATE, W, H, cdt, min(chunk, F) if chunk > 0 else min(8, F), nfrac)
    if ws is None:
        ws = workspace(need, dev)
    fh = (_lib.ExwFrame * F)()
    fd = (_lib.ExwFrame * F)()
    oh = (_lib.ExwFrameOut * (F * nfrac))()
    od = (_lib.ExwFrameOut * (F * nfrac))()
    for f in range(F):
        fh[f] = _lib.ExwFrame(color[f].data_ptr(), depth[f].data_ptr(), mv[f].data_ptr(), W, H, cdt)
        fd[f] = _lib.ExwFrame(dc[f].data_ptr(), dd[f].data_ptr(), dm[f].data_ptr(), W, H, cdt)
        for j in range(nfrac):
            oh[f * nfrac + j] = _lib.ExwFrameOut(out[f, j].data_ptr(), mask[f, j].data_ptr())
            od[f * nfrac + j] = _lib.ExwFrameOut(do[f, j].data_ptr(), dk[f, j].data_ptr())
    flags = (0 if fill else FLAG_NO_FILL) | (0 if tma else FLAG_NO_TMA)
    _check(lib().exw_extrapolate_host(ctypes.cast(fh, ctypes.c_void_p), ctypes.cast(fd, ctypes.c_void_p), F,
                                      int(nfrac), flags, ctypes.cast(oh, ctypes.c_void_p),
                                      None if direct else ctypes.cast(od, ctypes.c_void_p), int(chunk),
                                      ws.data_ptr(), ws.numel(),
                                      _stream(stream, dev)))
    return out, mask


OP_STATS = 4
OP_WARP_RECURSIVE = 5
OP_WARP_L2_GRAD = 6


def exw_carry_motion(keys, mask, depth, mv, depth_out=None, mv_out=None, stream=None):
    """Depth and motion of a warped frame for warping it again (Table V, S5/S6): returns (depth [H][W], motion
    [2][H][W]) -- the winners' for non-holes, NaN depth and zero motion for holes."""
    W, H = _hw(depth)
    dev = depth.device
    if depth_out is None:
        depth_out = torch.empty((H, W), dtype=torch.float32, device=dev)
    if mv_out is None:
        mv_out = torch.empty((2, H, W), dtype=torch.float32, device=dev)
    _check(lib().exw_carry_motion(_dev(keys, "keys", torch.int64, (H, W)), _dev(mask, "mask", torch.uint8, (H, W)),
                                  _dev(depth, "depth", torch.float32), _dev(mv, "mv", torch.float32, (2, H, W)), W, H,
                                  _dev(depth_out, "depth_out", torch.float32, (H, W)),
                                  _dev(mv_out, "mv_out", torch.float32, (2, H, W)), _stream(stream, dev)))
    return depth_out, mv_out


def exw_warp_recursive(color, depth, mv, steps: int = 3, fill: bool = True, out=None, mask=None, ws=None,
                       stream=None):
    """Decision path S6 (Table V): P_1 = W(F), P_{i+1} = W(P_i), each a quarter step (k = 1 of 4) of the motion
    every pixel carries, chained on the device by the library (exw_warp_recursive).  Returns [(colour [3][H][W],
    mask [H][W])] for the ``steps`` frames (views of ``out`` [steps][3][H][W] and ``mask`` [steps][H][W])."""
    W, H = _hw(depth)
    dev = color.device
    steps = int(steps)
    if out is None:
        out = torch.empty((steps, 3, H, W), dtype=color.dtype, device=dev)
    if mask is None:
        mask = torch.empty((steps, H, W), dtype=torch.uint8, device=dev)
    _dev(out, "out", color.dtype, (steps, 3, H, W))
    _dev(mask, "mask", torch.uint8, (steps, H, W))
    if ws is None:
        ws = workspace(exw_workspace_bytes(OP_WARP_RECURSIVE, W, H, _cdt(color)), dev)
    outs = (_lib.ExwFrameOut * steps)()
    for i in range(steps):
        outs[i] = _lib.ExwFrameOut(out[i].data_ptr(), mask[i].data_ptr())
    _check(lib().exw_warp_recursive(_dev(color, "color", None, (3, H, W)), _cdt(color),
                                    _dev(depth, "depth", torch.float32), _dev(mv, "mv", torch.float32, (2, H, W)), W,
                                    H, steps, 0 if fill else FLAG_NO_FILL, ctypes.cast(outs, ctypes.c_void_p),
                                    ws.data_ptr(), ws.numel(), _stream(stream, dev)))
    return [(out[i], mask[i]) for i in range(steps)]


def exw_mv_variance(mv, ws=None, stream=None):
    """Motion-variance features (count, Var_x, Var_y) of a [2][H][W] float32 motion field (Sec. IV-C, Eq. 1):
    population variances over the pixels whose two components are finite, FP64 on the device (reads the result
    back, so it synchronises with the stream)."""
    H, W = int(mv.shape[1]), int(mv.shape[2])
    _dev(mv, "mv", torch.float32, (2, H, W))
    dev = mv.device
    if ws is None:
        ws = workspace(exw_workspace_bytes(OP_STATS, W, H, F32, 1, 1), dev)
    out = torch.empty(3, dtype=torch.float64, device=dev)
    _check(lib().exw_mv_variance(mv.data_ptr(), W, H, out.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream, dev)))
    n, vx, vy = out.tolist()
    return n, vx, vy


def exw_color_mse(a, b, ws=None, stream=None) -> float:
    """Mean squared difference of two [3][H][W] colour images of one dtype over all 3 W H values, FP64 on the
    device (Sec. IV-C, Eq. 3's MSE; synchronises to read it back)."""
    H, W = int(a.shape[1]), int(a.shape[2])
    _dev(a, "a", None, (3, H, W))
    _dev(b, "b", a.dtype, (3, H, W))
    dev = a.device
    if ws is None:
        ws = workspace(exw_workspace_bytes(OP_STATS, W, H, F32, 1, 1), dev)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    _check(lib().exw_color_mse(a.data_ptr(), b.data_ptr(), _cdt(a), W, H, out.data_ptr(), ws.data_ptr(), ws.numel(),
                               _stream(stream, dev)))
    return float(out.item())


def exw_ssim(a, b, ws=None, stream=None) -> float:
    """Mean SSIM of two [3][H][W] colour images in [0, 1] of one dtype (Sec. IV-C, Eq. 3; 11 x 11 Gaussian window,
    valid positions; W, H >= 11).  Synchronises to read the result back."""
    H, W = int(a.shape[1]), int(a.shape[2])
    _dev(a, "a", None, (3, H, W))
    _dev(b, "b", a.dtype, (3, H, W))
    dev = a.device
    if ws is None:
        ws = workspace(exw_workspace_bytes(OP_STATS, W, H, F32, 1, 1), dev)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    _check(lib().exw_ssim(a.data_ptr(), b.data_ptr(), _cdt(a), W, H, out.data_ptr(), ws.data_ptr(), ws.numel(),
                          _stream(stream, dev)))
    return float(out.item())


def exw_psnr(a, b, ws=None, stream=None) -> float:
    """PSNR = 10 log10(255^2 / MSE) of colours in [0, 1] scaled by 255 (Sec. IV-C, Eq. 3), computed on the device
    (exw_psnr); inf for equal images.  Synchronises to read it back."""
    H, W = int(a.shape[1]), int(a.shape[2])
    _dev(a, "a", None, (3, H, W))
    _dev(b, "b", a.dtype, (3, H, W))
    dev = a.device
    if ws is None:
        ws = workspace(exw_workspace_bytes(OP_STATS, W, H, F32, 1, 1), dev)
    out = torch.empty(2, dtype=torch.float64, device=dev)
    _check(lib().exw_psnr(a.data_ptr(), b.data_ptr(), _cdt(a), W, H, out.data_ptr(), ws.data_ptr(), ws.numel(),
                          _stream(stream, dev)))
    return float(out[1].item())


def exw_tuner_create() -> int:
    """Host-side autotuner handle for exw_extrapolate_batched (free it with exw_tuner_destroy)."""
    return int(lib().exw_tuner_create())


def exw_tuner_destroy(tuner: int):
    lib().exw_tuner_destroy(tuner)


def exw_tuner_fix(tuner: int, shape: int, lag: int = 1, pair: bool = True):
    """Make ``tuner`` run one schedule (window shape 0 or 1, queue distance, smooth-tile sharing) for every batch."""
    _check(lib().exw_tuner_fix(tuner, int(shape), int(lag), 1 if pair else 0))


def exw_tuner_report(tuner: int) -> str:
    need = int(lib().exw_tuner_report(tuner, None, 0))
    buf = ctypes.create_string_buffer(need)
    lib().exw_tuner_report(tuner, buf, need)
    return buf.value.decode()


def _stream_descs(streams, outs, nfrac):
    descs = (_lib.ExwStreamDesc * len(streams))()
    for i, ((color, depth, mv), (out, mask)) in enumerate(zip(streams, outs)):
        H, W = int(depth.shape[0]), int(depth.shape[1])
        _dev(color, "color", None, (3, H, W))
        _dev(depth, "depth", torch.float32, (H, W))
        _dev(mv, "mv", torch.float32, (2, H, W))
        _dev(out, "out", color.dtype, (nfrac, 3, H, W))
        _dev(mask, "mask", torch.uint8, (nfrac, H, W))
        descs[i].src = _lib.ExwFrame(color.data_ptr(), depth.data_ptr(), mv.data_ptr(), W, H, _cdt(color))
        for j in range(nfrac):
            descs[i].out[j] = _lib.ExwFrameOut(out[j].data_ptr(), mask[j].data_ptr())
    return descs


def exw_batched_workspace_bytes(streams, nfrac: int = 3) -> int:
    descs = (_lib.ExwStreamDesc * len(streams))()
    for i, (color, depth, mv) in enumerate(streams):
        descs[i].src = _lib.ExwFrame(0, 0, 0, int(depth.shape[1]), int(depth.shape[0]), _cdt(color))
    return int(lib().exw_batched_workspace_bytes(ctypes.cast(descs, ctypes.c_void_p), len(streams), int(nfrac)))


def exw_extrapolate_batched(streams, nfrac: int = 3, fill: bool = True, outs=None, ws=None, tuner=None, stream=None,
                            tma: bool = True):
    """All stages for many independent streams in one persistent launch.  ``streams`` is a list of (colour
    [3][H][W], depth [H][W], motion [2][H][W]) with per-stream sizes and colour types.  Returns a list of
    (out [nfrac][3][H][W], mask [nfrac][H][W]).  ``tuner``: handle from exw_tuner_create (or None)."""
    dev = streams[0][0].device
    if outs is None:
        outs = [(torch.empty((nfrac,) + tuple(c.shape), dtype=c.dtype, device=dev),
                 torch.empty((nfrac,) + tuple(d.shape), dtype=torch.uint8, device=dev)) for c, d, _ in streams]
    descs = _stream_descs(streams, outs, nfrac)
    need = int(lib().exw_batched_workspace_bytes(ctypes.cast(descs, ctypes.c_void_p), len(streams), int(nfrac)))
    if ws is None:
        ws = workspace(need, dev)
    flags = (0 if fill else FLAG_NO_FILL) | (0 if tma else FLAG_NO_TMA)
    _check(lib().exw_extrapolate_batched(ctypes.cast(descs, ctypes.c_void_p), len(streams), int(nfrac), flags,
                                         ws.data_ptr(), ws.numel(), tuner or None, _stream(stream, dev)))
    return outs


def exw_warp_backward(grad_out, color, depth, mv, keys, k: int, denom: int = 4, grad_color=None, grad_mv=None,
                      ws=None, stream=None):
    """Adjoint of stage (b); accumulates into (and returns) grad_color [3][H][W] and grad_mv [2][H][W] float32.
    ``keys=None`` recomputes the keys into the workspace."""
    W, H = _hw(depth)
    dev = color.device
    if grad_color is None:
        grad_color = torch.zeros((3, H, W), dtype=torch.float32, device=dev)
    if grad_mv is None:
        grad_mv = torch.zeros((2, H, W), dtype=torch.float32, device=dev)
    kptr = 0 if keys is None else _dev(keys, "keys", torch.int64, (H, W))
    wsp, wsn = 0, 0
    if keys is None:
        if ws is None:
            ws = workspace(exw_workspace_bytes(OP_WARP_BACKWARD, W, H, _cdt(color)), dev)
        wsp, wsn = ws.data_ptr(), ws.numel()
    _check(lib().exw_warp_backward(_dev(grad_out, "grad_out", torch.float32, (3, H, W)),
                                   _dev(color, "color", None, (3, H, W)), _cdt(color),
                                   _dev(depth, "depth", torch.float32), _dev(mv, "mv", torch.float32, (2, H, W)),
                                   kptr, W, H, int(k), int(denom),
                                   _dev(grad_color, "grad_color", torch.float32, (3, H, W)),
                                   _dev(grad_mv, "grad_mv", torch.float32, (2, H, W)), wsp, wsn,
                                   _stream(stream, dev)))
    return grad_color, grad_mv


def exw_warp_l2_grad(color, depth, mv, targets, nfrac: int = 3, grad_color=None, grad_mv=None, loss=None, ws=None,
                     stream=None):
    """Forward warp, L2 loss and adjoint of P_1..P_nfrac for a batch of frames in one call (exw_warp_l2_grad):
    colour [F][3][H][W], depth [F][H][W], motion [F][2][H][W], targets [F][nfrac][3][H][W] (the colour dtype).
    Returns (loss [F] float64 -- per frame, the sum over fractions, non-hole targets and channels of the squared
    difference --, grad_color [F][3][H][W], grad_mv [F][2][H][W]); the gradients are accumulated into the tensors
    passed (zeros when None)."""
    F, _, H, W = (int(v) for v in color.shape)
    dev = color.device
    cdt = _cdt(color)
    if grad_color is None:
        grad_color = torch.zeros((F, 3, H, W), dtype=torch.float32, device=dev)
    if grad_mv is None:
        grad_mv = torch.zeros((F, 2, H, W), dtype=torch.float32, device=dev)
    if loss is None:
        loss = torch.empty(F, dtype=torch.float64, device=dev)
    _dev(color, "color", None, (F, 3, H, W))
    _dev(depth, "depth", torch.float32, (F, H, W))
    _dev(mv, "mv", torch.float32, (F, 2, H, W))
    _dev(targets, "targets", color.dtype, (F, nfrac, 3, H, W))
    _dev(grad_color, "grad_color", torch.float32, (F, 3, H, W))
    _dev(grad_mv, "grad_mv", torch.float32, (F, 2, H, W))
    _dev(loss, "loss", torch.float64, (F,))
    if ws is None:
        ws = workspace(exw_workspace_bytes(OP_WARP_L2_GRAD, W, H, cdt, 1, nfrac), dev)
    frames = (_lib.ExwTrainFrame * F)()
    for f in range(F):
        frames[f].src = _lib.ExwFrame(color[f].data_ptr(), depth[f].data_ptr(), mv[f].data_ptr(), W, H, cdt)
        for j in range(nfrac):
            frames[f].target[j] = targets[f, j].data_ptr()
        frames[f].grad_color = grad_color[f].data_ptr()
        frames[f].grad_mv = grad_mv[f].data_ptr()
    _check(lib().exw_warp_l2_grad(ctypes.cast(frames, ctypes.c_void_p), F, int(nfrac), loss.data_ptr(),
                                  ws.data_ptr(), ws.numel(), _stream(stream, dev)))
    return loss, grad_color, grad_mv


def exw_l2_loss_grad(out, target, mask, grad_out=None, loss=None, stream=None):
    """L2 loss over non-hole pixels.  Returns (loss [1] float32, accumulated; grad_out [3][H][W] float32)."""
    H, W = int(mask.shape[0]), int(mask.shape[1])
    dev = out.device
    if grad_out is None:
        grad_out = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
    _check(lib().exw_l2_loss_grad(_dev(out, "out", None, (3, H, W)), _dev(target, "target", out.dtype, (3, H, W)),
                                  _cdt(out), _dev(mask, "mask", torch.uint8, (H, W)), W, H,
                                  _dev(grad_out, "grad_out", torch.float32, (3, H, W)),
                                  _dev(loss, "loss", torch.float32), _stream(stream, dev)))
    return loss, grad_out


def frame_stats(ws, frame: int = 0) -> dict:
    """Diagnostics an exw_extrapolate call leaves in its workspace for source frame ``frame``: tiles per staging
    mode (smooth uniform motion / other uniform motion / one window for all fractions / one per fraction / global
    memory / nothing lands), per fraction, tiles without any valid pixel, and the lazy level-5 nodes the coarse
    passes computed (smooth tiles from their source, other tiles without a hole from their stored outputs).  Reads
    the 128-byte frame header at byte 256 + 128 * frame (see csrc/exw_internal.h)."""
    words = ws[256 + 128 * frame: 256 + 128 * (frame + 1)].view(torch.int32).cpu().tolist()
    return {"tiles_smooth": words[15], "tiles_uniform": words[10], "tiles_window_all": words[11],
            "tiles_window_each": words[12], "tiles_global": words[13], "tiles_nothing_lands": words[14],
            "tiles_without_valid_pixel": words[5:8],
            "lazy_nodes_computed": {"smooth": words[18], "from_outputs": words[19]}}


def exw_device_status(ws, stream=None) -> int:
    return int(lib().exw_device_status(ws.data_ptr(), _stream(stream, ws.device)))


def exw_timing_enable(on: bool = True):
    lib().exw_timing_enable(1 if on else 0)


def exw_timing_query(name: str):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int(0)
    rc = lib().exw_timing_query(name.encode(), ctypes.byref(ms), ctypes.byref(n))
    return (float(ms.value), int(n.value)) if rc == 0 else (0.0, 0)


def exw_timing_names():
    need = int(lib().exw_timing_names(None, 0))
    buf = ctypes.create_string_buffer(need)
    lib().exw_timing_names(buf, need)
    s = buf.value.decode()
    return [x for x in s.split(",") if x]


def exw_launch_count() -> int:
    return int(lib().exw_launch_count())
