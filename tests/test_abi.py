"""CPU checks of the C ABI: the library builds and loads, exports every function include/*.h declares, the Python
binding's prototype table matches the header, and the host-side argument checks reject bad input before any CUDA
call.  No kernel runs here (there is no GPU on the build machine)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"^EXW_API\s+[\w\s\*]*?\b(exw_\w+)\s*\(", text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2307_12607_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("exw_splat_motion", "exw_warp", "exw_fill_holes", "exw_extrapolate", "exw_warp_backward",
                     "exw_extrapolate_batched", "exw_motion_bounds", "exw_workspace_bytes"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2307_12607_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(_lib.PROTOTYPES) == declared_functions()


def test_status_strings_and_version(lib):
    assert lib.exw_status_string(0) == b"EXW_OK"
    for s in range(1, 6):
        assert lib.exw_status_string(s).startswith(b"EXW_ERR_")
    assert lib.exw_version() >= 100


def test_workspace_sizes(lib):
    from paper_2307_12607_gb300 import binding as b
    n1 = b.exw_workspace_bytes(b.OP_EXTRAPOLATE, 1920, 1080, b.F32, 1, 3)
    n60 = b.exw_workspace_bytes(b.OP_EXTRAPOLATE, 1920, 1080, b.F32, 60, 3)
    # per frame: a header; per frame in flight (at most 48 per launch): bounds, plans with their candidate source
    # tiles (1 KB per 32 x 32 target tile), pyramid nodes -- a few percent of the frames' own input bytes
    assert 0 < n1 < n60 < 0.06 * 60 * 1920 * 1080 * (12 + 4 + 8)
    assert n60 < 49 * n1  # frames beyond the 48 of a launch add only their 128-byte header
    assert b.exw_workspace_bytes(b.OP_WARP_BACKWARD, 64, 64) >= 64 * 64 * 8
    assert b.exw_workspace_bytes(b.OP_EXTRAPOLATE, 0, 10) == 0
    assert b.exw_workspace_bytes(b.OP_EXTRAPOLATE, 16385, 10) == 0
    assert b.exw_workspace_bytes(b.OP_EXTRAPOLATE, 64, 64, b.F32, 1, 4) == 0


def test_invalid_arguments_rejected_on_host(lib):
    # null / misaligned pointers and bad sizes return EXW_ERR_INVALID_ARG (1) before touching the GPU
    aligned = 4096
    assert lib.exw_splat_motion(None, None, 8, 8, 1, 4, None, None) == 1
    assert lib.exw_splat_motion(aligned, aligned, 8, 8, 1, 4, aligned + 4, None) == 1   # misaligned keys
    assert lib.exw_splat_motion(aligned, aligned, 0, 8, 1, 4, aligned, None) == 1       # W = 0
    assert lib.exw_splat_motion(aligned, aligned, 8, 8, 5, 4, aligned, None) == 1       # k > denom
    assert lib.exw_splat_motion(aligned, aligned, 8, 8, 1, 3, aligned, None) == 1       # denom not a power of 2
    assert lib.exw_splat_motion(aligned, aligned, 8, 8, 1, 128, aligned, None) == 1     # denom > 64
    assert lib.exw_warp(aligned, 7, aligned, aligned, aligned, 8, 8, 1, 4, aligned, aligned, None) == 1  # dtype
    assert lib.exw_extrapolate(None, 1, 3, 0, None, aligned, 1 << 20, None) == 1
    assert lib.exw_fill_holes(aligned, 0, aligned, 8, 8, aligned, 16, None) == 5        # workspace too small


def test_extrapolate_descriptor_checks(lib):
    from paper_2307_12607_gb300 import _lib
    fr = (_lib.ExwFrame * 2)()
    fr[0] = _lib.ExwFrame(4096, 8192, 12288, 64, 64, 0)
    fr[1] = _lib.ExwFrame(4096, 8192, 12288, 64, 32, 0)      # size differs from frame 0
    outs = (_lib.ExwFrameOut * 6)()
    for i in range(6):
        outs[i] = _lib.ExwFrameOut(16384, 20480)
    ws = 1 << 20
    r = lib.exw_extrapolate(ctypes.cast(fr, ctypes.c_void_p), 2, 3, 0, ctypes.cast(outs, ctypes.c_void_p), 4096, ws,
                            None)
    assert r == 1
    r = lib.exw_extrapolate(ctypes.cast(fr, ctypes.c_void_p), 1, 4, 0, ctypes.cast(outs, ctypes.c_void_p), 4096, ws,
                            None)
    assert r == 1                                              # nfrac > 3
    r = lib.exw_extrapolate(ctypes.cast(fr, ctypes.c_void_p), 1, 3, 8, ctypes.cast(outs, ctypes.c_void_p), 4096, ws,
                            None)
    assert r == 1                                              # unknown flag


def test_extrapolate_host_argument_checks(lib):
    # null descriptor arrays, a negative chunk, nfrac out of range and mismatched host descriptors are refused on the
    # host, before any copy is queued
    from paper_2307_12607_gb300 import _lib
    fh = (_lib.ExwFrame * 2)()
    fd = (_lib.ExwFrame * 2)()
    for f in range(2):
        fd[f] = _lib.ExwFrame(4096, 8192, 12288, 64, 64, 0)
        fh[f] = _lib.ExwFrame(4096, 8192, 12288, 64, 64 if f == 0 else 32, 0)   # frame 1's size differs
    oh = (_lib.ExwFrameOut * 6)()
    for i in range(6):
        oh[i] = _lib.ExwFrameOut(16384, 20480)
    P = lambda a: ctypes.cast(a, ctypes.c_void_p)
    assert lib.exw_extrapolate_host(None, P(fd), 2, 3, 0, P(oh), None, 2, 4096, 1 << 20, None) == 1
    assert lib.exw_extrapolate_host(P(fh), P(fd), 2, 3, 0, None, None, 2, 4096, 1 << 20, None) == 1
    assert lib.exw_extrapolate_host(P(fh), P(fd), 2, 3, 0, P(oh), None, -1, 4096, 1 << 20, None) == 1
    assert lib.exw_extrapolate_host(P(fh), P(fd), 1, 4, 0, P(oh), None, 2, 4096, 1 << 20, None) == 1
    assert lib.exw_extrapolate_host(P(fh), P(fd), 2, 3, 0, P(oh), None, 2, 4096, 1 << 20, None) == 1


def test_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    from paper_2307_12607_gb300 import binding as b
    d = torch.ones(8, 8)
    m = torch.zeros(2, 8, 8)
    with pytest.raises(ValueError, match="CUDA"):
        b.exw_splat_motion(d, m, 1)


def test_recursive_and_statistics_argument_checks(lib):
    # exw_carry_motion, exw_mv_variance, exw_color_mse, exw_ssim: null / misaligned pointers, bad sizes and colour
    # types are refused with EXW_ERR_INVALID_ARG (1), a short or misaligned workspace with EXW_ERR_WORKSPACE (5)
    a = 4096
    big = 1 << 20
    assert lib.exw_carry_motion(None, a, a, a, 8, 8, a, a, None) == 1
    assert lib.exw_carry_motion(a + 4, a, a, a, 8, 8, a, a, None) == 1           # keys not 8-byte aligned
    assert lib.exw_carry_motion(a, a, a, a, 0, 8, a, a, None) == 1               # W = 0
    assert lib.exw_carry_motion(a, a, a, a, 8, 8, a + 2, a, None) == 1           # depth_out misaligned
    assert lib.exw_mv_variance(None, 8, 8, a, a, big, None) == 1
    assert lib.exw_mv_variance(a, 8, 8, a + 4, a, big, None) == 1                # out not 8-byte aligned
    assert lib.exw_mv_variance(a, 8, 16385, a, a, big, None) == 1                # H too large
    assert lib.exw_mv_variance(a, 8, 8, a, a, 16, None) == 5                     # workspace too small
    assert lib.exw_mv_variance(a, 8, 8, a, a + 8, big, None) == 5                # workspace misaligned
    assert lib.exw_color_mse(a, a, 7, 8, 8, a, a, big, None) == 1                # unknown colour type
    assert lib.exw_color_mse(a, a + 2, 0, 8, 8, a, a, big, None) == 1            # FP32 b misaligned
    assert lib.exw_color_mse(a, a, 1, 8, 8, a, None, big, None) == 5             # no workspace
    assert lib.exw_ssim(a, a, 0, 10, 64, a, a, big, None) == 1                   # narrower than the window
    assert lib.exw_ssim(a, a, 0, 64, 10, a, a, big, None) == 1                   # lower than the window
    assert lib.exw_ssim(a, a + 1, 1, 64, 64, a, a, big, None) == 1               # FP16 b misaligned
    assert lib.exw_ssim(a, a, 0, 64, 64, a, a, 8, None) == 5


def test_psnr_and_recursive_warp_argument_checks(lib):
    # exw_psnr follows exw_color_mse's rules; exw_warp_recursive refuses bad steps, flags, sizes and descriptors
    # with EXW_ERR_INVALID_ARG (1) and a short workspace with EXW_ERR_WORKSPACE (5), before any launch
    from paper_2307_12607_gb300 import _lib, binding as b
    a = 4096
    big = 1 << 26
    assert lib.exw_psnr(a, a, 7, 8, 8, a, a, big, None) == 1                     # unknown colour type
    assert lib.exw_psnr(a, a, 0, 8, 8, a + 4, a, big, None) == 1                 # out not 8-byte aligned
    assert lib.exw_psnr(a, a, 0, 8, 8, a, a, 8, None) == 5                       # workspace too small
    outs = (_lib.ExwFrameOut * 3)()
    for i in range(3):
        outs[i] = _lib.ExwFrameOut(16384, 20480)
    P = lambda x: ctypes.cast(x, ctypes.c_void_p)
    rec = lib.exw_warp_recursive
    assert rec(a, 0, a, a, 64, 64, 0, 0, P(outs), a, big, None) == 1             # no step
    assert rec(a, 0, a, a, 64, 64, 65, 0, P(outs), a, big, None) == 1            # too many steps
    assert rec(a, 0, a, a, 64, 64, 3, 2, P(outs), a, big, None) == 1             # only EXW_FLAG_NO_FILL is known
    assert rec(a, 0, a, a, 64, 64, 3, 0, None, a, big, None) == 1                # no descriptors
    assert rec(a + 2, 0, a, a, 64, 64, 3, 0, P(outs), a, big, None) == 1         # FP32 colour misaligned
    outs[1].mask = None
    assert rec(a, 0, a, a, 64, 64, 3, 0, P(outs), a, big, None) == 1            # a step without a mask buffer
    outs[1].mask = 20480
    need = b.exw_workspace_bytes(b.OP_WARP_RECURSIVE, 64, 64)
    assert need >= 64 * 64 * (8 + 2 * 12)                                        # keys + two carried fields
    assert rec(a, 0, a, a, 64, 64, 3, 0, P(outs), a, need - 1, None) == 5


def test_backward_bounds_and_fill_argument_checks(lib):
    a = 4096
    big = 1 << 20
    bwd = lib.exw_warp_backward
    assert bwd(a, a, 0, a, a, a, 8, 8, 1, 3, a, a, a, big, None) == 1            # denom not a power of 2
    assert bwd(a, a, 0, a, a, a, 8, 8, 5, 4, a, a, a, big, None) == 1            # k > denom
    assert bwd(a, a, 0, a, a, a + 4, 8, 8, 1, 4, a, a, a, big, None) == 1        # keys misaligned
    assert bwd(a, a, 0, a, a, a, 8, 8, 1, 4, None, a, a, big, None) == 1         # no grad_color
    assert bwd(a, a, 0, a, a, None, 8, 8, 1, 4, a, a, a, 16, None) == 5          # keys recomputed: workspace short
    assert lib.exw_l2_loss_grad(a, a, 0, a, 8, 8, a, None, None) == 1            # no loss scalar
    assert lib.exw_l2_loss_grad(a, a, 3, a, 8, 8, a, a, None) == 1               # unknown colour type
    assert lib.exw_motion_bounds(a, a, 8, 8, a + 4, a, a, big, None) == 1        # tile bounds not 16-byte aligned
    assert lib.exw_motion_bounds(a, a, 8, 8, None, None, a, big, None) == 1      # no frame bounds
    assert lib.exw_motion_bounds(a, a, 8, 8, None, a, a, 64, None) == 5
    assert lib.exw_fill_holes_static(a, 0, a, 16385, 8, None) == 1
    assert lib.exw_fill_holes_static(a + 2, 0, a, 8, 8, None) == 1               # FP32 colour misaligned
    assert lib.exw_fill_holes_static(a, 1, None, 8, 8, None) == 1                # no mask
    assert lib.exw_fill_holes_static(a, 0, a, 16384, 16384, None) == 5           # 262,144 fill tiles > 16,384
    assert lib.exw_device_status(a + 8, None) == 1


def _streams(sizes, cdt=0):
    from paper_2307_12607_gb300 import _lib
    d = (_lib.ExwStreamDesc * len(sizes))()
    for i, (W, H) in enumerate(sizes):
        d[i].src = _lib.ExwFrame(4096, 8192, 12288, W, H, cdt)
        for j in range(3):
            d[i].out[j] = _lib.ExwFrameOut(16384, 20480)
    return d


def test_batched_argument_checks_and_workspace(lib):
    P = lambda x: ctypes.cast(x, ctypes.c_void_p)
    d = _streams([(64, 64), (128, 72)])
    ws = 1 << 24
    assert lib.exw_extrapolate_batched(None, 1, 3, 0, 4096, ws, None, None) == 1
    assert lib.exw_extrapolate_batched(P(d), 0, 3, 0, 4096, ws, None, None) == 1
    assert lib.exw_extrapolate_batched(P(d), 2, 4, 0, 4096, ws, None, None) == 1          # nfrac > 3
    assert lib.exw_extrapolate_batched(P(d), 2, 3, 1 << 7, 4096, ws, None, None) == 1     # unknown flag
    many = _streams([(64, 64)] * 49)
    assert lib.exw_extrapolate_batched(P(many), 49, 3, 0, 4096, ws, None, None) == 2      # > 48 streams
    bad = _streams([(64, 64), (128, 72)])
    bad[1].src.cdt = 7
    assert lib.exw_extrapolate_batched(P(bad), 2, 3, 0, 4096, ws, None, None) == 1
    bad = _streams([(64, 64), (128, 72)])
    bad[0].out[2].mask = None
    assert lib.exw_extrapolate_batched(P(bad), 2, 3, 0, 4096, ws, None, None) == 1
    bad = _streams([(64, 64)], cdt=1)
    bad[0].src.color = 4097                                                            # FP16 colour misaligned
    assert lib.exw_extrapolate_batched(P(bad), 1, 3, 0, 4096, ws, None, None) == 1
    # workspace: zero for bad descriptors, positive and growing with the streams and fractions otherwise
    wb = lib.exw_batched_workspace_bytes
    assert wb(None, 1, 3) == 0 and wb(P(d), 0, 3) == 0 and wb(P(d), 2, 0) == 0
    assert wb(P(_streams([(0, 64)])), 1, 3) == 0
    one, two = wb(P(d), 1, 3), wb(P(d), 2, 3)
    assert 0 < one < two
    assert wb(P(d), 2, 1) <= two
    assert wb(P(_streams([(64, 64)] * 49)), 49, 3) == 0


def test_tuner_lifecycle_on_host(lib):
    t = lib.exw_tuner_create()
    assert t
    try:
        assert lib.exw_tuner_fix(t, 2, 1, 1) == 1          # only window shapes 0 and 1
        assert lib.exw_tuner_fix(t, 0, 0, 1) == 1          # queue distance >= 1
        assert lib.exw_tuner_fix(t, 1, 2, 2) == 1          # pair is 0 or 1
        assert lib.exw_tuner_fix(None, 0, 1, 1) == 1
        assert lib.exw_tuner_fix(t, 1, 2, 0) == 0
        buf = ctypes.create_string_buffer(64)
        assert lib.exw_tuner_report(t, buf, 64) == 1 and buf.value == b""       # nothing tuned yet
        assert lib.exw_tuner_report(None, None, 0) == 1
    finally:
        lib.exw_tuner_destroy(t)
    lib.exw_tuner_destroy(None)                                                     # deleting NULL is a no-op
