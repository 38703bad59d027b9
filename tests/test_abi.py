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
    # per frame: a header; per frame in flight (at most 48 per launch): bounds, plans, pyramid nodes -- a few
    # percent of the frames' own bytes
    assert 0 < n1 < n60 < 0.03 * 60 * 1920 * 1080 * (12 + 4 + 8)
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
