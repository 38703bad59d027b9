"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same seeded inputs.

Bars: splat keys, hole masks and motion bounds bit-exact; colour within 2e-6 absolute for float32 storage and 1e-3
for float16 storage (values in [0, 1]); gradients within 1e-5 absolute + 1e-4 relative.  The float32 colour bar
covers the float32 gather (a few ulp of a value <= 1) and the float32 pull-push pyramid (one rounding per level
and at most 14 levels), against the oracle's float64.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2307_12607_gb300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {torch.float32: 2e-6, torch.float16: 1e-3}
NPDT = {torch.float32: np.float32, torch.float16: np.float16}


@pytest.fixture(scope="module")
def b():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the gpu-marked tests")
    from paper_2307_12607_gb300 import build, binding
    build.build()
    return binding


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def keys_np(t):
    return t.cpu().numpy().view(np.uint64)


def frame_case(name):
    """Named small inputs: (colour float32 [3][H][W], depth, mv)."""
    kind, W, H, seed = name
    if kind == "scene":
        s = scenes.make_scene(W, H, seed, 6, vmax=6.0, pan_max=2.0, sliver_fraction=0.2)
        return scenes.render(s, 0.0)
    if kind == "ties":
        return scenes.random_frame(W, H, seed, depth_levels=2, mv_scale=3.0, quarter_grid=True, invalid_fraction=0.05)
    if kind == "invalid":
        return scenes.random_frame(W, H, seed, depth_levels=0, mv_scale=6.0, invalid_fraction=0.3)
    return scenes.random_frame(W, H, seed, mv_scale=4.0)


CASES = [("rand", 8, 8, 1), ("ties", 37, 29, 2), ("invalid", 64, 64, 3), ("rand", 1, 1, 4), ("rand", 1, 50, 5),
         ("rand", 50, 1, 6), ("scene", 257, 131, 7), ("ties", 100, 70, 8), ("scene", 640, 360, 9)]


def as_storage(color, dtype):
    return color.astype(NPDT[dtype])


# ------------------------------------------------------------------------------------------------------------
# (a) splat, (a0) bounds
# ------------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("case", CASES)
def test_splat_keys_bit_exact(b, case):
    _, depth, mv = frame_case(case)
    d, m = dev(depth), dev(mv)
    for k, denom in [(0, 4), (1, 4), (2, 4), (3, 4), (4, 4), (1, 2), (3, 8), (5, 8), (37, 64), (1, 1)]:
        got = keys_np(b.exw_splat_motion(d, m, k, denom))
        want = oracle.splat(depth, mv, k, denom)
        np.testing.assert_array_equal(got, want, err_msg=f"{case} k={k}/{denom}")


@pytest.mark.parametrize("case", CASES)
def test_motion_bounds_bit_exact(b, case):
    _, depth, mv = frame_case(case)
    mv = mv.copy()
    mv[0].flat[0] = 1e7   # clamped
    tiles, frame = b.exw_motion_bounds(dev(depth), dev(mv))
    wt, wf = oracle.motion_bounds(depth, mv, 8)
    np.testing.assert_array_equal(tiles.cpu().numpy().view(np.uint32), wt.view(np.uint32))
    np.testing.assert_array_equal(frame.cpu().numpy().view(np.uint32), wf.view(np.uint32))


# ------------------------------------------------------------------------------------------------------------
# (b) staged warp
# ------------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("case", CASES)
def test_warp_matches_oracle(b, case, dtype):
    color, depth, mv = frame_case(case)
    cs = as_storage(color, dtype)
    c, d, m = dev(cs), dev(depth), dev(mv)
    for k in (1, 2, 3):
        keys = b.exw_splat_motion(d, m, k, 4)
        out, mask = b.exw_warp(c, d, m, keys, k, 4)
        wo, wm = oracle.warp(cs.astype(np.float64), depth, mv, keys_np(keys), k, 4)
        np.testing.assert_array_equal(mask.cpu().numpy(), wm, err_msg=f"{case} k={k}")
        got = out.float().cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got, wo, rtol=0, atol=TOL[dtype], err_msg=f"{case} k={k}")
        assert np.all(got[:, wm != 0] == 0.0)


# ------------------------------------------------------------------------------------------------------------
# (c) staged fill
# ------------------------------------------------------------------------------------------------------------

def fill_inputs(kind, W, H, seed):
    rng = np.random.default_rng(seed)
    color = rng.uniform(size=(3, H, W)).astype(np.float32)
    if kind == "none":
        mask = np.zeros((H, W), np.uint8)
    elif kind == "all":
        mask = np.ones((H, W), np.uint8)
    elif kind == "single":
        mask = np.ones((H, W), np.uint8)
        mask[rng.integers(H), rng.integers(W)] = 0
    elif kind == "blobs":           # large holes: whole 32x32 tiles without a valid pixel
        mask = np.zeros((H, W), np.uint8)
        for _ in range(6):
            y, x = rng.integers(H), rng.integers(W)
            mask[y:y + rng.integers(20, 120), x:x + rng.integers(20, 120)] = 2
    else:
        mask = (rng.uniform(size=(H, W)) < 0.4).astype(np.uint8)
    color[:, mask != 0] = 0.0
    return color, mask


FILL_CASES = [("none", 40, 30, 1), ("all", 70, 33, 2), ("single", 100, 90, 3), ("blobs", 300, 200, 4),
              ("random", 1, 1, 5), ("random", 33, 33, 6), ("blobs", 1000, 37, 7), ("single", 5, 700, 8),
              ("blobs", 1920, 1080, 9)]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("case", FILL_CASES)
def test_fill_matches_oracle(b, case, dtype):
    color, mask = fill_inputs(*case)
    cs = as_storage(color, dtype)
    c = dev(cs)
    b.exw_fill_holes(c, dev(mask))
    got = c.float().cpu().numpy().astype(np.float64)
    want = oracle.fill_holes(cs.astype(np.float64), mask)
    np.testing.assert_allclose(got, want, rtol=0, atol=TOL[dtype], err_msg=str(case))
    valid = mask == 0
    np.testing.assert_array_equal(got[:, valid], cs.astype(np.float64)[:, valid])   # valid pixels untouched


# ------------------------------------------------------------------------------------------------------------
# fused (a0)+(a)+(b)+(c)
# ------------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("fill", [True, False])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("case", CASES)
def test_extrapolate_matches_oracle_and_staged(b, case, dtype, fill):
    color, depth, mv = frame_case(case)
    cs = as_storage(color, dtype)
    c, d, m = dev(cs), dev(depth), dev(mv)
    out, mask = b.exw_extrapolate(c, d, m, nfrac=3, fill=fill)
    ref = oracle.extrapolate(cs.astype(np.float64), depth, mv, 3, storage=NPDT[dtype], fill=fill)
    for j, (wo, wm, wk) in enumerate(ref):
        np.testing.assert_array_equal(mask[j].cpu().numpy(), wm, err_msg=f"{case} k={j + 1}")
        np.testing.assert_allclose(out[j].float().cpu().numpy().astype(np.float64), wo, rtol=0, atol=TOL[dtype],
                                   err_msg=f"{case} k={j + 1}")
        # the fused pass is bit-identical to the staged entry points
        keys = b.exw_splat_motion(d, m, j + 1, 4)
        np.testing.assert_array_equal(keys_np(keys), wk)
        so, sm = b.exw_warp(c, d, m, keys, j + 1, 4)
        if fill:
            b.exw_fill_holes(so, sm)
        assert torch.equal(sm, mask[j])
        assert torch.equal(so.view(torch.int16 if dtype == torch.float16 else torch.int32),
                           out[j].view(torch.int16 if dtype == torch.float16 else torch.int32))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("case", [("scene", 640, 360, 9), ("scene", 256, 128, 15), ("ties", 96, 64, 16),
                                  ("invalid", 64, 64, 3)])
def test_tma_and_plain_paths_identical(b, case, dtype):
    color, depth, mv = frame_case(case)
    cs = as_storage(color, dtype)
    c, d, m = dev(cs), dev(depth), dev(mv)
    for fill in (True, False):
        o1, m1 = b.exw_extrapolate(c, d, m, nfrac=3, fill=fill, tma=True)
        o2, m2 = b.exw_extrapolate(c, d, m, nfrac=3, fill=fill, tma=False)
        assert torch.equal(m1, m2)
        iv = torch.int16 if dtype == torch.float16 else torch.int32
        assert torch.equal(o1.view(iv), o2.view(iv))


def test_tma_staging_modes_cover_all_tiles(b):
    # a fast pixel forces the widest candidate search; wide tiles fall back per fraction or to global memory
    color, depth, mv = scenes.random_frame(320, 192, 5, mv_scale=1.0)
    mv[:, 50:60, 100:120] = np.float32(60.0)
    c, d, m = dev(color), dev(depth), dev(mv)
    ws = b.workspace(b.exw_workspace_bytes(b.OP_EXTRAPOLATE, 320, 192, b.F32, 1, 3), c.device)
    out, mask = b.exw_extrapolate(c, d, m, ws=ws)
    st = b.frame_stats(ws)
    assert sum(v for k, v in st.items() if k.startswith("tiles_") and k != "tiles_without_valid_pixel") == 10 * 6
    assert st["tiles_window_all"] > 0 and st["tiles_global"] + st["tiles_window_each"] > 0
    ref = oracle.extrapolate(color.astype(np.float64), depth, mv, 3)
    for j, (wo, wm, _) in enumerate(ref):
        np.testing.assert_array_equal(mask[j].cpu().numpy(), wm)
        np.testing.assert_allclose(out[j].cpu().numpy(), wo, rtol=0, atol=2e-6)


@pytest.mark.parametrize("dtype", [np.float32, np.float16])
def test_fast_motion_mixed_staging(b, dtype):
    # motion up to 16 pixels in every direction: the sources of most tiles overflow a staging window and are read
    # from global memory; a slow band keeps ordinary windows, a fast block lands far from its sources
    W, H = 264, 200
    color, depth, mv = scenes.random_frame(W, H, 21, mv_scale=16.0)
    mv[:, :40, :] *= 0.125
    mv[:, 60:80, 40:72] = np.float32(70.0)
    color = color.astype(dtype)
    c, d, m = dev(color), dev(depth), dev(mv)
    ws = b.workspace(b.exw_workspace_bytes(b.OP_EXTRAPOLATE, W, H, b.F16 if dtype == np.float16 else b.F32, 1, 3),
                     c.device)
    tol = 1e-3 if dtype == np.float16 else 2e-6
    iv = torch.int16 if dtype == np.float16 else torch.int32
    for fill in (True, False):
        out, mask = b.exw_extrapolate(c, d, m, fill=fill, ws=ws)
        st = b.frame_stats(ws)
        assert st["tiles_window_all"] > 0 and st["tiles_global"] + st["tiles_window_each"] > 0
        out2, mask2 = b.exw_extrapolate(c, d, m, fill=fill, tma=False)
        assert torch.equal(mask, mask2) and torch.equal(out.view(iv), out2.view(iv))
        ref = oracle.extrapolate(color.astype(np.float64), depth, mv, 3, fill=fill, storage=dtype)
        for j, (wo, wm, _) in enumerate(ref):
            np.testing.assert_array_equal(mask[j].cpu().numpy(), wm)
            np.testing.assert_allclose(out[j].cpu().numpy().astype(np.float64), wo, rtol=0, atol=tol)


@pytest.mark.parametrize("pan", [(1.3, -0.7), (-2.6, 0.0), (0.0, 1.9), (0.5, 0.5), (4.0, -8.0), (0.0, 0.0),
                                 (-0.25, -3.75)])
@pytest.mark.parametrize("dtype", [np.float32, np.float16])
def test_smooth_tiles_every_residual_sign(b, pan, dtype):
    # a slanted but smooth surface (depth within 1/32 over each tile's sources) under one motion: interior tiles are
    # pure bilinear resamplings; the pans give every combination of residual signs, including none
    W, H = 288, 160
    rng = np.random.default_rng(11)
    color = rng.uniform(size=(3, H, W)).astype(np.float32).astype(dtype)
    yy, xx = np.mgrid[0:H, 0:W]
    depth = (40.0 + 0.002 * xx + 0.003 * yy).astype(np.float32)
    mv = np.empty((2, H, W), np.float32)
    mv[0], mv[1] = pan
    c, d, m = dev(color), dev(depth), dev(mv)
    ws = b.workspace(b.exw_workspace_bytes(b.OP_EXTRAPOLATE, W, H, b.F16 if dtype == np.float16 else b.F32, 1, 3),
                     c.device)
    for fill in (True, False):
        out, mask = b.exw_extrapolate(c, d, m, fill=fill, ws=ws)
        assert b.frame_stats(ws)["tiles_smooth"] > 0
        out2, mask2 = b.exw_extrapolate(c, d, m, fill=fill, tma=False)
        assert torch.equal(mask, mask2)
        iv = torch.int16 if dtype == np.float16 else torch.int32
        assert torch.equal(out.view(iv), out2.view(iv))
        ref = oracle.extrapolate(color.astype(np.float64), depth, mv, 3, fill=fill, storage=dtype)
        tol = 1e-3 if dtype == np.float16 else 2e-6
        for j, (wo, wm, _) in enumerate(ref):
            np.testing.assert_array_equal(mask[j].cpu().numpy(), wm)
            np.testing.assert_allclose(out[j].cpu().numpy().astype(np.float64), wo, rtol=0, atol=tol)


@pytest.mark.parametrize("dtype", [np.float32, np.float16])
@pytest.mark.parametrize("hole", [(128, 256, 64, 160), (0, 384, 0, 256), (32, 480, 96, 168)])
@pytest.mark.parametrize("motion", ["uniform", "varying"])
def test_lazy_nodes_under_large_holes(b, dtype, hole, motion):
    # tiles without a hole do not build their pyramid; when a fraction has tiles without any valid pixel, the coarse
    # pass computes the level-5 nodes it needs -- up to most of the frame when the hole covers three quarters of it:
    # a smooth tile's (one motion over a smooth surface) from its source colour, another tile's (a motion that
    # varies from pixel to pixel: one-window splat tiles) from its stored outputs -- and the fill must equal the
    # staged fill bit for bit
    W, H = 512, 256
    rng = np.random.default_rng(sum(hole))
    color = rng.uniform(size=(3, H, W)).astype(np.float32).astype(dtype)
    yy, xx = np.mgrid[0:H, 0:W]
    depth = (40.0 + 0.002 * xx + 0.003 * yy).astype(np.float32)
    x0, x1, y0, y1 = hole
    depth[y0:y1, x0:x1] = np.nan                      # sources that never land: whole tiles without a valid pixel
    mv = np.empty((2, H, W), np.float32)
    if motion == "uniform":
        mv[0], mv[1] = 1.3, -0.7
    else:
        mv[0], mv[1] = 1.3 + 0.002 * xx, -0.7 + 0.001 * yy
    c, d, m = dev(color), dev(depth), dev(mv)
    ws = b.workspace(b.exw_workspace_bytes(b.OP_EXTRAPOLATE, W, H, b.F16 if dtype == np.float16 else b.F32, 1, 3),
                     c.device)
    out, mask = b.exw_extrapolate(c, d, m, fill=True, ws=ws)
    st = b.frame_stats(ws)
    lazy = st["lazy_nodes_computed"]
    assert min(st["tiles_without_valid_pixel"]) > 0 and lazy["from_outputs"] > 0
    if motion == "uniform":
        assert st["tiles_smooth"] > 0 and st["tiles_uniform"] > 0
        if hole == (0, 384, 0, 256):  # the ancestors of the hole over three quarters of the frame hold smooth tiles
            assert lazy["smooth"] > 0
    else:
        assert st["tiles_window_all"] > 0
    iv = torch.int16 if dtype == np.float16 else torch.int32
    for j in range(3):
        keys = b.exw_splat_motion(d, m, j + 1, 4)
        so, sm = b.exw_warp(c, d, m, keys, j + 1, 4)
        b.exw_fill_holes(so, sm)
        assert torch.equal(sm, mask[j]) and torch.equal(so.view(iv), out[j].view(iv)), f"P_{j + 1}"
    ref = oracle.extrapolate(color.astype(np.float64), depth, mv, 3, storage=dtype)
    tol = 1e-3 if dtype == np.float16 else 2e-6
    for j, (wo, wm, _) in enumerate(ref):
        np.testing.assert_array_equal(mask[j].cpu().numpy(), wm)
        np.testing.assert_allclose(out[j].cpu().numpy().astype(np.float64), wo, rtol=0, atol=tol)


def test_uniform_tiles_with_foreign_motion_inside_their_source(b):
    # a uniformly panning background holds a small object moving so fast that it lands far away: tiles whose
    # candidate sources all pan are uniform, yet their source window contains the object's pixels, which must not
    # be taken as winners
    W, H = 256, 128
    color = np.random.default_rng(7).uniform(size=(3, H, W)).astype(np.float32)
    depth = np.full((H, W), 50.0, np.float32)
    mv = np.zeros((2, H, W), np.float32)
    mv[0] = 2.0
    depth[40:60, 100:120] = 10.0
    mv[0, 40:60, 100:120] = 40.0
    mv[1, 40:60, 100:120] = -1.5
    depth[5, 5] = np.nan                       # an invalid source pixel inside a uniform tile
    mv[0, 90, 200] = -2.0                      # and one with a different (slow) motion
    c, d, m = dev(color), dev(depth), dev(mv)
    ws = b.workspace(b.exw_workspace_bytes(b.OP_EXTRAPOLATE, W, H, b.F32, 1, 3), c.device)
    for fill in (True, False):
        out, mask = b.exw_extrapolate(c, d, m, fill=fill, ws=ws)
        st = b.frame_stats(ws)
        assert st["tiles_uniform"] > 0 and st["tiles_smooth"] > 0
        ref = oracle.extrapolate(color.astype(np.float64), depth, mv, 3, fill=fill)
        for j, (wo, wm, _) in enumerate(ref):
            np.testing.assert_array_equal(mask[j].cpu().numpy(), wm)
            np.testing.assert_allclose(out[j].cpu().numpy(), wo, rtol=0, atol=2e-6)
        o2, m2 = b.exw_extrapolate(c, d, m, fill=fill, tma=False)
        assert torch.equal(m2, mask) and torch.equal(o2.view(torch.int32), out.view(torch.int32))


@pytest.mark.parametrize("direct", [False, True])
@pytest.mark.parametrize("chunk", [2, 3, 8])
def test_host_buffers_match_device_path(b, chunk, direct):
    # 7 frames in host memory, chunks of 2 or 3 (a ragged last chunk) or one chunk: copies in, work and copies out
    # overlap on three streams; the results are the device path's, bit for bit
    frames = [frame_case(("scene", 96, 64, 20 + s)) for s in range(7)]
    hc = torch.from_numpy(np.stack([f[0] for f in frames]).astype(np.float16)).pin_memory()
    hd = torch.from_numpy(np.stack([f[1] for f in frames])).pin_memory()
    hm = torch.from_numpy(np.stack([f[2] for f in frames])).pin_memory()
    out, mask = b.exw_extrapolate_host(hc, hd, hm, nfrac=3, chunk=chunk, direct=direct)
    torch.cuda.synchronize()
    o1, k1 = b.exw_extrapolate(hc.cuda(), hd.cuda(), hm.cuda(), nfrac=3)
    assert torch.equal(mask, k1.cpu()) and torch.equal(out.view(torch.int16), o1.cpu().view(torch.int16))


def test_extrapolate_fewer_fractions_and_sequences(b):
    frames = [frame_case(("scene", 96, 64, s)) for s in range(4)]
    c = dev(np.stack([f[0] for f in frames]))
    d = dev(np.stack([f[1] for f in frames]))
    m = dev(np.stack([f[2] for f in frames]))
    for nfrac in (1, 2, 3):
        out, mask = b.exw_extrapolate(c, d, m, nfrac=nfrac)
        assert out.shape == (4, nfrac, 3, 64, 96)
        for f in range(4):
            single, smask = b.exw_extrapolate(c[f], d[f], m[f], nfrac=nfrac)
            assert torch.equal(single, out[f]) and torch.equal(smask, mask[f])


# ------------------------------------------------------------------------------------------------------------
# edge cases
# ------------------------------------------------------------------------------------------------------------

def test_no_valid_source_pixel(b):
    color, depth, mv = scenes.random_frame(70, 45, 1)
    depth[...] = np.nan
    out, mask = b.exw_extrapolate(dev(color), dev(depth), dev(mv))
    assert torch.all(mask == b.MASK_EMPTY)
    assert torch.all(out == 0)


def test_huge_and_nonfinite_motion_never_lands(b):
    color, depth, mv = scenes.random_frame(64, 40, 2, mv_scale=2.0)
    mv[0, :10] = 1e30
    mv[1, 10:20] = -3e38
    mv[0, 20:25] = np.nan
    mv[1, 25:30] = np.inf
    c, d, m = dev(color), dev(depth), dev(mv)
    out, mask = b.exw_extrapolate(c, d, m)
    ref = oracle.extrapolate(color.astype(np.float64), depth, mv, 3)
    for j, (wo, wm, wk) in enumerate(ref):
        np.testing.assert_array_equal(mask[j].cpu().numpy(), wm)
        np.testing.assert_allclose(out[j].cpu().numpy(), wo, rtol=0, atol=2e-6)


def test_max_width_row(b):
    W, H = 16384, 2
    color, depth, mv = scenes.random_frame(W, H, 3, mv_scale=40.0)
    out, mask = b.exw_extrapolate(dev(color), dev(depth), dev(mv))
    ref = oracle.extrapolate(color.astype(np.float64), depth, mv, 3)
    for j, (wo, wm, _) in enumerate(ref):
        np.testing.assert_array_equal(mask[j].cpu().numpy(), wm)
        np.testing.assert_allclose(out[j].cpu().numpy(), wo, rtol=0, atol=2e-6)


def test_large_motion_search_window(b):
    # one fast pixel widens the frame bounds; every tile's candidate scan must still find the right sources
    color, depth, mv = scenes.random_frame(300, 200, 4, mv_scale=1.0)
    mv[:, 100, 150] = (250.0, -170.0)
    out, mask = b.exw_extrapolate(dev(color), dev(depth), dev(mv), fill=False)
    ref = oracle.extrapolate(color.astype(np.float64), depth, mv, 3, fill=False)
    for j, (wo, wm, _) in enumerate(ref):
        np.testing.assert_array_equal(mask[j].cpu().numpy(), wm)
        np.testing.assert_allclose(out[j].cpu().numpy(), wo, rtol=0, atol=2e-6)


def test_invalid_arguments_raise(b):
    d = torch.ones(8, 8, device="cuda")
    m = torch.zeros(2, 8, 8, device="cuda")
    with pytest.raises(b.ExwError) as e:
        b.exw_splat_motion(d, m, 5, 4)
    assert e.value.status == 1
    with pytest.raises(b.ExwError):
        b.exw_splat_motion(d, m, 1, 3)


# ------------------------------------------------------------------------------------------------------------
# adjoint
# ------------------------------------------------------------------------------------------------------------

def grad_close(got, want):
    got = got.astype(np.float64)
    err = np.abs(got - want)
    bound = 1e-5 + 1e-4 * np.abs(want)
    assert np.all(err <= bound), f"max excess {np.max(err - bound)} at {np.unravel_index(np.argmax(err - bound), err.shape)}"


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("case", [("ties", 37, 29, 11), ("scene", 257, 131, 12), ("rand", 64, 48, 13),
                                  ("invalid", 40, 40, 14)])
def test_backward_matches_oracle(b, case, dtype):
    color, depth, mv = frame_case(case)
    cs = as_storage(color, dtype)
    c, d, m = dev(cs), dev(depth), dev(mv)
    rng = np.random.default_rng(case[3])
    H, W = depth.shape
    for k in (1, 2, 3):
        g = rng.standard_normal((3, H, W)).astype(np.float32)
        keys = b.exw_splat_motion(d, m, k, 4)
        gc, gm = b.exw_warp_backward(dev(g), c, d, m, keys, k, 4)
        wc, wmv = oracle.warp_backward(g, cs.astype(np.float64), depth, mv, keys_np(keys), k, 4)
        grad_close(gc.cpu().numpy(), wc)
        grad_close(gm.cpu().numpy(), wmv)
        # recomputed keys (checkpointing) give bit-identical gradients; accumulation adds
        gc2, gm2 = b.exw_warp_backward(dev(g), c, d, m, None, k, 4)
        assert torch.equal(gc2, gc) and torch.equal(gm2, gm)
        b.exw_warp_backward(dev(g), c, d, m, keys, k, 4, grad_color=gc2, grad_mv=gm2)
        assert torch.equal(gc2, 2 * gc) and torch.equal(gm2, 2 * gm)


def test_autograd_function_and_loss(b):
    from paper_2307_12607_gb300 import autograd
    color, depth, mv = frame_case(("scene", 160, 96, 21))
    H, W = depth.shape
    target = np.random.default_rng(0).uniform(size=(3, H, W)).astype(np.float32)
    k = 3
    for checkpoint in (True, False):
        c = dev(color).requires_grad_(True)
        m = dev(mv).requires_grad_(True)
        out, mask = autograd.warp(c, dev(depth), m, k, 4, checkpoint=checkpoint)
        loss = (((out - dev(target)) ** 2) * (mask == 0)).sum()
        loss.backward()
        keys = oracle.splat(depth, mv, k)
        wo, wm = oracle.warp(color.astype(np.float64), depth, mv, keys, k)
        wl, wg = oracle.l2_loss_grad(wo, target, wm)
        wc, wmv = oracle.warp_backward(wg, color.astype(np.float64), depth, mv, keys, k)
        assert abs(loss.item() - wl) <= 1e-4 * max(1.0, abs(wl))
        grad_close(c.grad.cpu().numpy(), wc)
        grad_close(m.grad.cpu().numpy(), wmv)
    # the library's own loss kernel agrees
    keys = b.exw_splat_motion(dev(depth), dev(mv), k, 4)
    out, mask = b.exw_warp(dev(color), dev(depth), dev(mv), keys, k, 4)
    lv, g = b.exw_l2_loss_grad(out, dev(target), mask)
    assert abs(lv.item() - wl) <= 1e-4 * max(1.0, abs(wl))
    np.testing.assert_allclose(g.cpu().numpy(), wg, rtol=0, atol=2e-6)


# ------------------------------------------------------------------------------------------------------------
# full-size workloads, in the launch configuration the benchmark times
# ------------------------------------------------------------------------------------------------------------

def test_full_size_4k_fp16(b):
    s = scenes.frame_4k_scene()
    color, depth, mv = scenes.render(s, 0.0, np.float16)
    c, d, m = dev(color), dev(depth), dev(mv)
    for fill in (False, True):
        out, mask = b.exw_extrapolate(c, d, m, nfrac=3, fill=fill)
        ref = oracle.extrapolate(color.astype(np.float64), depth, mv, 3, storage=np.float16, fill=fill)
        for j, (wo, wm, _) in enumerate(ref):
            np.testing.assert_array_equal(mask[j].cpu().numpy(), wm)
            np.testing.assert_allclose(out[j].float().cpu().numpy().astype(np.float64), wo, rtol=0, atol=1e-3)
        assert (mask != 0).float().mean().item() > 0.01      # the occluders open real holes
        o2, m2 = b.exw_extrapolate(c, d, m, nfrac=3, fill=fill, tma=False)
        assert torch.equal(m2, mask) and torch.equal(o2.view(torch.int16), out.view(torch.int16))


def test_full_size_1080p_sequence_sampled(b):
    s = scenes.sequence_1080p_scene()
    F = 60
    H, W = s.H, s.W
    c = torch.empty((F, 3, H, W), dtype=torch.float32, device="cuda")
    d = torch.empty((F, H, W), dtype=torch.float32, device="cuda")
    m = torch.empty((F, 2, H, W), dtype=torch.float32, device="cuda")
    check = {0: None, 31: None, 59: None}
    for f in range(F):
        col, dep, mv = scenes.render(s, float(f))
        c[f].copy_(torch.from_numpy(col))
        d[f].copy_(torch.from_numpy(dep))
        m[f].copy_(torch.from_numpy(mv))
        if f in check:
            check[f] = (col, dep, mv)
    out, mask = b.exw_extrapolate(c, d, m, nfrac=3)
    for f, (col, dep, mv) in check.items():
        ref = oracle.extrapolate(col.astype(np.float64), dep, mv, 3)
        for j, (wo, wm, _) in enumerate(ref):
            np.testing.assert_array_equal(mask[f, j].cpu().numpy(), wm, err_msg=f"frame {f} k={j + 1}")
            np.testing.assert_allclose(out[f, j].cpu().numpy(), wo, rtol=0, atol=2e-6)


def test_timing_and_launch_count(b):
    color, depth, mv = frame_case(("scene", 128, 96, 30))
    n0 = b.exw_launch_count()
    b.exw_timing_enable(True)
    b.exw_extrapolate(dev(color), dev(depth), dev(mv))
    torch.cuda.synchronize()
    assert "exw_engine" in b.exw_timing_names()
    ms, n = b.exw_timing_query("exw_engine")
    assert n == 1 and ms > 0
    b.exw_timing_enable(False)
    assert b.exw_launch_count() - n0 == 4   # header zeroing, bounds and plans of the first frame, the engine
