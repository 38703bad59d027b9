"""Pins for the FP64 CPU oracle: each check ties it to something other than itself -- exact rational arithmetic,
brute force on tiny inputs, closed forms for structured scenes, hand-derived cases (tests/golden/) and the
algebra of the adjoint.  A plausible slip in the oracle (a dropped term, a wrong sign, a transposed index, a
swapped tie break) fails at least one of these.  CPU only."""
from fractions import Fraction
import math
import os
import struct

import numpy as np
import pytest

import oracle
from paper_2307_12607_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EMPTY = int(oracle.EMPTY)


def fbits(x) -> int:
    return struct.unpack("<I", struct.pack("<f", float(x)))[0]


def exact_offset(mv, k, denom=4):
    d = Fraction(float(np.float32(mv))) * k / denom
    return math.floor(Fraction(1, 2) + d), d


# ----------------------------------------------------------------------------------------------------------------
# Target rounding: floor(1/2 + k mv / denom), checked against exact rational arithmetic
# ----------------------------------------------------------------------------------------------------------------

def test_target_offset_golden_cases():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "target_rounding_cases.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) >= 20
    for mv, k, denom, off, rho in rows:
        got = oracle.target_offset(float(mv), int(k), int(denom))
        assert got == int(off), (mv, k)
        num, den = rho.split("/")
        assert Fraction(got) - Fraction(float(mv)) * int(k) / int(denom) == Fraction(int(num), int(den))


def _boundary_values():
    vals = []
    for k in (1, 2, 3):
        for j in range(-70, 71):
            # mv whose exact displacement is a half-integer: k mv / 4 = j + 1/2
            mv = np.float32((j + 0.5) * 4 / k)
            vals += [mv, np.nextafter(mv, np.float32(np.inf)), np.nextafter(mv, np.float32(-np.inf))]
    return vals


@pytest.mark.parametrize("denom", [4, 2, 8])
def test_target_offset_matches_exact_rationals(denom):
    rng = np.random.default_rng(1)
    vals = list(rng.uniform(-70, 70, 3000).astype(np.float32)) + _boundary_values()
    vals += [np.float32(x) for x in (0.0, -0.0, 1e-30, -1e-30, 1e-45, -1e-45, 3e-39, 2.0 ** -24, -2.0 ** -24)]
    for mv in vals:
        for k in range(0, denom + 1):
            want, _ = exact_offset(mv, k, denom)
            assert oracle.target_offset(float(mv), k, denom) == want, (mv, k, denom)


def test_target_offset_huge_motion_never_lands():
    for mv in (1e30, -1e30, 3.4e38, -3.4e38):
        off = oracle.target_offset(mv, 3, 4)
        assert off is None or abs(off) > 1 << 20


# ----------------------------------------------------------------------------------------------------------------
# Forward splat: brute force, closed forms, tie break, order independence
# ----------------------------------------------------------------------------------------------------------------

def brute_force_splat(depth, mv, k, denom=4, order=None):
    """Enumerate every source pixel with exact rational targets; keep (depth, index) lexicographic minimum."""
    H, W = depth.shape
    best = {}
    idx = range(W * H) if order is None else order
    for i in idx:
        y, x = divmod(int(i), W)
        D = depth[y, x]
        mx, my = mv[0, y, x], mv[1, y, x]
        if not (np.isfinite(D) and D > 0 and np.isfinite(mx) and np.isfinite(my)):
            continue
        ox, _ = exact_offset(mx, k, denom)
        oy, _ = exact_offset(my, k, denom)
        qx, qy = x + ox, y + oy
        if not (0 <= qx < W and 0 <= qy < H):
            continue
        cand = (float(D), int(i))
        q = qy * W + qx
        if q not in best or cand < best[q]:
            best[q] = cand
    keys = np.full((H, W), EMPTY, np.uint64)
    for q, (D, i) in best.items():
        keys.flat[q] = (fbits(D) << 32) | i
    return keys


@pytest.mark.parametrize("size,seed,levels,quarter,invalid", [
    ((8, 8), 0, 0, False, 0.0), ((8, 8), 1, 2, True, 0.0), ((16, 16), 2, 3, True, 0.1),
    ((16, 16), 3, 0, False, 0.15), ((13, 7), 4, 2, True, 0.05), ((16, 16), 5, 1, True, 0.0)])
def test_splat_brute_force(size, seed, levels, quarter, invalid):
    W, H = size
    _, depth, mv = scenes.random_frame(W, H, seed, depth_levels=levels, mv_scale=3.0, quarter_grid=quarter,
                                       invalid_fraction=invalid)
    for k in (1, 2, 3, 4):
        got = oracle.splat(depth, mv, k)
        want = brute_force_splat(depth, mv, k)
        np.testing.assert_array_equal(got, want)
        # order independence: enumerate the sources in a random order
        perm = np.random.default_rng(seed + k).permutation(W * H)
        np.testing.assert_array_equal(got, brute_force_splat(depth, mv, k, order=perm))


def test_splat_zero_motion_is_identity():
    _, depth, mv = scenes.random_frame(20, 11, 7, invalid_fraction=0.1)
    mv[...] = 0.0
    mv[:, ~np.isfinite(mv[0])] = 0.0
    keys = oracle.splat(depth, mv, 3)
    H, W = depth.shape
    for q in range(W * H):
        D = depth.flat[q]
        if np.isfinite(D) and D > 0:
            assert int(keys.flat[q]) == (fbits(D) << 32) | q
        else:
            assert int(keys.flat[q]) == EMPTY


@pytest.mark.parametrize("m", [(1, 0), (-2, 1), (3, -3), (0, 2)])
def test_splat_integer_shift(m):
    W, H = 17, 12
    _, depth, mv = scenes.random_frame(W, H, 11)
    mv[0] = 4.0 * m[0]
    mv[1] = 4.0 * m[1]
    for k in (1, 2, 3):
        keys = oracle.splat(depth, mv, k)
        for qy in range(H):
            for qx in range(W):
                sx, sy = qx - k * m[0], qy - k * m[1]
                if 0 <= sx < W and 0 <= sy < H:
                    assert int(keys[qy, qx]) & 0xFFFFFFFF == sy * W + sx
                else:
                    assert int(keys[qy, qx]) == EMPTY


def test_splat_tie_break_and_nearest_depth():
    W, H = 4, 1
    depth = np.array([[5.0, 5.0, 3.0, 9.0]], np.float32)
    mv = np.zeros((2, H, W), np.float32)
    # pixels 0 and 1 both land on x = 2 at k = 4 (full motion): 0 + 2, 1 + 1; pixel 2 stays at 2 but is nearer
    mv[0, 0, 0], mv[0, 0, 1] = 2.0, 1.0
    keys = oracle.splat(depth, mv, 4, 4)
    assert int(keys[0, 2]) == (fbits(3.0) << 32) | 2            # nearest depth wins
    depth[0, 2] = 5.0
    keys = oracle.splat(depth, mv, 4, 4)
    assert int(keys[0, 2]) == (fbits(5.0) << 32) | 0            # equal depth: smallest index wins
    assert int(keys[0, 0]) == EMPTY and int(keys[0, 1]) == EMPTY


# ----------------------------------------------------------------------------------------------------------------
# Mask: closed form for one rectangle over a static background, brute-force crack rule
# ----------------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("v", [(4, 0), (-8, 4), (12, -12), (0, -4)])
def test_mask_single_rectangle_closed_form(v):
    W, H = 40, 30
    depth = np.full((H, W), 100.0, np.float32)
    mv = np.zeros((2, H, W), np.float32)
    x0, x1, y0, y1 = 10, 22, 8, 19
    depth[y0:y1, x0:x1] = 10.0
    mv[0, y0:y1, x0:x1] = v[0]
    mv[1, y0:y1, x0:x1] = v[1]
    for k in (1, 2, 3):
        dx, dy = k * v[0] // 4, k * v[1] // 4
        keys = oracle.splat(depth, mv, k)
        mask = oracle.mask_from_keys(keys)
        R = np.zeros((H, W), bool)
        R[y0:y1, x0:x1] = True
        Rd = np.zeros((H, W), bool)
        Rd[max(0, y0 + dy):max(0, min(H, y1 + dy)), max(0, x0 + dx):max(0, min(W, x1 + dx))] = True
        want = np.where(R & ~Rd, oracle.MASK_EMPTY, 0).astype(np.uint8)
        np.testing.assert_array_equal(mask, want)


def brute_force_mask(keys):
    H, W = keys.shape
    out = np.zeros((H, W), np.uint8)
    for y in range(H):
        for x in range(W):
            kq = int(keys[y, x])
            if kq == EMPTY:
                out[y, x] = 1
                continue
            Dq = Fraction(float(struct.unpack("<f", struct.pack("<I", kq >> 32))[0]))
            cnt = 0
            for nx, ny in ((x - 1, y), (x + 1, y), (x, y - 1), (x, y + 1)):
                if 0 <= nx < W and 0 <= ny < H and int(keys[ny, nx]) != EMPTY:
                    Dn = Fraction(float(struct.unpack("<f", struct.pack("<I", int(keys[ny, nx]) >> 32))[0]))
                    if Dq - Dn > Dq / 32:
                        cnt += 1
            out[y, x] = 2 if cnt >= 3 else 0
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mask_brute_force(seed):
    _, depth, mv = scenes.random_frame(18, 14, 100 + seed, depth_levels=4, mv_scale=2.0, invalid_fraction=0.1)
    for k in (1, 3):
        keys = oracle.splat(depth, mv, k)
        np.testing.assert_array_equal(oracle.mask_from_keys(keys), brute_force_mask(keys))


def test_crack_threshold_is_exact_at_one_thirtysecond():
    # q's depth 32, neighbours at 31 (exactly D_q - D_q/32: not nearer by MORE than D_q/32) vs 31 - ulp
    W, H = 3, 3
    for dn, want in ((np.float32(31.0), 0), (np.nextafter(np.float32(31.0), np.float32(0)), 2)):
        depth = np.full((H, W), dn, np.float32)
        depth[1, 1] = 32.0
        mv = np.zeros((2, H, W), np.float32)
        keys = oracle.splat(depth, mv, 1)
        assert oracle.mask_from_keys(keys)[1, 1] == want


# ----------------------------------------------------------------------------------------------------------------
# Gather: identity, exact shifts, constants, linear ramps, half-pixel average, partition of unity
# ----------------------------------------------------------------------------------------------------------------

def test_warp_zero_motion_identity():
    color, depth, mv = scenes.random_frame(23, 17, 5)
    mv[...] = 0.0
    keys = oracle.splat(depth, mv, 2)
    out, mask = oracle.warp(color, depth, mv, keys, 2)
    np.testing.assert_array_equal(mask, brute_force_mask(keys))
    valid = mask == 0
    assert valid.mean() > 0.5
    np.testing.assert_array_equal(out[:, valid], color.astype(np.float64)[:, valid])
    assert np.all(out[:, ~valid] == 0.0)


@pytest.mark.parametrize("m", [(1, 0), (-1, 2), (2, -1)])
def test_warp_integer_shift_is_exact_copy(m):
    W, H = 19, 15
    color, depth, mv = scenes.random_frame(W, H, 9)
    depth[...] = 7.0
    mv[0], mv[1] = 4.0 * m[0], 4.0 * m[1]
    for k in (1, 2, 3):
        keys = oracle.splat(depth, mv, k)
        out, mask = oracle.warp(color, depth, mv, keys, k)
        for qy in range(H):
            for qx in range(W):
                sx, sy = qx - k * m[0], qy - k * m[1]
                if 0 <= sx < W and 0 <= sy < H:
                    assert mask[qy, qx] == 0
                    np.testing.assert_array_equal(out[:, qy, qx], color[:, sy, sx].astype(np.float64))
                else:
                    assert mask[qy, qx] == oracle.MASK_EMPTY


def test_warp_constant_image_preserved():
    color, depth, mv = scenes.random_frame(31, 21, 12, depth_levels=3, mv_scale=4.0)
    color[...] = np.float32(0.3)
    for k in (1, 2, 3):
        keys = oracle.splat(depth, mv, k)
        out, mask = oracle.warp(color, depth, mv, keys, k)
        v = mask == 0
        assert np.max(np.abs(out[:, v] - np.float64(np.float32(0.3)))) <= 4e-16


def test_warp_reproduces_linear_ramp():
    # dyadic slopes: a*x + b*y + c is exact in float32, so bilinear sampling must return the plane itself
    W, H = 40, 30
    a, b, c = 2.0 ** -6, -(2.0 ** -7), 0.5
    ys, xs = np.mgrid[0:H, 0:W]
    ramp = (a * xs + b * ys + c).astype(np.float32)
    assert np.array_equal(ramp.astype(np.float64), a * xs + b * ys + c)
    color = np.stack([ramp, ramp * 0.5, 1 - ramp]).astype(np.float32)
    depth = np.full((H, W), 5.0, np.float32)
    mv = np.zeros((2, H, W), np.float32)
    mv[0], mv[1] = np.float32(2.6), np.float32(-1.3)
    checked = 0
    for k in (1, 2, 3):
        dx, dy = k * float(np.float32(2.6)) / 4, k * float(np.float32(-1.3)) / 4
        keys = oracle.splat(depth, mv, k)
        out, mask = oracle.warp(color, depth, mv, keys, k)
        for qy in range(H):
            for qx in range(W):
                if mask[qy, qx]:
                    continue
                sx, sy = qx - dx, qy - dy       # q's centre in source coordinates
                if not (0 <= sx <= W - 1 and 0 <= sy <= H - 1):
                    continue
                r = a * sx + b * sy + c
                np.testing.assert_allclose(out[:, qy, qx], [r, 0.5 * r, 1 - r], rtol=0, atol=1e-14)
                checked += 1
    assert checked > 2000


def test_warp_half_pixel_shift_is_two_tap_average():
    W, H = 12, 5
    color, depth, mv = scenes.random_frame(W, H, 13)
    depth[...] = 3.0
    mv[0], mv[1] = 2.0, 0.0
    keys = oracle.splat(depth, mv, 1)
    out, mask = oracle.warp(color, depth, mv, keys, 1)
    C = color.astype(np.float64)
    assert np.all(mask[:, 0] == oracle.MASK_EMPTY)
    np.testing.assert_array_equal(mask[:, 1:], 0)
    np.testing.assert_allclose(out[:, :, 1:], 0.5 * C[:, :, :-1] + 0.5 * C[:, :, 1:], rtol=0, atol=1e-16)


def test_warp_depth_edge_excludes_foreign_taps():
    # winner at depth 10 with a fractional residual; its x-neighbour is at depth 50 (foreign surface)
    W, H = 4, 1
    color = np.zeros((3, H, W), np.float32)
    color[:, 0, :] = np.array([0.1, 0.2, 0.9, 0.4], np.float32)
    depth = np.array([[10.0, 10.0, 50.0, 10.0]], np.float32)
    mv = np.zeros((2, H, W), np.float32)
    mv[0, 0, 1] = np.float32(-1.0)   # k=1: d = -0.25 -> lands on x = 1, rho = +0.25 -> taps x=1 (0.75), x=2 (0.25)
    keys = oracle.splat(depth, mv, 1)
    assert int(keys[0, 1]) & 0xFFFFFFFF == 1
    out, mask = oracle.warp(color, depth, mv, keys, 1)
    assert mask[0, 1] == 0
    np.testing.assert_allclose(out[:, 0, 1], np.float64(np.float32(0.2)), rtol=0, atol=0)  # tap at depth 50 left out
    want = 0.75 * np.float64(np.float32(0.2)) + 0.25 * np.float64(np.float32(0.9))
    # |D(t) - D(p)| <= D(p)/32 = 0.3125 exactly at the boundary: takes part; one ulp further or a D/16 gap: not
    for dt, takes_part in ((10.25, True), (10.3125, True), (9.6875, True),
                           (np.nextafter(np.float32(10.3125), np.float32(99)), False),
                           (np.nextafter(np.float32(9.6875), np.float32(0)), False), (10.5, False), (9.5, False)):
        depth[0, 2] = np.float32(dt)
        out, _ = oracle.warp(color, depth, mv, keys, 1)
        np.testing.assert_allclose(out[:, 0, 1], want if takes_part else np.float64(np.float32(0.2)), rtol=0,
                                   atol=1e-16, err_msg=str(dt))


def test_weights_partition_of_unity():
    _, depth, mv = scenes.random_frame(25, 19, 21, mv_scale=5.0)
    for k in (1, 2, 3):
        keys = oracle.splat(depth, mv, k)
        for q in np.flatnonzero(keys.ravel() != oracle.EMPTY):
            assert abs(oracle.weight_sum(mv, keys, int(q), k) - 1.0) <= 1e-15


# ----------------------------------------------------------------------------------------------------------------
# Pull-push fill: hand cases, identity, constants, single valid pixel
# ----------------------------------------------------------------------------------------------------------------

def _read_pullpush_cases():
    lines = [l.rstrip() for l in open(os.path.join(GOLDEN, "pullpush_hand_cases.txt")) if l.strip() and l[0] != "#"]
    cases, i = [], 0
    while i < len(lines):
        _, name, H, W = lines[i].split()
        H, W = int(H), int(W)
        grid = [lines[i + 1 + r].split() for r in range(H)]
        assert lines[i + 1 + H] == "expect"
        exp = [[float(v) for v in lines[i + 2 + H + r].split()] for r in range(H)]
        cases.append((name, grid, np.array(exp)))
        i += 2 + 2 * H
    return cases


def test_pullpush_hand_cases():
    cases = _read_pullpush_cases()
    assert len(cases) == 5
    for name, grid, exp in cases:
        H, W = len(grid), len(grid[0])
        mask = np.array([[1 if v == "*" else 0 for v in row] for row in grid], np.uint8)
        val = np.array([[0.0 if v == "*" else float(v) for v in row] for row in grid])
        color = np.stack([val, 2 * val, -val])
        out = oracle.fill_holes(color, mask)
        np.testing.assert_array_equal(out[0], exp, err_msg=name)
        np.testing.assert_array_equal(out[1], 2 * exp, err_msg=name)
        np.testing.assert_array_equal(out[2], -exp, err_msg=name)


def test_pullpush_identity_and_constants():
    rng = np.random.default_rng(3)
    color = rng.uniform(size=(3, 37, 53))
    np.testing.assert_array_equal(oracle.fill_holes(color, np.zeros((37, 53), np.uint8)), color)
    mask = (rng.uniform(size=(37, 53)) < 0.7).astype(np.uint8)
    const = np.full((3, 37, 53), 0.625)
    np.testing.assert_array_equal(oracle.fill_holes(np.where(mask[None] == 0, const, 0.0), mask), const)
    out = oracle.fill_holes(np.where(mask[None] == 0, color, 0.0), mask)
    np.testing.assert_array_equal(out[:, mask == 0], color[:, mask == 0])       # valid pixels unchanged
    assert np.all(out >= color[:, mask == 0].min(axis=1)[:, None, None] - 1e-15)  # fill = convex combination
    assert np.all(out <= color[:, mask == 0].max(axis=1)[:, None, None] + 1e-15)


@pytest.mark.parametrize("shape,pos", [((31, 45), (17, 3)), ((1, 9), (0, 8)), ((64, 64), (0, 0)), ((5, 1), (4, 0))])
def test_pullpush_single_valid_pixel_fills_frame(shape, pos):
    H, W = shape
    mask = np.ones((H, W), np.uint8)
    mask[pos] = 0
    color = np.zeros((3, H, W))
    color[:, pos[0], pos[1]] = (0.1, 0.5, 0.9)
    out = oracle.fill_holes(color, mask)
    for c, v in enumerate((0.1, 0.5, 0.9)):
        assert np.all(out[c] == v)


def test_pullpush_no_valid_pixel_gives_zero():
    out = oracle.fill_holes(np.full((3, 7, 9), 0.5), np.ones((7, 9), np.uint8))
    assert np.all(out == 0.0)


# ----------------------------------------------------------------------------------------------------------------
# Adjoint: exact dot-product test in colour (the warp is linear in colour), central differences in motion
# ----------------------------------------------------------------------------------------------------------------

def test_backward_colour_dot_product():
    color, depth, mv = scenes.random_frame(29, 23, 31, depth_levels=3, mv_scale=3.0)
    rng = np.random.default_rng(4)
    for k in (1, 2, 3):
        keys = oracle.splat(depth, mv, k)
        v = rng.standard_normal((3, 23, 29))
        u = rng.standard_normal((3, 23, 29))
        Jv, _ = oracle.warp(v, depth, mv, keys, k)
        gc, _ = oracle.warp_backward(u, color, depth, mv, keys, k)
        lhs, rhs = float(np.sum(Jv * u)), float(np.sum(v * gc))
        assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


def _rho_signs(mv, keys, k):
    H, W = keys.shape
    sig = np.zeros((2, H, W), np.int8)
    for q in np.flatnonzero(keys.ravel() != oracle.EMPTY):
        q = int(q)
        p = int(keys.flat[q]) & 0xFFFFFFFF
        for a, (t, s) in enumerate(((q % W, p % W), (q // W, p // W))):
            rho = Fraction(t - s) - Fraction(float(mv[a].flat[p])) * k / 4
            sig[a].flat[q] = int(rho > 0) - int(rho < 0)
    return sig


@pytest.mark.parametrize("k", [1, 2, 3])
def test_backward_motion_central_differences(k):
    W, H = 14, 12
    color, depth, mv = scenes.random_frame(W, H, 40 + k, depth_levels=2, mv_scale=2.5)
    target = np.random.default_rng(k).uniform(size=(3, H, W))
    keys = oracle.splat(depth, mv, k)
    out, mask = oracle.warp(color, depth, mv, keys, k)
    _, g = oracle.l2_loss_grad(out, target, mask)
    _, gm = oracle.warp_backward(g, color, depth, mv, keys, k)
    sig0 = _rho_signs(mv, keys, k)
    checked = 0
    for a in range(2):
        for p in range(W * H):
            vals = []
            for sgn in (1, -1):
                mvp = mv.copy()
                mvp[a].flat[p] = np.float32(mv[a].flat[p] + sgn * 1e-3)
                kp = oracle.splat(depth, mvp, k)
                if not np.array_equal(kp, keys) or not np.array_equal(_rho_signs(mvp, kp, k), sig0):
                    vals = None
                    break
                o, m = oracle.warp(color, depth, mvp, kp, k)
                vals.append((oracle.l2_loss_grad(o, target, m)[0], float(mvp[a].flat[p])))
            if vals is None:
                continue
            (lp, xp), (lm, xm) = vals
            fd = (lp - lm) / (xp - xm)
            assert abs(fd - gm[a].flat[p]) <= 1e-5 + 1e-4 * abs(fd), (a, p, fd, gm[a].flat[p])
            checked += 1
    assert checked > 0.9 * 2 * W * H


def test_backward_colour_central_differences():
    W, H = 10, 9
    color, depth, mv = scenes.random_frame(W, H, 77, depth_levels=2, mv_scale=2.0)
    target = np.random.default_rng(5).uniform(size=(3, H, W))
    keys = oracle.splat(depth, mv, 3)
    out, mask = oracle.warp(color, depth, mv, keys, 3)
    _, g = oracle.l2_loss_grad(out, target, mask)
    gc, _ = oracle.warp_backward(g, color, depth, mv, keys, 3)
    C = color.astype(np.float64)
    for idx in np.random.default_rng(6).choice(3 * W * H, 60, replace=False):
        e = 1e-4
        Cp, Cm = C.copy(), C.copy()
        Cp.flat[idx] += e
        Cm.flat[idx] -= e
        lp = oracle.l2_loss_grad(oracle.warp(Cp, depth, mv, keys, 3)[0], target, mask)[0]
        lm = oracle.l2_loss_grad(oracle.warp(Cm, depth, mv, keys, 3)[0], target, mask)[0]
        assert abs((lp - lm) / (2 * e) - gc.flat[idx]) <= 1e-8


def test_backward_accumulates():
    color, depth, mv = scenes.random_frame(9, 8, 3)
    keys = oracle.splat(depth, mv, 2)
    g = np.ones((3, 8, 9))
    gc1, gm1 = oracle.warp_backward(g, color, depth, mv, keys, 2)
    gc2, gm2 = oracle.warp_backward(g, color, depth, mv, keys, 2, grad_color=gc1, grad_mv=gm1)
    np.testing.assert_allclose(gc2, 2 * gc1, rtol=1e-15)
    np.testing.assert_allclose(gm2, 2 * gm1, rtol=1e-15)


# ----------------------------------------------------------------------------------------------------------------
# Motion bounds: independent numpy reduction
# ----------------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("W,H,block", [(37, 29, 8), (64, 64, 8), (20, 9, 4)])
def test_motion_bounds_brute_force(W, H, block):
    _, depth, mv = scenes.random_frame(W, H, 55, mv_scale=20.0, invalid_fraction=0.2)
    mv[0, 0, 0] = np.float32(-1e6)
    mv[1, 1, 1] = np.float32(2e5)
    mv[0, 2, 2] = np.float32(-0.0)
    tiles, frame = oracle.motion_bounds(depth, mv, block)
    ok = np.isfinite(depth) & (depth > 0) & np.isfinite(mv[0]) & np.isfinite(mv[1])
    cl = np.clip(mv, -65536, 65536) + np.float32(0.0)
    for by in range((H + block - 1) // block):
        for bx in range((W + block - 1) // block):
            sl = (slice(by * block, (by + 1) * block), slice(bx * block, (bx + 1) * block))
            m = ok[sl]
            if not m.any():
                assert list(tiles[by, bx]) == [np.inf, -np.inf, np.inf, -np.inf]
                continue
            xs, ys = cl[0][sl][m], cl[1][sl][m]
            assert list(tiles[by, bx]) == [xs.min(), xs.max(), ys.min(), ys.max()]
    xs, ys = cl[0][ok], cl[1][ok]
    assert list(frame) == [xs.min(), xs.max(), ys.min(), ys.max()]
    assert frame[0] == -65536.0
    for k in (1, 2, 3):
        brute = 0
        for p in np.flatnonzero(ok.ravel()):
            brute = max(brute, abs(exact_offset(cl[0].flat[p], k)[0]), abs(exact_offset(cl[1].flat[p], k)[0]))
        assert oracle.halo(frame, k) == brute


def test_halo_is_the_largest_offset_magnitude():
    # all motion leftwards and upwards: the farthest reach is the most negative bound, -40 px per frame -> 10 k px
    frame = np.array([-40.0, -3.0, -20.0, -1.0], np.float32)
    assert [oracle.halo(frame, k) for k in (1, 2, 3)] == [10, 20, 30]
    assert oracle.halo(np.array([np.inf, -np.inf, np.inf, -np.inf], np.float32), 3) == 0  # nothing can land


# ----------------------------------------------------------------------------------------------------------------
# Motion-variance features (Sec. IV-C Eq. 1) and the colour MSE / PSNR of the reward (Eq. 3)
# ----------------------------------------------------------------------------------------------------------------

def _exact_var(values):
    """Population variance of float32 values by exact rational arithmetic."""
    vs = [Fraction(float(v)) for v in values]
    if not vs:
        return Fraction(0)
    m = sum(vs) / len(vs)
    return sum((v - m) ** 2 for v in vs) / len(vs)


def test_mv_variance_closed_forms():
    # constant field: 0; x = column index 0..W-1 on every row: (W^2 - 1) / 12 exactly; y = row index likewise
    W, H = 13, 7
    mv = np.zeros((2, H, W), np.float32)
    mv[0] = 2.5
    mv[1] = -4.0
    assert oracle.mv_variance(mv) == (W * H, 0.0, 0.0)
    mv[0] = np.arange(W, dtype=np.float32)[None, :]
    mv[1] = np.arange(H, dtype=np.float32)[:, None]
    n, vx, vy = oracle.mv_variance(mv)
    assert n == W * H and vx == (W * W - 1) / 12 and vy == (H * H - 1) / 12


def test_mv_variance_excludes_non_finite_and_matches_exact_arithmetic():
    rng = np.random.default_rng(3)
    mv = (rng.integers(-64, 65, size=(2, 9, 11)) * 0.25).astype(np.float32)
    mv[0, 1, 2] = np.nan
    mv[1, 3, 4] = np.inf
    mv[0, 5, 6] = -np.inf
    ok = np.isfinite(mv[0]) & np.isfinite(mv[1])
    n, vx, vy = oracle.mv_variance(mv)
    assert n == ok.sum() == 9 * 11 - 3
    assert vx == pytest.approx(float(_exact_var(mv[0][ok])), rel=1e-15, abs=0)
    assert vy == pytest.approx(float(_exact_var(mv[1][ok])), rel=1e-15, abs=0)
    # a second routine: numpy's variance of the finite subset
    assert vx == pytest.approx(float(np.var(mv[0][ok].astype(np.float64))), rel=1e-14)
    # no finite vector at all: count 0, variances 0
    assert oracle.mv_variance(np.full((2, 3, 4), np.nan, np.float32)) == (0.0, 0.0, 0.0)


def test_color_mse_and_psnr_pins():
    rng = np.random.default_rng(4)
    a = rng.uniform(size=(3, 5, 6))
    assert oracle.color_mse(a, a) == 0.0 and oracle.psnr(a, a) == float("inf")
    assert oracle.color_mse(a, a + 0.25) == pytest.approx(0.0625, rel=1e-14)       # constant offset: delta^2
    assert oracle.psnr(a, a + 0.1) == pytest.approx(20.0, abs=1e-9)                 # 10 log10(1 / 0.01)
    b = rng.uniform(size=(3, 5, 6))
    exact = sum((Fraction(float(x)) - Fraction(float(y))) ** 2 for x, y in zip(a.ravel(), b.ravel())) / a.size
    assert oracle.color_mse(a, b) == pytest.approx(float(exact), rel=1e-14)


def _ssim_reference(a, b):
    """SSIM by a second route: the Gaussian window as an outer product, numpy's correlation over valid positions."""
    from scipy.signal import correlate2d
    x = np.arange(11) - 5
    g = np.exp(-(x * x) / 4.5)
    w = np.outer(g, g)
    w /= w.sum()
    C1, C2 = 1e-4, 9e-4
    vals = []
    for c in range(3):
        f = lambda img: correlate2d(img, w, mode="valid")
        ma, mb = f(a[c]), f(b[c])
        va, vb, cab = f(a[c] * a[c]) - ma * ma, f(b[c] * b[c]) - mb * mb, f(a[c] * b[c]) - ma * mb
        vals.append(((2 * ma * mb + C1) * (2 * cab + C2)) / ((ma * ma + mb * mb + C1) * (va + vb + C2)))
    return float(np.mean(vals))


def test_ssim_pins():
    rng = np.random.default_rng(5)
    a = rng.uniform(size=(3, 19, 23))
    assert oracle.ssim(a, a) == 1.0                                     # identical images: exactly 1
    b = np.clip(a + rng.normal(scale=0.1, size=a.shape), 0, 1)
    assert oracle.ssim(a, b) == pytest.approx(oracle.ssim(b, a), rel=1e-14)   # symmetric
    assert oracle.ssim(a, b) == pytest.approx(_ssim_reference(a, b), rel=1e-12)
    # constant images p and q: the structure terms vanish, SSIM = (2pq + C1) / (p^2 + q^2 + C1)
    p, q = 0.3, 0.7
    want = (2 * p * q + 1e-4) / (p * p + q * q + 1e-4)
    assert oracle.ssim(np.full((3, 12, 15), p), np.full((3, 12, 15), q)) == pytest.approx(want, rel=1e-9)
    assert math.isnan(oracle.ssim(np.zeros((3, 10, 40)), np.zeros((3, 10, 40))))   # no window fits


# ----------------------------------------------------------------------------------------------------------------
# Recursive warps (Table V, S5/S6): the warped frame carries its winners' depth and motion
# ----------------------------------------------------------------------------------------------------------------

def test_carry_motion_zero_motion_is_identity():
    # a smooth surface (no crack can form) that does not move: every pixel is its own winner
    color, _, _ = scenes.random_frame(23, 17, 31)
    yy, xx = np.mgrid[0:17, 0:23]
    depth = (40.0 + 0.01 * xx + 0.02 * yy).astype(np.float32)
    mv = np.zeros((2, 17, 23), np.float32)
    keys = oracle.splat(depth, mv, 1, 4)
    out, mask = oracle.warp(color, depth, mv, keys, 1, 4)
    d1, m1 = oracle.carry_motion(keys, mask, depth, mv)
    assert np.array_equal(d1, depth) and np.array_equal(m1, mv) and np.array_equal(out, color.astype(np.float64))


def test_two_quarter_steps_of_a_translation_equal_one_half_step():
    # every pixel moves by (8, -4) per frame: a quarter step is (2, -1) whole pixels; warping the warped frame again
    # (with the carried motion) equals warping the source by 2/4 wherever both sources lie in the frame
    W, H = 40, 30
    color, _, _ = scenes.random_frame(W, H, 32)
    yy, xx = np.mgrid[0:H, 0:W]
    depth = (40.0 + 0.01 * xx + 0.02 * yy).astype(np.float32)
    mv = np.empty((2, H, W), np.float32)
    mv[0], mv[1] = 8.0, -4.0
    two = oracle.warp_recursive(color, depth, mv, 2, fill=False)
    keys2 = oracle.splat(depth, mv, 2, 4)
    half, hmask = oracle.warp(color, depth, mv, keys2, 2, 4)
    inner = (slice(2, H - 2), slice(4, W - 4))
    assert np.array_equal(two[1][1][inner], hmask[inner]) and not hmask[inner].any()
    # the holes of P_1 carry no motion and never land again, so P_2 is uncovered exactly where the half step is
    yy, xx = np.mgrid[0:H, 0:W]
    assert np.array_equal(two[1][1] != 0, (xx < 4) | (yy >= H - 2)) and np.array_equal(two[1][1], hmask)
    assert np.array_equal(two[1][0][(slice(None),) + inner], half[(slice(None),) + inner])


def test_carried_holes_never_land_again():
    color, depth, mv = scenes.random_frame(31, 21, 33, mv_scale=6.0, invalid_fraction=0.1)
    keys = oracle.splat(depth, mv, 1, 4)
    _, mask = oracle.warp(color, depth, mv, keys, 1, 4)
    d1, m1 = oracle.carry_motion(keys, mask, depth, mv)
    holes = mask != 0
    assert holes.any() and np.isnan(d1[holes]).all() and (m1[:, holes] == 0).all()
    idx = (keys.view(np.uint64)[~holes] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert np.array_equal(d1[~holes], depth.ravel()[idx])
    assert np.array_equal(m1[0][~holes], mv[0].ravel()[idx]) and np.array_equal(m1[1][~holes], mv[1].ravel()[idx])


# ----------------------------------------------------------------------------------------------------------------
# The composite P_1..P_3 (Sec. IV-B): closed forms for zero motion and whole-pixel translations, FP16 storage
# ----------------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("fill", [True, False])
def test_extrapolate_zero_motion_returns_the_source(fill):
    color, depth, mv = scenes.random_frame(21, 13, 41)
    mv[...] = 0.0
    yy, xx = np.mgrid[0:13, 0:21]
    depth = (30.0 + 0.01 * xx + 0.02 * yy).astype(np.float32)  # smooth: no pixel is a crack
    res = oracle.extrapolate(color, depth, mv, 3, fill=fill)
    ident = (depth.view(np.uint32).astype(np.uint64) << np.uint64(32)) | np.arange(21 * 13, dtype=np.uint64).reshape(13, 21)
    for out, mask, keys in res:
        assert not mask.any()
        assert np.array_equal(keys.view(np.uint64), ident)
        assert np.array_equal(out, color.astype(np.float64))


def test_extrapolate_translation_uncovers_a_strip_that_the_fill_closes():
    # every pixel moves by (8, 4) per frame on one depth: P_k is the source shifted by (2k, k) whole pixels; the
    # first 2k columns and k rows are uncovered (EMPTY) and, with the fill, take values inside the frame's range
    W, H = 24, 16
    color, depth, mv = scenes.random_frame(W, H, 42)
    depth[...] = 3.0
    mv[0], mv[1] = 8.0, 4.0
    c64 = color.astype(np.float64)
    for fill in (False, True):
        for k, (out, mask, _) in enumerate(oracle.extrapolate(color, depth, mv, 3, fill=fill), start=1):
            yy, xx = np.mgrid[0:H, 0:W]
            uncovered = (xx < 2 * k) | (yy < k)
            assert np.array_equal(mask != 0, uncovered) and np.all(mask[uncovered] == oracle.MASK_EMPTY)
            assert np.array_equal(out[:, k:, 2 * k:], c64[:, :H - k, :W - 2 * k])
            if fill:
                lo, hi = c64[:, :H - k, :W - 2 * k].min(), c64[:, :H - k, :W - 2 * k].max()
                assert np.all(out[:, uncovered] >= lo) and np.all(out[:, uncovered] <= hi)
            else:
                assert np.all(out[:, uncovered] == 0.0)


def test_extrapolate_fp16_storage_rounds_the_warped_colour_once():
    # a half-pixel shift averages two taps; with FP16 storage the valid pixels are those averages rounded to FP16
    # (reading 9), and a frame without holes is left as stored
    W, H = 16, 9
    color, depth, mv = scenes.random_frame(W, H, 43)
    color = color.astype(np.float16).astype(np.float32)
    depth[...] = 5.0
    mv[0], mv[1] = 2.0, 0.0                           # k = 1: half a pixel to the right
    out, mask, _ = oracle.extrapolate(color, depth, mv, 1, storage=np.float16, fill=True)[0]
    c = color.astype(np.float64)
    # T(p) = p + floor(1/2 + 1/2) = p + 1, rho = 1 - 1/2 = +1/2: the tap is p + 1 -> q's colour averages
    # source columns q - 1 and q (the winner p = q - 1 and its right neighbour)
    avg = 0.5 * (c[:, :, :-1] + c[:, :, 1:])
    assert not mask[:, 1:].any() and np.all(mask[:, 0] == oracle.MASK_EMPTY)
    assert np.array_equal(out[:, :, 1:], avg.astype(np.float16).astype(np.float64))
