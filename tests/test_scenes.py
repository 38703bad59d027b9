"""CPU checks of the seeded input generator against the workload recipes it implements: determinism, object counts
and kinds, motion and depth ranges, occluder coverage, the stream mix of the batched workload, and that the rendered
motion is the visible surface's velocity."""
import math

import numpy as np

from paper_2307_12607_gb300 import scenes


def _speed(r):
    return math.hypot(float(r.vx), float(r.vy))


def test_seeded_and_deterministic():
    s1, (c1, d1, m1) = scenes.plain_360p()
    s2, (c2, d2, m2) = scenes.plain_360p()
    assert np.array_equal(c1, c2) and np.array_equal(d1, d2) and np.array_equal(m1, m2)
    _, (c3, _, _) = scenes.plain_360p(seed=scenes.workload_seed(0) + 1)
    assert not np.array_equal(c1, c3)
    assert scenes.workload_seed(2, 5) == 0x5EED + 2005


def test_plain_360p_recipe():
    s, (c, d, m) = scenes.plain_360p()
    assert (s.W, s.H, len(s.rects)) == (640, 360, 8)
    assert c.shape == (3, 360, 640) and c.dtype == np.float32 and 0.0 <= c.min() and c.max() <= 1.0
    assert d.min() >= np.float32(0.1) and d.max() == np.float32(100.0)
    assert np.hypot(m[0], m[1]).max() <= 16.0 + 1e-5
    assert math.hypot(float(s.pan[0]), float(s.pan[1])) <= 4.0 + 1e-6


def test_sequence_1080p_recipe_and_motion_is_the_visible_surface():
    s = scenes.sequence_1080p_scene()
    assert (s.W, s.H, len(s.rects)) == (1920, 1080, 32)
    slivers = [r for r in s.rects if min(r.w, r.h) <= 3.0]
    assert len(slivers) == 2 and all(min(r.w, r.h) in (1.0, 2.0, 3.0) for r in slivers)  # 5% of 32
    assert max(_speed(r) for r in s.rects) <= 16.0 + 1e-5
    c, d, m = scenes.render(s, 3.0)
    bg = d == scenes.BACKGROUND_DEPTH
    assert bg.any() and np.all(m[0][bg] == s.pan[0]) and np.all(m[1][bg] == s.pan[1])
    for r in s.rects:  # each rendered object pixel carries its object's velocity and depth
        sel = (d == r.depth) & ~bg
        if sel.any() and sum(1 for o in s.rects if o.depth == r.depth) == 1:
            assert np.all(m[0][sel] == r.vx) and np.all(m[1][sel] == r.vy)


def test_4k_recipe_with_fast_occluders():
    s = scenes.frame_4k_scene()
    assert (s.W, s.H) == (3840, 2160) and len(s.rects) == 64 + 4
    occ = s.rects[64:]
    assert all(0.1 <= float(r.depth) <= 0.5 for r in occ)
    pan = math.hypot(float(s.pan[0]), float(s.pan[1]))
    assert pan <= 16.0 + 1e-5
    for r in occ:  # occluder speed 24-48 px before the pan is added
        v = math.hypot(float(r.vx) - float(s.pan[0]), float(r.vy) - float(s.pan[1]))
        assert 24.0 - 1e-3 <= v <= 48.0 + 1e-3
    assert max(_speed(r) for r in s.rects) <= 64.0 + 1e-4
    area = sum(r.w * r.h for r in occ) / (s.W * s.H)
    assert 0.15 <= area <= 0.2 + 1e-9


def test_batched_stream_mix():
    scs = scenes.batched_scenes()
    assert len(scs) == 48
    sizes = [(s.W, s.H) for s in scs]
    for res in scenes.BATCHED_RESOLUTIONS:
        assert sizes.count(res) == 12
    assert all(16 <= len(s.rects) <= 64 for s in scs)


def test_ground_truth_is_the_scene_at_the_fractional_time():
    s = scenes.make_scene(160, 96, 7, 6)
    for k in (1, 2, 3, 4):
        assert np.array_equal(scenes.ground_truth(s, 2.0, k), scenes.render(s, 2.0 + k / 4)[0])


def test_random_frame_structure():
    c, d, m = scenes.random_frame(64, 48, 3, depth_levels=3, quarter_grid=True, invalid_fraction=0.2)
    finite = d[np.isfinite(d) & (d > 0)]
    assert len(np.unique(finite)) <= 3                       # ties from three depth levels
    mm = m[np.isfinite(m)]
    assert np.all(mm * 2 == np.round(mm * 2))                # on the half-pixel grid
    assert np.isnan(d).any() and np.isinf(d).any() and (d == 0).any() and (d < 0).any()
