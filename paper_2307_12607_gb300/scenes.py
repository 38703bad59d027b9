"""Seeded synthetic scenes standing in for the paper's game workloads.

ExWarp evaluates on Unreal Engine scenes whose renderer emits colour, depth and screen-space motion-vector
G-buffers at 30 fps (Sec. III-A, Table I; Sec. IV-C, Eq. 1 uses the motion-vector buffer).  Those scenes are not
available, so this module rasterises a 2-D stand-in: a value-noise textured background plane at depth 100 that
moves with a global camera pan, plus axis-aligned textured rectangles at random depths, each with its own rigid
2-D velocity.  Every quantity is drawn from a seeded ``numpy.random.Generator(PCG64)``.

Conventions shared with the rest of the package (pixel centres at integer coordinates, x right, y down):

* colour ``[3][H][W]`` float32 in [0, 1] (cast to float16 where a workload stores colour in FP16);
* depth ``[H][W]`` float32 in [0.1, 100];
* motion ``[2][H][W]`` float32, plane 0 = x, the displacement in pixels of the visible surface over one source
  frame interval, forward in time.

A pixel belongs to a rectangle when its centre lies inside it (``x0 <= x < x0 + w``); rectangles are painted far
to near.  The module also renders ground truth at fractional times ``t + k/4`` (objects advanced by ``k/4`` of
their motion), which serves as the loss target of the differentiation workload and as quality context.

This module holds no warping arithmetic.  It only produces inputs, and it is the one module that both the CUDA
path's tests/benchmarks and the CPU oracle's tests draw inputs from.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BACKGROUND_DEPTH = np.float32(100.0)
LATTICE_SPACING = 8.0          # value-noise lattice pitch in pixels
BACKGROUND_PERIOD = 64         # lattice cells per period of the (periodic) background texture
SEED_BASE = 0x5EED


def workload_seed(config: int, stream: int = 0) -> int:
    """Seed for workload ``config`` (0..4) and independent stream ``stream``."""
    return SEED_BASE + 1000 * config + stream


@dataclasses.dataclass
class Rect:
    x0: float           # left edge at t = 0 (pixels)
    y0: float           # top edge at t = 0
    w: float
    h: float
    vx: np.float32      # velocity incl. camera pan, pixels / frame
    vy: np.float32
    depth: np.float32
    lattice: np.ndarray  # [3][Ly][Lx] float32 value-noise lattice in [0, 1]


@dataclasses.dataclass
class Scene:
    W: int
    H: int
    pan: tuple           # (float32, float32) camera pan, pixels / frame
    background: np.ndarray  # [3][P][P] periodic lattice
    rects: list


def _disc(rng: np.random.Generator, rmax: float, rmin: float = 0.0):
    r = math.sqrt(rng.uniform(rmin * rmin, rmax * rmax)) if rmax > 0 else 0.0
    th = rng.uniform(0.0, 2.0 * math.pi)
    return r * math.cos(th), r * math.sin(th)


def _lattice(rng: np.random.Generator, w: float, h: float) -> np.ndarray:
    lx = int(math.ceil(w / LATTICE_SPACING)) + 2
    ly = int(math.ceil(h / LATTICE_SPACING)) + 2
    base = rng.uniform(0.0, 1.0, size=(3, 1, 1))
    amp = rng.uniform(0.2, 0.6)
    lat = base + amp * (rng.uniform(0.0, 1.0, size=(3, ly, lx)) - 0.5)
    return np.clip(lat, 0.0, 1.0).astype(np.float32)


def make_scene(W: int, H: int, seed: int, n_objects: int, vmax: float = 12.0, pan_max: float = 4.0,
               sliver_fraction: float = 0.0, occluder_coverage: float = 0.0, occluder_speed: float | None = None,
               size_range=(1.0 / 24, 1.0 / 6)) -> Scene:
    """Draw a scene.  ``|mv| <= vmax + pan_max`` for ordinary objects; occluders move at up to ``occluder_speed``
    (default ``vmax``) and sit at the nearest depths, together covering about ``occluder_coverage`` of the frame."""
    rng = np.random.Generator(np.random.PCG64(seed))
    px, py = _disc(rng, pan_max)
    pan = (np.float32(px), np.float32(py))
    bg = rng.uniform(0.05, 0.95, size=(3, BACKGROUND_PERIOD, BACKGROUND_PERIOD)).astype(np.float32)
    rects = []
    n_sliver = int(round(sliver_fraction * n_objects))
    for i in range(n_objects):
        if i < n_sliver:
            thin = float(rng.integers(1, 4))
            long = rng.uniform(H / 8, H / 2)
            w, h = (thin, long) if rng.uniform() < 0.5 else (long, thin)
        else:
            w = rng.uniform(size_range[0] * W, size_range[1] * W)
            h = rng.uniform(size_range[0] * H, size_range[1] * H)
        x0 = rng.uniform(-0.5 * w, W - 0.5 * w)
        y0 = rng.uniform(-0.5 * h, H - 0.5 * h)
        vx, vy = _disc(rng, vmax)
        depth = np.float32(rng.uniform(0.1, 100.0))
        if depth >= BACKGROUND_DEPTH:
            depth = np.float32(99.0)
        rects.append(Rect(x0, y0, w, h, np.float32(vx + px), np.float32(vy + py), depth, _lattice(rng, w, h)))
    if occluder_coverage > 0.0:
        speed = vmax if occluder_speed is None else occluder_speed
        n_occ = 4
        area = occluder_coverage * W * H / n_occ
        for _ in range(n_occ):
            aspect = rng.uniform(0.5, 2.0)
            w = min(math.sqrt(area * aspect), 0.9 * W)
            h = min(area / w, 0.9 * H)
            x0 = rng.uniform(0.0, W - w)
            y0 = rng.uniform(0.0, H - h)
            vx, vy = _disc(rng, speed, 0.5 * speed)
            depth = np.float32(rng.uniform(0.1, 0.5))
            rects.append(Rect(x0, y0, w, h, np.float32(vx + px), np.float32(vy + py), depth,
                              _lattice(rng, w, h)))
    return Scene(W, H, pan, bg, rects)


def _noise(lattice: np.ndarray, u: np.ndarray, v: np.ndarray, periodic: bool) -> np.ndarray:
    """Value noise at the outer product of 1-D coordinates ``v`` (rows) x ``u`` (cols): [3][len(v)][len(u)]."""
    fu = u / LATTICE_SPACING
    fv = v / LATTICE_SPACING
    iu = np.floor(fu)
    iv = np.floor(fv)
    tu = (fu - iu).astype(np.float32)
    tv = (fv - iv).astype(np.float32)
    su = tu * tu * (np.float32(3.0) - np.float32(2.0) * tu)
    sv = tv * tv * (np.float32(3.0) - np.float32(2.0) * tv)
    iu = iu.astype(np.int64)
    iv = iv.astype(np.int64)
    _, ly, lx = lattice.shape
    if periodic:
        i0, i1 = iu % lx, (iu + 1) % lx
        j0, j1 = iv % ly, (iv + 1) % ly
    else:
        i0 = np.clip(iu, 0, lx - 1)
        i1 = np.clip(iu + 1, 0, lx - 1)
        j0 = np.clip(iv, 0, ly - 1)
        j1 = np.clip(iv + 1, 0, ly - 1)
    su = su[None, None, :]
    sv = sv[None, :, None]
    top = lattice[:, j0[:, None], i0[None, :]] * (1 - su) + lattice[:, j0[:, None], i1[None, :]] * su
    bot = lattice[:, j1[:, None], i0[None, :]] * (1 - su) + lattice[:, j1[:, None], i1[None, :]] * su
    return (top * (1 - sv) + bot * sv).astype(np.float32)


def render(scene: Scene, t: float, color_dtype=np.float32, out=None):
    """Render colour, depth and motion of ``scene`` at time ``t`` (frames).  Returns (color, depth, mv)."""
    W, H = scene.W, scene.H
    if out is None:
        color = np.empty((3, H, W), np.float32)
        depth = np.empty((H, W), np.float32)
        mv = np.empty((2, H, W), np.float32)
    else:
        color, depth, mv = out
    xs = np.arange(W, dtype=np.float64)
    ys = np.arange(H, dtype=np.float64)
    pan_x, pan_y = float(scene.pan[0]), float(scene.pan[1])
    chunk = 512
    for r0 in range(0, H, chunk):
        r1 = min(H, r0 + chunk)
        color[:, r0:r1, :] = _noise(scene.background, xs - pan_x * t, ys[r0:r1] - pan_y * t, periodic=True)
    depth[...] = BACKGROUND_DEPTH
    mv[0] = scene.pan[0]
    mv[1] = scene.pan[1]
    for rc in sorted(scene.rects, key=lambda r: -float(r.depth)):
        x0 = rc.x0 + float(rc.vx) * t
        y0 = rc.y0 + float(rc.vy) * t
        xa = max(0, math.ceil(x0))
        xb = min(W - 1, math.ceil(x0 + rc.w) - 1)
        ya = max(0, math.ceil(y0))
        yb = min(H - 1, math.ceil(y0 + rc.h) - 1)
        if xa > xb or ya > yb:
            continue
        color[:, ya:yb + 1, xa:xb + 1] = _noise(rc.lattice, xs[xa:xb + 1] - x0, ys[ya:yb + 1] - y0, periodic=False)
        depth[ya:yb + 1, xa:xb + 1] = rc.depth
        mv[0, ya:yb + 1, xa:xb + 1] = rc.vx
        mv[1, ya:yb + 1, xa:xb + 1] = rc.vy
    if color_dtype != np.float32:
        color = color.astype(color_dtype)
    return color, depth, mv


# ---------------------------------------------------------------------------------------------------------------
# The five workloads (sizes, object counts and motion ranges as stated for each)
# ---------------------------------------------------------------------------------------------------------------

def plain_360p(seed: int | None = None):
    """640x360, FP32, 8 rectangles, |mv| <= 16 px.  One source frame."""
    s = make_scene(640, 360, workload_seed(0) if seed is None else seed, 8, vmax=12.0, pan_max=4.0)
    return s, render(s, 0.0)


def sequence_1080p_scene(seed: int | None = None) -> Scene:
    """1920x1080, FP32, 32 rectangles of which 5% are 1-3 px slivers, |mv| <= 16 px."""
    return make_scene(1920, 1080, workload_seed(1) if seed is None else seed, 32, vmax=12.0, pan_max=4.0,
                      sliver_fraction=0.05)


def frame_4k_scene(seed: int | None = None) -> Scene:
    """3840x2160, 64 rectangles, |mv| <= 64 px, fast occluders at the nearest depths covering ~20%."""
    return make_scene(3840, 2160, workload_seed(2) if seed is None else seed, 64, vmax=48.0, pan_max=16.0,
                      occluder_coverage=0.20, occluder_speed=48.0)


BATCHED_RESOLUTIONS = ((1280, 720), (1920, 1080), (2560, 1440), (3840, 2160))


def batched_scenes(n_streams: int = 48, seed_config: int = 3):
    """``n_streams`` independent streams, equal shares of the four resolutions, 16-64 objects each."""
    scenes = []
    for s in range(n_streams):
        W, H = BATCHED_RESOLUTIONS[s * len(BATCHED_RESOLUTIONS) // n_streams]
        seed = workload_seed(seed_config, s)
        n_obj = int(np.random.Generator(np.random.PCG64(seed ^ 0xABCDEF)).integers(16, 65))
        scenes.append(make_scene(W, H, seed, n_obj, vmax=12.0, pan_max=4.0))
    return scenes


def diff_scene(seed: int | None = None) -> Scene:
    """1920x1080 FP32 scene for the differentiation workload (8 source frames t = 0..7)."""
    return make_scene(1920, 1080, workload_seed(4) if seed is None else seed, 32, vmax=12.0, pan_max=4.0)


def ground_truth(scene: Scene, t: float, k: int, denom: int = 4):
    """Colour of ``scene`` rendered at ``t + k/denom`` (what a perfect extrapolator would show)."""
    return render(scene, t + k / denom)[0]


# ---------------------------------------------------------------------------------------------------------------
# Small structured inputs for tests (no warping arithmetic: just arrays with known structure)
# ---------------------------------------------------------------------------------------------------------------

def random_frame(W: int, H: int, seed: int, depth_levels: int = 0, mv_scale: float = 3.0, quarter_grid=False,
                 invalid_fraction: float = 0.0):
    """Unstructured random frame: colour U[0,1], depth U[0.1,100) (or one of ``depth_levels`` values, which
    creates equal-depth ties), motion U(-mv_scale, mv_scale) (or multiples of 1/2 when ``quarter_grid``, which puts
    many targets exactly on rounding boundaries), and ``invalid_fraction`` of pixels with a non-finite or
    non-positive depth or a non-finite motion component."""
    rng = np.random.Generator(np.random.PCG64(seed))
    color = rng.uniform(0.0, 1.0, size=(3, H, W)).astype(np.float32)
    if depth_levels > 0:
        levels = rng.uniform(0.1, 100.0, size=depth_levels).astype(np.float32)
        depth = levels[rng.integers(0, depth_levels, size=(H, W))]
    else:
        depth = rng.uniform(0.1, 100.0, size=(H, W)).astype(np.float32)
    if quarter_grid:
        mv = (rng.integers(-2 * int(mv_scale), 2 * int(mv_scale) + 1, size=(2, H, W)) * 0.5).astype(np.float32)
    else:
        mv = rng.uniform(-mv_scale, mv_scale, size=(2, H, W)).astype(np.float32)
    if invalid_fraction > 0.0:
        bad = rng.uniform(size=(H, W)) < invalid_fraction
        kinds = rng.integers(0, 6, size=(H, W))
        depth = depth.copy()
        depth[bad & (kinds == 0)] = np.nan
        depth[bad & (kinds == 1)] = np.inf
        depth[bad & (kinds == 2)] = 0.0
        depth[bad & (kinds == 3)] = -1.0
        mv[0][bad & (kinds == 4)] = np.nan
        mv[1][bad & (kinds == 5)] = np.inf
    return color, np.ascontiguousarray(depth), mv
