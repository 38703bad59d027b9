"""GPU parity of the recursive warps of decision paths S5/S6 (Table V) against the FP64 oracle: the carried depth
and motion are bit copies of the winners' (bit-exact), and a chain of quarter-step warps keeps every mask
bit-exact; its colours stay within steps x 2e-6 of the oracle's (each step is a convex combination of its
input -- bilinear taps, pull-push means -- so an input error is not amplified, and each step adds at most the
single-warp bar of 2e-6)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2307_12607_gb300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the gpu-marked tests")
    from paper_2307_12607_gb300 import build, binding
    build.build()
    return binding


def case(name):
    kind, W, H, seed = name
    if kind == "scene":
        s = scenes.make_scene(W, H, seed, 8, vmax=8.0, pan_max=2.0, sliver_fraction=0.2)
        return scenes.render(s, 0.0)
    if kind == "invalid":
        return scenes.random_frame(W, H, seed, mv_scale=6.0, invalid_fraction=0.2)
    return scenes.random_frame(W, H, seed, depth_levels=3, mv_scale=4.0, quarter_grid=True)


CASES = [("scene", 257, 131, 41), ("invalid", 64, 64, 42), ("ties", 37, 29, 43), ("scene", 640, 360, 44)]


@pytest.mark.parametrize("c", CASES)
def test_carry_motion_bit_exact(b, c):
    color, depth, mv = case(c)
    d, m = torch.from_numpy(depth).cuda(), torch.from_numpy(mv).cuda()
    keys = b.exw_splat_motion(d, m, 1, 4)
    _, mask = b.exw_warp(torch.from_numpy(color).cuda(), d, m, keys, 1, 4)
    d1, m1 = b.exw_carry_motion(keys, mask, d, m)
    wd, wm = oracle.carry_motion(keys.cpu().numpy(), mask.cpu().numpy(), depth, mv)
    assert np.array_equal(d1.cpu().numpy().view(np.uint32), wd.view(np.uint32))
    assert np.array_equal(m1.cpu().numpy().view(np.uint32), wm.view(np.uint32))


@pytest.mark.parametrize("fill", [True, False])
@pytest.mark.parametrize("c", CASES[:3])
def test_recursive_chain_matches_oracle(b, c, fill):
    color, depth, mv = case(c)
    steps = 3
    got = b.exw_warp_recursive(torch.from_numpy(color).cuda(), torch.from_numpy(depth).cuda(),
                               torch.from_numpy(mv).cuda(), steps, fill=fill)
    want = oracle.warp_recursive(color, depth, mv, steps, fill=fill)
    for s, ((go, gm), (wo, wmask)) in enumerate(zip(got, want)):
        np.testing.assert_array_equal(gm.cpu().numpy(), wmask, err_msg=f"step {s + 1}")
        np.testing.assert_allclose(go.cpu().numpy(), wo, rtol=0, atol=(s + 1) * 2e-6, err_msg=f"step {s + 1}")


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_recursive_chain_is_the_staged_composition(b, dtype):
    # exw_warp_recursive chains splat, warp, fill and carry on the device: bit-identical to the same entry points
    # called one by one (FP16 colour too, rounded once per step as each exw_warp rounds its output)
    color, depth, mv = case(("scene", 257, 131, 45))
    c = torch.from_numpy(color).to(dtype).cuda()
    d, m = torch.from_numpy(depth).cuda(), torch.from_numpy(mv).cuda()
    got = b.exw_warp_recursive(c, d, m, 3)
    iv = torch.int16 if dtype == torch.float16 else torch.int32
    for s, (go, gm) in enumerate(got):
        keys = b.exw_splat_motion(d, m, 1, 4)
        out, mask = b.exw_warp(c, d, m, keys, 1, 4)
        b.exw_fill_holes(out, mask)
        assert torch.equal(mask, gm) and torch.equal(out.view(iv), go.view(iv)), f"step {s + 1}"
        d, m = b.exw_carry_motion(keys, mask, d, m)
        c = out
