"""GPU parity of the frame statistics against the FP64 oracle: the motion-variance features Var_x, Var_y
(Sec. IV-C, Eq. 1) and the colour MSE of the reward's PSNR (Eq. 3).  Both are FP64 reductions in a fixed order:
counts are exact, the moments agree with the two-pass oracle within the error bound of its sequential FP64 sums
(n * 2^-53 relative; the kernels sum in trees), and two calls give identical bits."""
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


def mv_case(name):
    kind, W, H, seed = name
    if kind == "scene":
        s = scenes.make_scene(W, H, seed, 12, vmax=12.0, pan_max=4.0)
        return scenes.render(s, 0.0)[2]
    _, _, mv = scenes.random_frame(W, H, seed, mv_scale=30.0, invalid_fraction=0.1 if kind == "invalid" else 0.0)
    return mv


@pytest.mark.parametrize("case", [("rand", 1, 1, 1), ("rand", 7, 3, 2), ("invalid", 97, 61, 3), ("scene", 640, 360, 4),
                                  ("scene", 1920, 1080, 5), ("invalid", 333, 1, 6)])
def test_mv_variance_matches_oracle(b, case):
    mv = mv_case(case)
    want = oracle.mv_variance(mv)
    m = torch.from_numpy(np.ascontiguousarray(mv)).cuda()
    got = b.exw_mv_variance(m)
    assert got[0] == want[0]
    np.testing.assert_allclose(got[1:], want[1:], rtol=max(1e-10, 4 * mv[0].size * 2.0 ** -53), atol=1e-12)
    assert b.exw_mv_variance(m) == got                 # deterministic


def test_mv_variance_edge_cases(b):
    mv = np.full((2, 5, 9), np.nan, np.float32)
    assert b.exw_mv_variance(torch.from_numpy(mv).cuda()) == (0.0, 0.0, 0.0)
    mv = np.full((2, 40, 50), 3.25, np.float32)       # constant: exactly 0
    assert b.exw_mv_variance(torch.from_numpy(mv).cuda()) == (2000.0, 0.0, 0.0)
    # a large common offset with a small spread: the shifted sums keep the variance accurate
    rng = np.random.default_rng(9)
    mv = (60000.0 + rng.uniform(-0.5, 0.5, size=(2, 300, 400))).astype(np.float32)
    want = oracle.mv_variance(mv)
    got = b.exw_mv_variance(torch.from_numpy(mv).cuda())
    np.testing.assert_allclose(got[1:], want[1:], rtol=1e-9)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("W,H", [(1, 1), (37, 29), (1920, 1080)])
def test_color_mse_matches_oracle(b, dtype, W, H):
    rng = np.random.default_rng(W + H)
    x = rng.uniform(size=(3, H, W)).astype(np.float32)
    y = np.clip(x + rng.normal(scale=0.05, size=x.shape), 0, 1).astype(np.float32)
    xa, ya = torch.from_numpy(x).to(dtype).cuda(), torch.from_numpy(y).to(dtype).cuda()
    want = oracle.color_mse(xa.cpu().double().numpy(), ya.cpu().double().numpy())
    got = b.exw_color_mse(xa, ya)
    # the oracle adds the 3 W H positive terms one after another (relative error up to 3 W H * 2^-53), the
    # kernel in a tree: the bar is that bound
    assert got == pytest.approx(want, rel=max(1e-12, 3 * W * H * 2.0 ** -53), abs=0)
    assert b.exw_color_mse(xa, ya) == got
    assert b.exw_color_mse(xa, xa) == 0.0 and b.exw_psnr(xa, xa) == float("inf")
    # PSNR on the device: -10 log10 of the same MSE (the log adds a few ulp)
    assert b.exw_psnr(xa, ya) == pytest.approx(oracle.psnr(xa.cpu().double().numpy(), ya.cpu().double().numpy()),
                                               rel=1e-12 + 3 * W * H * 2.0 ** -53, abs=0)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("W,H", [(11, 11), (37, 29), (200, 150), (640, 360)])
def test_ssim_matches_oracle(b, dtype, W, H):
    # the kernel keeps the window moments in FP32 on values shifted to [-1/2, 1/2]: each moment is within about
    # 1e-7 of the FP64 one, and an error e in a variance moves a window's SSIM by at most e / C2 (C2 = 9e-4), so
    # the bar on the mean is 2e-4
    rng = np.random.default_rng(W * H)
    x = rng.uniform(size=(3, H, W)).astype(np.float32)
    y = np.clip(x + rng.normal(scale=0.08, size=x.shape), 0, 1).astype(np.float32)
    y[:, : H // 3, : W // 3] = 0.25                        # a flat patch: small variances
    xa, ya = torch.from_numpy(x).to(dtype).cuda(), torch.from_numpy(y).to(dtype).cuda()
    want = oracle.ssim(xa.cpu().double().numpy(), ya.cpu().double().numpy())
    got = b.exw_ssim(xa, ya)
    assert abs(got - want) <= 2e-4
    assert b.exw_ssim(xa, ya) == got
    assert abs(b.exw_ssim(xa, xa) - 1.0) <= 1e-6
