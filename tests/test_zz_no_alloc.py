"""exw_fill_holes_static: the fill for callers that cannot allocate device memory (its scratch is a fixed array
built into the library).  Called through the C ABI and compared with exw_fill_holes, which takes a caller
workspace, on two calls in a row: the second call must not be affected by what the first left in the shared
array.  Collected last (file name) so that a failure here cannot hide the other tests; self-contained, so it also
passes alone in a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the gpu-marked tests")
    from paper_2307_12607_gb300 import build, _lib
    build.build()
    return _lib.load()


def holes(W, H, seed, dtype):
    rng = np.random.default_rng(seed)
    color = rng.uniform(size=(3, H, W)).astype(np.float32)
    mask = (rng.uniform(size=(H, W)) < 0.3).astype(np.uint8)
    for _ in range(5):  # large holes, so some 32x32 tiles have no valid pixel and the coarse levels are used
        y, x = rng.integers(H), rng.integers(W)
        mask[y:y + rng.integers(30, 150), x:x + rng.integers(30, 150)] = 2
    color[:, mask != 0] = 0.0
    return torch.from_numpy(color).to(dtype).cuda(), torch.from_numpy(mask).cuda()


def call_static(lib, color, mask):
    H, W = mask.shape
    cdt = 1 if color.dtype == torch.float16 else 0
    return lib.exw_fill_holes_static(color.data_ptr(), cdt, mask.data_ptr(), W, H,
                                     torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_static_fill_matches_workspace_fill_twice(lib, dtype):
    from paper_2307_12607_gb300 import binding
    iv = torch.int32 if dtype == torch.float32 else torch.int16
    for W, H, seed in ((1920, 1080, 1), (333, 517, 2)):   # two calls in a row, different frames
        color, mask = holes(W, H, seed, dtype)
        want = binding.exw_fill_holes(color.clone(), mask)
        got = color.clone()
        assert call_static(lib, got, mask) == 0
        torch.cuda.synchronize()
        # the same kernels on the same scratch layout: the results are identical bit for bit (a stale node or fill
        # value left in the shared array by the previous call would show here)
        assert torch.equal(got.view(iv), want.view(iv))
        valid = (mask == 0).unsqueeze(0).expand_as(got)
        assert torch.equal(got[valid], color[valid])


def test_static_fill_rejects_frames_beyond_its_scratch(lib):
    color = torch.zeros(16, dtype=torch.float32, device="cuda")
    mask = torch.zeros(16, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # 8192 x 8192 needs 65536 fill tiles; the built-in scratch holds 16384 (status 5: EXW_ERR_WORKSPACE)
    assert lib.exw_fill_holes_static(color.data_ptr(), 0, mask.data_ptr(), 8192, 8192, stream) == 5
    assert lib.exw_fill_holes_static(color.data_ptr(), 0, mask.data_ptr(), 0, 8, stream) == 1
