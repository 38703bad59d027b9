"""GPU tests of the batched persistent path: every stream against the FP64 CPU oracle (masks bit-exact, colour within
2e-6 for float32 storage and 1e-3 for float16 storage), and bit-identical to exw_extrapolate per stream (mixed sizes,
colour types and widths that do or do not allow TMA staging); the autotuner, replay from a CUDA graph, and a bounded
wait that runs out (injected on the host with EXW_FAULT=timeout) reporting EXW_ERR_TIMEOUT without faulting the GPU."""
import os

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


SIZES = [(256, 144, torch.float16), (320, 180, torch.float32), (200, 120, torch.float16), (97, 61, torch.float32),
         (640, 360, torch.float16), (130, 77, torch.float16), (96, 64, torch.float32)]


def make_streams(seed=0, sizes=SIZES):
    streams = []
    for i, (W, H, dt) in enumerate(sizes):
        s = scenes.make_scene(W, H, 1000 + seed * 100 + i, 10, vmax=10.0, pan_max=3.0, sliver_fraction=0.1)
        c, d, m = scenes.render(s, 0.0)
        streams.append((torch.from_numpy(c).to(dt).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(m).cuda()))
    return streams


def same(a, b_):
    iv = torch.int16 if a.dtype == torch.float16 else torch.int32
    return torch.equal(a.view(iv), b_.view(iv))


TOL = {torch.float32: 2e-6, torch.float16: 1e-3}
NPDT = {torch.float32: np.float32, torch.float16: np.float16}


def assert_matches_oracle(stream, out, nfrac, fill, what=""):
    """One stream's batched outputs against the oracle run on the same inputs: the warped colour rounded once to
    the storage type before the fill, masks bit-exact, colour within the storage type's tolerance."""
    c, d, m = stream
    o, k = out
    cs = c.cpu().numpy()
    ref = oracle.extrapolate(cs.astype(np.float64), d.cpu().numpy(), m.cpu().numpy(), nfrac, storage=NPDT[c.dtype],
                             fill=fill)
    for j, (wo, wm, _) in enumerate(ref):
        np.testing.assert_array_equal(k[j].cpu().numpy(), wm, err_msg=f"{what} mask of P_{j + 1}")
        np.testing.assert_allclose(o[j].float().cpu().numpy().astype(np.float64), wo, rtol=0, atol=TOL[c.dtype],
                                   err_msg=f"{what} colour of P_{j + 1}")


@pytest.mark.parametrize("fill", [True, False])
@pytest.mark.parametrize("tma", [True, False])
def test_batched_matches_oracle(b, fill, tma):
    # every stream of the mixed set (sizes, FP16 / FP32 colour, widths with and without TMA staging) against the
    # oracle itself, not only against the single-stream launch
    streams = make_streams(seed=5)
    outs = b.exw_extrapolate_batched(streams, nfrac=3, fill=fill, tma=tma)
    for i, (s, o) in enumerate(zip(streams, outs)):
        assert_matches_oracle(s, o, 3, fill, f"stream {i} {tuple(s[1].shape)} {s[0].dtype}")


@pytest.mark.parametrize("fill", [True, False])
@pytest.mark.parametrize("tma", [True, False])
def test_batched_matches_single_stream(b, fill, tma):
    streams = make_streams()
    outs = b.exw_extrapolate_batched(streams, nfrac=3, fill=fill, tma=tma)
    for (c, d, m), (o, k) in zip(streams, outs):
        o1, k1 = b.exw_extrapolate(c, d, m, nfrac=3, fill=fill)
        assert torch.equal(k, k1)
        assert same(o, o1)


@pytest.mark.parametrize("shape", [0, 1])
@pytest.mark.parametrize("lag,pair", [(1, True), (2, False), (3, True)])
def test_every_schedule_the_tuner_can_choose_matches_oracle(b, shape, lag, pair):
    # each window shape, queue distance and smooth-tile sharing, forced through exw_tuner_fix: every stream against
    # the oracle and bit-identical to the single-stream launch (which runs the default schedule)
    streams = make_streams(seed=6)
    t = b.exw_tuner_create()
    try:
        b.exw_tuner_fix(t, shape, lag, pair)
        for fill in (True, False):
            outs = b.exw_extrapolate_batched(streams, nfrac=3, fill=fill, tuner=t)
            for i, (s, o) in enumerate(zip(streams, outs)):
                assert_matches_oracle(s, o, 3, fill, f"shape {shape} lag {lag} pair {pair} stream {i}")
                o1, k1 = b.exw_extrapolate(*s, nfrac=3, fill=fill)
                assert torch.equal(o[1], k1) and same(o[0], o1)
    finally:
        b.exw_tuner_destroy(t)


def test_batched_with_tuner_and_fewer_fractions(b):
    streams = make_streams(seed=1)
    t = b.exw_tuner_create()
    try:
        for nfrac in (3, 2):
            outs = b.exw_extrapolate_batched(streams, nfrac=nfrac, tuner=t)
            for (c, d, m), (o, k) in zip(streams, outs):
                o1, k1 = b.exw_extrapolate(c, d, m, nfrac=nfrac)
                assert torch.equal(k, k1) and same(o, o1)
            for i in (0, 3, 4):
                assert_matches_oracle(streams[i], outs[i], nfrac, True, f"tuned, nfrac {nfrac}, stream {i}")
        rep = b.exw_tuner_report(t)
        assert rep.count("best") == 2 and "lag" in rep
        # both window shapes were timed (each trial line names its window)
        assert "FP32 56x48 / FP16 64x56" in rep and "FP32 64x42 / FP16 56x64" in rep
    finally:
        b.exw_tuner_destroy(t)


def test_batched_graph_capture_and_replay(b):
    streams = make_streams(seed=2)
    nfrac = 3
    outs = [(torch.empty((nfrac,) + tuple(c.shape), dtype=c.dtype, device="cuda"),
             torch.empty((nfrac,) + tuple(d.shape), dtype=torch.uint8, device="cuda")) for c, d, _ in streams]
    ws = b.workspace(b.exw_batched_workspace_bytes([s for s in streams], nfrac), "cuda")
    t = b.exw_tuner_create()
    try:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            b.exw_extrapolate_batched(streams, nfrac, outs=outs, ws=ws, tuner=t)   # tunes outside the capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            b.exw_extrapolate_batched(streams, nfrac, outs=outs, ws=ws, tuner=t)
        for rep in range(2):
            fresh = make_streams(seed=10 + rep)
            for (c, d, m), (c2, d2, m2) in zip(streams, fresh):
                c.copy_(c2)
                d.copy_(d2)
                m.copy_(m2)
            g.replay()
            torch.cuda.synchronize()
            assert b.exw_device_status(ws) == 0
            for i, ((c, d, m), (o, k)) in enumerate(zip(streams, outs)):
                o1, k1 = b.exw_extrapolate(c, d, m, nfrac=nfrac)
                assert torch.equal(k, k1) and same(o, o1)
                assert_matches_oracle((c, d, m), (o, k), nfrac, True, f"replay {rep} stream {i}")
    finally:
        b.exw_tuner_destroy(t)


def test_batched_bounded_wait_times_out_and_context_survives(b):
    streams = make_streams(seed=3, sizes=SIZES[:4])
    ws = b.workspace(b.exw_batched_workspace_bytes(streams, 3), "cuda")
    os.environ["EXW_FAULT"] = "timeout"
    try:
        b.exw_extrapolate_batched(streams, 3, ws=ws)
        torch.cuda.synchronize()
        assert b.exw_device_status(ws) == 4          # EXW_ERR_TIMEOUT
    finally:
        del os.environ["EXW_FAULT"]
    outs = b.exw_extrapolate_batched(streams, 3, ws=ws)  # the context is intact: a normal call succeeds
    torch.cuda.synchronize()
    assert b.exw_device_status(ws) == 0
    for (c, d, m), (o, k) in zip(streams, outs):
        o1, k1 = b.exw_extrapolate(c, d, m, nfrac=3)
        assert torch.equal(k, k1) and same(o, o1)


def test_batched_full_config_sampled(b):
    # the 48-stream workload: 12 each of 720p, 1080p, 1440p and 4K, FP16 colour; four streams checked in full
    scs = scenes.batched_scenes()
    streams = []
    for s in scs:
        c, d, m = scenes.render(s, 0.0, np.float16)
        streams.append((torch.from_numpy(c).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(m).cuda()))
    outs = b.exw_extrapolate_batched(streams, 3)
    for i in (0, 13, 30, 47):   # one stream of each resolution: 720p, 1080p, 1440p, 4K
        c, d, m = streams[i]
        o1, k1 = b.exw_extrapolate(c, d, m, nfrac=3)
        assert torch.equal(outs[i][1], k1) and same(outs[i][0], o1)
        assert_matches_oracle(streams[i], outs[i], 3, True, f"48-stream launch, stream {i} {tuple(d.shape)}")
