"""Benchmark of the warping fast path: extrapolated Mpixel/s on one or more GB300s.

Default workload (one "step"): the 1920x1080 FP32 sequence of 60 source frames with 32 moving rectangles (5% of
them 1-3 px slivers); every step extrapolates P_1..P_3 at t + k/4 for all 60 frames with hole fill = 180 output
frames = 373,248,000 output pixels, through one exw_extrapolate call.  Inputs (3.0 GB) and outputs (4.9 GB) are
far larger than the 129 MB L2, so no flush is needed between steps.

Reported (one JSON line on rank 0):
  value       whole-job output Mpixel/s with inputs resident in HBM (device-timed with CUDA events)
  e2e         the same through the C ABI with host buffers (exw_extrapolate_host): pinned host -> device copies
              of the step's inputs, the extrapolation and device -> host copies of its outputs, overlapped chunk by
              chunk on three streams, all inside the timed region
  roofline    the dominant kernel's algorithmic bytes per launch / its mean event-timed duration, against the
              measured HBM copy bandwidth
  cpu_baseline the CPU oracle (FP64, single thread) on a bounded sample of the same workload
  clocks      nvidia-smi SM clocks and throttle reasons sampled during the timed region
--impl reference times the CPU oracle on the host cores instead (the benchmark's reference arm).
Multi-GPU: one process per GPU (torchrun), each extrapolating its own sequence (replicas, weak scaling, no data
collective); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

W1080, H1080, NFRAMES, NFRAC = 1920, 1080, 60, 3
METRIC, UNIT = "extrapolated Mpixel/s (fwd) at 1080p", "Mpixel/s"  # both arms report this metric
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["exw", "reference"], default="exw")
    ap.add_argument("--frames", type=int, default=NFRAMES)
    ap.add_argument("--e2e-steps", type=int, default=0, help="end-to-end steps (0: as many as --steps)")
    ap.add_argument("--e2e-chunk", type=int, default=8, help="frames per overlapped copy/compute chunk (e2e)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--case", choices=CASES, default=None,
                    help="time only this one configuration and print its JSON (for profiling)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of a kernel per SOURCE FRAME it processed, from one ncu
# capture (a smaller launch; the engine's traffic grows in proportion to the frames of a launch), with the hash of
# the kernel's sources (KERNEL_SOURCES) it was taken on: reported only while they are unchanged, else null.
MEASURED_TRAFFIC = {
    ("exw_engine", "sequence_1080p_fp32"): ((236.626e6 + 282.247e6) / 4, "1ffed5361dabe3d2"),
    ("exw_engine", "warp_4k_fp16"): (105.047e6 + 130.172e6, "1ffed5361dabe3d2"),
    ("exw_train", "fwd_bwd_1080p"): (215.129e6 + 28.325e6, "b1abf7c2171af943"),
}


# The sources of each kernel and its host-side launch (the kernels whose traffic is recorded above).
KERNEL_SOURCES = {
    "exw_engine": ("exw_engine.cu", "exw_engine.cuh", "exw_items.cuh", "exw_tile.cuh", "exw_device.cuh",
                   "exw_tma.cuh", "exw_internal.h", "exw_batched.cu"),
    "exw_train": ("exw_bwd.cu", "exw_device.cuh", "exw_internal.h"),
}
ENGINE_SOURCES = KERNEL_SOURCES["exw_engine"]


def csrc_hash(kernel: str = "exw_engine") -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        f = os.path.join(ROOT, "paper_2307_12607_gb300", "csrc", name)
        h.update(name.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, workload: str):
    t = MEASURED_TRAFFIC.get((kernel, workload))
    return t[0] if t is not None and t[1] == csrc_hash(kernel) else None


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def replica_seed(rank: int) -> int:
    """Scene seed of rank ``rank``'s replica: rank 0 extrapolates the configured sequence, every other rank its own
    independent sequence of the same recipe (weak scaling over independent problems)."""
    from paper_2307_12607_gb300 import scenes
    return scenes.workload_seed(1, rank)


def max_over_ranks(x: float, device) -> float:
    """The maximum of x over all ranks (the step time of a replicated run); x itself on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, seconds: float) -> float:
    """Units all ranks processed per second (millions), from the max-over-ranks time."""
    return world * units_per_rank / seconds / 1e6


def render_sequence(nframes, seed_scene=None):
    from paper_2307_12607_gb300 import scenes
    s = scenes.sequence_1080p_scene(seed_scene)
    col = np.empty((nframes, 3, s.H, s.W), np.float32)
    dep = np.empty((nframes, s.H, s.W), np.float32)
    mv = np.empty((nframes, 2, s.H, s.W), np.float32)
    for f in range(nframes):
        scenes.render(s, float(f), out=(col[f], dep[f], mv[f]))
    return s, col, dep, mv


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm = []
        smax = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                smax = float(r[1])
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_frames(inputs, threads):
    """Run the oracle's extrapolation (3 fractions with fill) over ``inputs`` on ``threads`` host threads; returns the
    wall time.  The oracle is C behind ctypes, which releases the GIL, so threads run it on separate cores."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    t0 = time.perf_counter()
    if threads <= 1:
        for cd, d, m in inputs:
            oracle.extrapolate(cd, d, m, NFRAC)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda a: oracle.extrapolate(a[0], a[1], a[2], NFRAC), inputs))
    return time.perf_counter() - t0


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(seconds: float, seq):
    """The CPU oracle as it stands (FP64 C) on whole frames of the benchmark's own 1080p sequence, timed on one
    thread and on every host core (one frame per thread at a time): one frame is timed first, then as many frames
    as fit in about ``seconds`` of single-thread work, and every frame of the sequence (at most) on all cores."""
    import oracle
    oracle.build()
    s, col, dep, mv = seq
    inputs = lambda n: [(col[f].astype(np.float64), dep[f], mv[f]) for f in range(n)]
    one = _oracle_frames(inputs(1), 1)
    n1 = int(max(1, min(len(col), seconds // max(one, 1e-3))))
    dt1 = _oracle_frames(inputs(n1), 1)
    cores = host_cores()
    nm = int(max(1, min(len(col), cores * max(1, seconds // max(one, 1e-3)) // 2)))
    dtm = _oracle_frames(inputs(nm), cores)
    px = NFRAC * s.W * s.H
    return {"value": nm * px / dtm / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{nm} of the 60 source frames of the 1920x1080 FP32 sequence on {cores} host threads (one "
                      f"frame per thread), {NFRAC} fractions each with hole fill, FP64 C oracle, {dtm:.1f} s",
            "single_thread": {"value": n1 * px / dt1 / 1e6, "unit": UNIT, "cores": 1,
                              "sample": f"{n1} frames on one thread, {dt1:.1f} s"}}


def sequence_config(frames: int, world: int) -> dict:
    """The workload of one step (both arms report it): ``frames`` source frames of the 1080p sequence per GPU."""
    return {"workload": "1920x1080 FP32 sequence: 60 source frames, 32 moving rectangles (5% 1-3 px slivers), "
                        "|mv| <= 16 px; P_1..P_3 at t+k/4 with pull-push hole fill = 180 output frames per step per GPU",
            "frames_per_step": frames, "fractions": NFRAC, "output_pixels_per_step_per_gpu": frames * NFRAC * W1080 * H1080,
            "l2_flush": "none needed: 3.0 GB inputs and 4.9 GB outputs per step exceed L2",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2307_12607_gb300 import scenes
    oracle.build()
    s = scenes.sequence_1080p_scene()
    cores = host_cores()
    nf = min(cores, 16)
    frames = [scenes.render(s, float(f)) for f in range(nf)]
    frames = [(c.astype(np.float64), d, m) for c, d, m in frames]
    # each step extrapolates nf source frames, one per host thread (a bounded sample of the 60-frame step)
    for i in range(args.warmup):
        _oracle_frames(frames[:1], 1)
    dt = 0.0
    for i in range(args.steps):
        dt += _oracle_frames(frames, nf)
    dt /= max(1, args.steps)
    mpx = nf * NFRAC * s.W * s.H / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": mpx, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": sequence_config(args.frames, world),
            "cpu_baseline": {"value": mpx, "unit": UNIT, "cores": nf, "kind": "oracle",
                             "sample": f"each step: {nf} source frames of the 1080p sequence (a bounded sample of "
                                       f"the step) on {nf} host threads, 3 fractions with fill, FP64 C oracle"},
            "e2e": {"value": mpx, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _event_ms(fn, reps):
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _kernel_means(b, fn):
    b.exw_timing_enable(True)
    fn()
    import torch
    torch.cuda.synchronize()
    out = {k: 1000.0 * b.exw_timing_query(k)[0] / max(1, b.exw_timing_query(k)[1]) for k in b.exw_timing_names()}
    b.exw_timing_enable(False)
    return {k: round(v, 2) for k, v in out.items()}


EXTRAS = ("warp_4k_fp16", "extrapolate_4k_fp16_fill", "batched_48_streams", "fwd_bwd_1080p", "quality_and_stats")
CASES = EXTRAS + ("fwd_bwd_fused_only",)  # the last: the fused training pass alone (for profiling it)


def run_extras(b, devc, names=EXTRAS):
    """The other configurations of the metric, each timed with CUDA events on the current stream:
    4K FP16 forward warp (no fill) and full extrapolation, the 48-stream batched launch against a loop of
    single-stream calls over the same frames, and forward+backward of the differentiation workload."""
    import torch
    from paper_2307_12607_gb300 import scenes
    peak, _ = peaks()
    ex = {}
    if "warp_4k_fp16" in names or "extrapolate_4k_fp16_fill" in names:
        _extras_4k(b, devc, names, peak, ex)
    if "batched_48_streams" in names:
        _extras_batched(b, devc, ex)
    if "fwd_bwd_1080p" in names:
        _extras_diff(b, devc, ex)
    if "fwd_bwd_fused_only" in names:
        _extras_diff(b, devc, ex, fused_only=True)
    if "quality_and_stats" in names:
        _extras_quality(b, devc, peak, ex)
    return ex


def _extras_quality(b, devc, peak, ex):
    """Context: PSNR (Sec. IV-C, Eq. 3) of P_1..P_3 with fill against the generator's ground truth at t + k/4 for 8
    frames of the 1080p sequence, and the timing of the two frame statistics (motion-variance features, Eq. 1;
    colour MSE) against the HBM roofline of the bytes they read (the inputs stay L2-resident between repetitions,
    so the fractions are upper bounds)."""
    import torch
    from paper_2307_12607_gb300 import scenes
    sc = scenes.sequence_1080p_scene()
    H, W = 1080, 1920
    psnr = {1: [], 2: [], 3: []}
    ssim = {1: [], 2: [], 3: []}
    ws = b.workspace(b.exw_workspace_bytes(b.OP_STATS, W, H), devc)
    for f in range(8):
        c, d, m = (torch.from_numpy(x).to(devc) for x in scenes.render(sc, float(f)))
        out, _ = b.exw_extrapolate(c, d, m, 3)
        for k in (1, 2, 3):
            gt = torch.from_numpy(scenes.ground_truth(sc, float(f), k)).to(devc)
            psnr[k].append(b.exw_psnr(out[k - 1], gt, ws))
            ssim[k].append(b.exw_ssim(out[k - 1], gt, ws))
    c, d, m = (torch.from_numpy(x).to(devc) for x in scenes.render(sc, 0.0))
    gt = torch.from_numpy(scenes.ground_truth(sc, 0.0, 1)).to(devc)
    out = torch.empty_like(c)
    res = torch.empty(3, dtype=torch.float64, device=devc)

    def var():
        b.lib().exw_mv_variance(m.data_ptr(), W, H, res.data_ptr(), ws.data_ptr(), ws.numel(),
                                b._stream(None, devc))

    def mse():
        b.lib().exw_color_mse(c.data_ptr(), gt.data_ptr(), b.F32, W, H, res.data_ptr(), ws.data_ptr(), ws.numel(),
                              b._stream(None, devc))
    def ssm():
        b.lib().exw_ssim(c.data_ptr(), gt.data_ptr(), b.F32, W, H, res.data_ptr(), ws.data_ptr(), ws.numel(),
                         b._stream(None, devc))
    ms_v = _event_ms(var, 50)
    ms_m = _event_ms(mse, 50)
    ms_s = _event_ms(ssm, 20)
    # decision path S6 (Table V): P_1 = W(F), P_2 = W(P_1), P_3 = W(P_2) through the carried depth and motion
    s6 = {1: [], 2: [], 3: []}
    for f in range(8):
        cf, df, mf = (torch.from_numpy(x).to(devc) for x in scenes.render(sc, float(f)))
        chain = b.exw_warp_recursive(cf, df, mf, 3)
        for k in (1, 2, 3):
            gt = torch.from_numpy(scenes.ground_truth(sc, float(f), k)).to(devc)
            s6[k].append(b.exw_psnr(chain[k - 1][0], gt, ws))
    ms_chain = _event_ms(lambda: b.exw_warp_recursive(c, d, m, 3), 10)
    ex["quality_and_stats"] = {
        "psnr_db_vs_ground_truth": {f"P_{k}": round(sum(v) / len(v), 3) for k, v in psnr.items()},
        "ssim_vs_ground_truth": {f"P_{k}": round(sum(v) / len(v), 5) for k, v in ssim.items()},
        "ssim_us": ms_s * 1e3,
        "s6_recursive_psnr_db": {f"P_{k}": round(sum(v) / len(v), 3) for k, v in s6.items()},
        "s6_recursive_chain_ms": ms_chain,
        "mv_variance_us": ms_v * 1e3, "mv_variance_hbm_frac": 8 * W * H / (ms_v / 1e3) / 1e9 / peak,
        "color_mse_us": ms_m * 1e3, "color_mse_hbm_frac": 24 * W * H / (ms_m / 1e3) / 1e9 / peak,
        "workload": "PSNR and SSIM: 8 frames of the 1920x1080 FP32 sequence, P_1..P_3 with fill against the scene "
                    "rendered at t + k/4 (direct warps of F_t, and the recursive chain of decision path S6); "
                    "statistics: one 1920x1080 frame (8 B/px motion, 2 x 12 B/px colour)"}


def _extras_4k(b, devc, names, peak, ex):
    import torch
    from paper_2307_12607_gb300 import scenes
    # 4K FP16: 3840x2160, 64 objects, |mv| <= 64, fast occluders
    s4 = scenes.frame_4k_scene()
    c4, d4, m4 = (torch.from_numpy(x).to(devc) for x in scenes.render(s4, 0.0, np.float16))
    npx = 3840 * 2160
    o4 = torch.empty((1, 3, 3, 2160, 3840), dtype=torch.float16, device=devc)
    k4 = torch.empty((1, 3, 2160, 3840), dtype=torch.uint8, device=devc)
    ws4 = b.workspace(b.exw_workspace_bytes(b.OP_EXTRAPOLATE, 3840, 2160, b.F16, 1, 3), devc)
    for fill, name in ((False, "warp_4k_fp16"), (True, "extrapolate_4k_fp16_fill")):
        if name not in names:
            continue
        fn = lambda: b.exw_extrapolate(c4[None], d4[None], m4[None], 3, fill, o4, k4, ws4)
        ms = _event_ms(fn, 10)
        km = _kernel_means(b, fn)
        compulsory = (6 + 4 + 8) + 3 * (6 + 1)
        ex[name] = {"value": 3 * npx / ms / 1e3, "unit": "Mpixel/s", "ms_per_frame": ms,
                    "compulsory_bytes_per_source_px": compulsory,
                    "hbm_frac_compulsory": compulsory * npx / (ms / 1e3) / 1e9 / peak, "kernel_us": km,
                    "tile_modes": b.frame_stats(ws4, 0),
                    "traffic_engine": measured_traffic("exw_engine", name),
                    "workload": "3840x2160 FP16 colour, 64 rectangles, |mv| <= 64 px, occluders ~20%; P_1..P_3"
                                + (" with hole fill" if fill else " without fill (the forward warp)")}


def _extras_batched(b, devc, ex):
    import torch
    from paper_2307_12607_gb300 import scenes
    # batched: 48 streams (12 each of 720p/1080p/1440p/4K), FP16, own scenes
    streams = []
    for sc in scenes.batched_scenes():
        c, d, m = scenes.render(sc, 0.0, np.float16)
        streams.append((torch.from_numpy(c).to(devc), torch.from_numpy(d).to(devc), torch.from_numpy(m).to(devc)))
    outs = [(torch.empty((3,) + tuple(c.shape), dtype=c.dtype, device=devc),
             torch.empty((3,) + tuple(d.shape), dtype=torch.uint8, device=devc)) for c, d, _ in streams]
    wsb = b.workspace(b.exw_batched_workspace_bytes(streams, 3), devc)
    tuner = b.exw_tuner_create()
    b.exw_extrapolate_batched(streams, 3, outs=outs, ws=wsb, tuner=tuner)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.exw_extrapolate_batched(streams, 3, outs=outs, ws=wsb, tuner=tuner)
    ms_b = _event_ms(g.replay, 5)
    wss = {}
    for c, d, _ in streams:
        key = (int(d.shape[1]), int(d.shape[0]))
        if key not in wss:
            wss[key] = b.workspace(b.exw_workspace_bytes(b.OP_EXTRAPOLATE, key[0], key[1], b.F16, 1, 3), devc)

    def single():
        for (c, d, m), (o, k) in zip(streams, outs):
            b.exw_extrapolate(c[None], d[None], m[None], 3, True, o[None], k[None],
                              wss[(int(d.shape[1]), int(d.shape[0]))])
    ms_s = _event_ms(single, 3)
    tot = sum(3 * int(d.shape[0]) * int(d.shape[1]) for _, d, _ in streams)
    ex["batched_48_streams"] = {"value": tot / ms_b / 1e3, "unit": "Mpixel/s", "ms_per_launch": ms_b,
                                "single_stream_loop": tot / ms_s / 1e3, "ratio_vs_single_stream": ms_s / ms_b,
                                "tuner": b.exw_tuner_report(tuner).strip(),
                                "workload": "48 streams: 12 each of 1280x720, 1920x1080, 2560x1440, 3840x2160, FP16 "
                                            "colour, 16-64 objects each, P_1..P_3 with fill, one persistent launch "
                                            "replayed from a CUDA graph"}
    b.exw_tuner_destroy(tuner)


def _extras_diff(b, devc, ex, fused_only=False):
    import torch
    from paper_2307_12607_gb300 import scenes
    # differentiation: 8 frames 1080p FP32, k = 1..3, L2 loss against the ground truth at t + k/4
    sd = scenes.diff_scene()
    frames = [scenes.render(sd, float(f)) for f in range(8)]
    targets = [[torch.from_numpy(scenes.ground_truth(sd, float(f), k)).to(devc) for k in (1, 2, 3)] for f in range(8)]
    fr = [tuple(torch.from_numpy(x).to(devc) for x in f) for f in frames]
    H, W = 1080, 1920
    keys = torch.empty((H, W), dtype=torch.int64, device=devc)
    out = torch.empty((3, H, W), device=devc)
    mask = torch.empty((H, W), dtype=torch.uint8, device=devc)
    gout = torch.empty((3, H, W), device=devc)
    loss = torch.zeros(1, device=devc)
    gc = torch.zeros((3, H, W), device=devc)
    gm = torch.zeros((2, H, W), device=devc)
    wsd = b.workspace(b.exw_workspace_bytes(b.OP_WARP_BACKWARD, W, H), devc)

    def fwd():
        for f in range(8):
            c, d, m = fr[f]
            for k in (1, 2, 3):
                b.exw_splat_motion(d, m, k, 4, keys)
                b.exw_warp(c, d, m, keys, k, 4, out, mask)
                b.exw_l2_loss_grad(out, targets[f][k - 1], mask, gout, loss)

    def fwd_bwd():
        for f in range(8):
            c, d, m = fr[f]
            for k in (1, 2, 3):
                b.exw_splat_motion(d, m, k, 4, keys)
                b.exw_warp(c, d, m, keys, k, 4, out, mask)
                b.exw_l2_loss_grad(out, targets[f][k - 1], mask, gout, loss)
                b.exw_warp_backward(gout, c, d, m, None, k, 4, gc, gm, wsd)   # keys recomputed (checkpointing)
    # the fused, batched pass: one call for the 8 frames and 3 fractions (keys recomputed per frame, each source
    # tile read once, deterministic gradients)
    c_all = torch.stack([f[0] for f in fr])
    d_all = torch.stack([f[1] for f in fr])
    m_all = torch.stack([f[2] for f in fr])
    t_all = torch.stack([torch.stack(t) for t in targets])
    gcb = torch.zeros((8, 3, H, W), device=devc)
    gmb = torch.zeros((8, 2, H, W), device=devc)
    lossb = torch.empty(8, dtype=torch.float64, device=devc)
    wsf = b.workspace(b.exw_workspace_bytes(b.OP_WARP_L2_GRAD, W, H, b.F32, 1, 3), devc)

    def fused():
        b.exw_warp_l2_grad(c_all, d_all, m_all, t_all, 3, grad_color=gcb, grad_mv=gmb, loss=lossb, ws=wsf)
    if fused_only:
        ms_fused = _event_ms(fused, 10)
        ex["fwd_bwd_fused_only"] = {"value": 8 * 3 * W * H / ms_fused / 1e3, "unit": "Mpixel/s",
                                    "ms_per_step": ms_fused}
        return
    ms_f = _event_ms(fwd, 3)
    ms_fb = _event_ms(fwd_bwd, 3)
    ms_fused = _event_ms(fused, 10)
    px = 8 * 3 * W * H
    peak, _ = peaks()
    # algorithmic bytes per source pixel of one frame (3 fractions): the source read once (colour 12, depth 4,
    # motion 8), the three targets (36), the colour and motion gradients read and written once (2 x (12 + 8))
    alg = (12 + 4 + 8) + 3 * 12 + 2 * (12 + 8)
    ex["fwd_bwd_1080p"] = {"value": px / ms_fused / 1e3, "unit": "Mpixel/s", "ms_per_step": ms_fused,
                           "kernel_us": _kernel_means(b, fused),
                           "roofline": {"bound": "hbm", "algorithmic_bytes_per_source_px": alg,
                                        "achieved_gbs": alg * 8 * W * H / (ms_fused / 1e3) / 1e9,
                                        "frac": alg * 8 * W * H / (ms_fused / 1e3) / 1e9 / peak,
                                        "traffic_train_kernel_per_frame": measured_traffic("exw_train",
                                                                                           "fwd_bwd_1080p")},
                           "staged_path": {"value": px / ms_fb / 1e3, "ms_per_step": ms_fb,
                                           "fwd_only": px / ms_f / 1e3, "kernel_us": _kernel_means(b, fwd_bwd)},
                           "ratio_vs_staged": ms_fb / ms_fused,
                           "workload": "8 frames 1920x1080 FP32, k = 1..3: forward warp + L2 loss against the ground "
                                       "truth at t + k/4 + adjoint w.r.t. colour and motion, the splat keys "
                                       "recomputed (activation checkpointing); value: the fused batched pass "
                                       "(exw_warp_l2_grad, one call); staged_path: splat, warp, loss and adjoint "
                                       "per frame and fraction"}


def copy_ceiling(host_in, dev_in, dev_out, host_out, reps=3):
    """The host link's own limit for one end-to-end step: the step's inputs copied host -> device and its outputs
    device -> host as single large cudaMemcpyAsync calls from page-locked memory, each direction alone and both at
    once on two streams (best of ``reps``, CUDA events).  No step can move its bytes faster than the
    both-directions time."""
    import torch
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def h2d():
        for d, h in zip(dev_in, host_in):
            d.copy_(h, non_blocking=True)

    def d2h():
        for h, d in zip(host_out, dev_out):
            h.copy_(d, non_blocking=True)

    def timed(fns_streams):
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            starts, ends = [], []
            for fn, st in fns_streams:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(st):
                    e0.record(st)
                    fn()
                    e1.record(st)
                starts.append(e0)
                ends.append(e1)
            torch.cuda.synchronize()
            t = max(starts[0].elapsed_time(e) for e in ends)
            for e0 in starts[1:]:
                t = max(t, max(e0.elapsed_time(e) for e in ends))
            best = min(best, t)
        return best

    ms_in = timed([(h2d, s_in)])
    ms_out = timed([(d2h, s_out)])
    ms_both = timed([(h2d, s_in), (d2h, s_out)])
    bin_ = sum(t.numel() * t.element_size() for t in host_in)
    bout = sum(t.numel() * t.element_size() for t in host_out)
    return {"h2d_gbs": bin_ / ms_in / 1e6, "d2h_gbs": bout / ms_out / 1e6, "h2d_ms": ms_in, "d2h_ms": ms_out,
            "both_directions_ms": ms_both}


def run_exw(args):
    import torch
    import torch.distributed as dist
    from paper_2307_12607_gb300 import binding as b, build

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    devc = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=devc)
    build.build()

    F = args.frames
    seq = render_sequence(F, replica_seed(rank))
    s, col, dep, mv = seq
    W, H = s.W, s.H
    c = torch.from_numpy(col).to(devc)
    d = torch.from_numpy(dep).to(devc)
    m = torch.from_numpy(mv).to(devc)
    out = torch.empty((F, NFRAC, 3, H, W), dtype=torch.float32, device=devc)
    mask = torch.empty((F, NFRAC, H, W), dtype=torch.uint8, device=devc)
    ws = b.workspace(b.exw_workspace_bytes(b.OP_EXTRAPOLATE, W, H, b.F32, F, NFRAC), devc)
    stream = torch.cuda.current_stream(devc)

    def step():
        b.exw_extrapolate(c, d, m, nfrac=NFRAC, fill=True, out=out, mask=mask, ws=ws)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] if \
        os.environ.get("CUDA_VISIBLE_DEVICES") else str(local)
    launches0 = b.exw_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_index) as clocks:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = b.exw_launch_count() - launches0
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, devc)
    out_px = F * NFRAC * W * H
    value = whole_job_rate(world, out_px, ms / 1e3)

    # per-kernel event timing over a second timed region (same steps), on the launching stream
    b.exw_timing_enable(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    kern = {}
    for name in b.exw_timing_names():
        tot, n = b.exw_timing_query(name)
        kern[name] = (tot, n)
    b.exw_timing_enable(False)
    dom = max(kern, key=lambda k: kern[k][0])
    tot, n = kern[dom]
    avg_ms = tot / n
    c_bytes = 12
    compulsory = (c_bytes + 4 + 8) + NFRAC * (c_bytes + 1)                 # source once, 3 outputs
    per_src_px = {"exw_fused": compulsory, "exw_engine": compulsory,
                  "exw_bounds": 8 + 16.0 / 64,                               # motion read + tile bounds written
                  "exw_fixup": 0.0}
    frames_per_launch = F * args.steps / n   # the engine takes up to 48 frames per launch
    alg_bytes = per_src_px.get(dom, 0.0) * W * H * frames_per_launch
    peak, peak_kind = peaks()
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": (measured_traffic(dom, "sequence_1080p_fp32") or 0.0) * frames_per_launch or None,
                "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": alg_bytes, "mean_launch_ms": avg_ms,
                "source_frames_per_launch": frames_per_launch,
                "kernel_share": {k: v[0] / sum(x[0] for x in kern.values()) for k, v in kern.items()},
                "tile_modes_frame0": b.frame_stats(ws, 0)}

    # end to end through the C ABI with host buffers
    hc = torch.from_numpy(col).pin_memory()
    hd = torch.from_numpy(dep).pin_memory()
    hm = torch.from_numpy(mv).pin_memory()
    ho = torch.empty(out.shape, dtype=out.dtype).pin_memory()
    hmask = torch.empty(mask.shape, dtype=mask.dtype).pin_memory()

    def e2e_step():  # exw_extrapolate_host: copies in, work and copies out overlap chunk by chunk inside the call
        b.exw_extrapolate_host(hc, hd, hm, NFRAC, True, ho, hmask, dev_in=(c, d, m), dev_out=(out, mask), ws=ws,
                               chunk=args.e2e_chunk)

    e2e_step()
    torch.cuda.synchronize()
    barrier()
    e2e_steps = args.e2e_steps if args.e2e_steps > 0 else args.steps
    t0 = time.perf_counter()   # wall clock: the host's own work per call counts too
    enqueue = 0.0
    for _ in range(e2e_steps):
        ta = time.perf_counter()
        e2e_step()
        enqueue += time.perf_counter() - ta
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, devc)
    barrier()
    h2d = (hc.numel() * 4 + hd.numel() * 4 + hm.numel() * 4)
    d2h = ho.numel() * 4 + hmask.numel()
    ceiling = copy_ceiling((hc, hd, hm), (c, d, m), (out, mask), (ho, hmask))

    extras = {} if (args.no_extras or world > 1) else run_extras(b, devc)

    if rank == 0:
        cpu = None if args.no_cpu_baseline else cpu_baseline(args.cpu_seconds, seq)
        line = {"metric": METRIC, "value": value, "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": sequence_config(F, world),
                "gpu_launches": launches, "launches_per_step": launches / args.steps,
                "clocks": clocks.summary(),
                "roofline": roofline,
                "cpu_baseline": cpu,
                "e2e": {"value": whole_job_rate(world, out_px, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3, "steps": e2e_steps,
                        "chunk_frames": args.e2e_chunk, "host_enqueue_ms_per_step": enqueue / e2e_steps * 1e3,
                        "copy_ceiling": ceiling,
                        "frac_of_copy_ceiling": ceiling["both_directions_ms"] / (e2e_s * 1e3)},
                "extras": extras}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.case is not None:
        import torch
        from paper_2307_12607_gb300 import binding as b, build
        build.build()
        devc = torch.device("cuda", 0)
        print(json.dumps({"case": args.case, **run_extras(b, devc, (args.case,))}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_exw(args)


if __name__ == "__main__":
    main()
