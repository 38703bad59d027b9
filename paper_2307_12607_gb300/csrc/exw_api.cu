// exw_api.cu -- the extern "C" entry points of libexw: argument checks, workspace carving, launches.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "exw_internal.h"

namespace exw {

// ------------------------------------------------------------------------------------------------------------
// Kernel timing: CUDA event pairs on the launching stream around every launch, while enabled.
// ------------------------------------------------------------------------------------------------------------
struct TimedLaunch {
    std::string name;
    cudaEvent_t start, stop;
};
static std::mutex g_tmu;
static bool g_timing = false;
static std::vector<TimedLaunch> g_timed;
static std::vector<cudaEvent_t> g_event_pool;
static std::atomic<uint64_t> g_launches{0};

static cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void timing_begin(const char *name, cudaStream_t s) {
    std::lock_guard<std::mutex> g(g_tmu);
    if (!g_timing) return;
    TimedLaunch t{name, take_event(), take_event()};
    if (t.start == nullptr || t.stop == nullptr) return;
    cudaEventRecord(t.start, s);
    g_timed.push_back(t);
}

void timing_end(const char *name, cudaStream_t s) {
    std::lock_guard<std::mutex> g(g_tmu);
    if (!g_timing || g_timed.empty() || g_timed.back().name != name) return;
    cudaEventRecord(g_timed.back().stop, s);
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }


static TileParams tile_params(const WsLayout &l, void *ws, int W, int H, int nfrac, int L, int k0, int frame) {
    TileParams p{};
    char *b = (char *)ws;
    p.W = W;
    p.H = H;
    p.nfrac = nfrac;
    p.L = L;
    p.k0 = k0;
    p.tile_bounds = (const float4 *)(b + l.tile_bounds);
    p.tile_depth = (const float2 *)(b + l.tile_depth);
    p.region_bounds = (const float4 *)(b + l.region_bounds);
    p.plans = (TilePlan *)(b + l.plans);
    p.nbx = l.nbx;
    p.nby = l.nby;
    p.fh = (FrameHeader *)(b + l.headers) + frame;
    p.nodes = (float4 *)(b + l.nodes);
    p.list = (uint32_t *)(b + l.list);
    p.fillval = (float4 *)(b + l.fillval);
    p.coarse = (float4 *)(b + l.coarse);
    p.n5x = l.n5x;
    p.n5y = l.n5y;
    p.ncoarse = l.ncoarse;
    p.status = (uint32_t *)ws;
    return p;
}

// Workspace of exw_warp_recursive: the keys of the current step, two ping-pong copies of the carried depth and
// motion, then the fill's workspace.
struct RecursiveLayout {
    size_t keys, depth[2], mv[2], fill, total;
};
static RecursiveLayout recursive_layout(int W, int H) {
    const size_t px = (size_t)W * H;
    RecursiveLayout r{};
    size_t off = 0;
    r.keys = off;
    off += align_up(px * 8);
    for (int i = 0; i < 2; ++i) {
        r.depth[i] = off;
        off += align_up(px * 4);
        r.mv[i] = off;
        off += align_up(px * 8);
    }
    r.fill = off;
    off += ws_layout(W, H, 1, 1, false).total;
    r.total = off;
    return r;
}

size_t recursive_workspace_bytes(int W, int H) { return recursive_layout(W, H).total; }

}  // namespace exw

using namespace exw;

extern "C" {

const char *exw_status_string(exw_status s) {
    switch (s) {
        case EXW_OK: return "EXW_OK";
        case EXW_ERR_INVALID_ARG: return "EXW_ERR_INVALID_ARG: null, misaligned or out-of-range argument";
        case EXW_ERR_UNSUPPORTED: return "EXW_ERR_UNSUPPORTED: valid but unimplemented combination";
        case EXW_ERR_CUDA: return "EXW_ERR_CUDA: a CUDA call or kernel launch failed";
        case EXW_ERR_TIMEOUT: return "EXW_ERR_TIMEOUT: a bounded device-side wait ran out";
        case EXW_ERR_WORKSPACE: return "EXW_ERR_WORKSPACE: workspace too small or misaligned";
    }
    return "EXW_ERR_UNKNOWN";
}

int exw_version(void) { return 100; }

size_t exw_workspace_bytes(exw_op op, int W, int H, exw_dtype cdt, int nframes, int nfrac) {
    if (!size_ok(W, H) || !dtype_ok(cdt)) return 0;
    switch (op) {
        case EXW_OP_MOTION_BOUNDS:
        case EXW_OP_FILL_HOLES: return ws_layout(W, H, 1, 1, false).total;
        case EXW_OP_EXTRAPOLATE: {
            if (nframes < 1 || nfrac < 1 || nfrac > EXW_MAX_FRAC) return 0;
            EngineSpec sp{};
            sp.src.W = W;
            sp.src.H = H;
            sp.src.cdt = cdt;
            std::vector<EngineSpec> one(1, sp);
            return engine_workspace_bytes(one.data(), nframes, nfrac, true);
        }
        case EXW_OP_WARP_BACKWARD: return ws_layout(W, H, 1, 1, true).total;
        case EXW_OP_STATS: return stats_workspace_bytes();
        case EXW_OP_WARP_RECURSIVE: return recursive_workspace_bytes(W, H);
        case EXW_OP_WARP_L2_GRAD:
            if (nfrac < 1 || nfrac > EXW_MAX_FRAC) return 0;
            return train_workspace_bytes(W, H, nfrac);
    }
    return 0;
}

exw_status exw_carry_motion(const uint64_t *keys, const uint8_t *mask, const float *depth, const float *mv, int W,
                            int H, float *depth_out, float *mv_out, exw_stream_t stream) {
    if (!size_ok(W, H) || !aligned(keys, 8) || !aligned(mask, 1) || !aligned(depth, 4) || !aligned(mv, 4) ||
        !aligned(depth_out, 4) || !aligned(mv_out, 4))
        return EXW_ERR_INVALID_ARG;
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
    return launch_carry_motion(keys, mask, depth, mv, W, H, depth_out, mv_out, (cudaStream_t)stream) == cudaSuccess
               ? EXW_OK
               : EXW_ERR_CUDA;
}

exw_status exw_mv_variance(const float *mv, int W, int H, double *out, void *ws, size_t ws_bytes,
                           exw_stream_t stream) {
    if (!size_ok(W, H) || !aligned(mv, 4) || !aligned(out, 8)) return EXW_ERR_INVALID_ARG;
    if (!aligned16(ws) || ws_bytes < stats_workspace_bytes()) return EXW_ERR_WORKSPACE;
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
    return launch_mv_variance(mv, W, H, out, ws, (cudaStream_t)stream) == cudaSuccess ? EXW_OK : EXW_ERR_CUDA;
}

exw_status exw_ssim(const void *a, const void *b, exw_dtype cdt, int W, int H, double *out, void *ws,
                    size_t ws_bytes, exw_stream_t stream) {
    if (!size_ok(W, H) || W < 11 || H < 11 || !dtype_ok(cdt) || !aligned(a, csize(cdt)) || !aligned(b, csize(cdt)) ||
        !aligned(out, 8))
        return EXW_ERR_INVALID_ARG;
    if (!aligned16(ws) || ws_bytes < stats_workspace_bytes()) return EXW_ERR_WORKSPACE;
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
    return launch_ssim(a, b, cdt, W, H, out, ws, (cudaStream_t)stream) == cudaSuccess ? EXW_OK : EXW_ERR_CUDA;
}

exw_status exw_color_mse(const void *a, const void *b, exw_dtype cdt, int W, int H, double *out, void *ws,
                         size_t ws_bytes, exw_stream_t stream) {
    if (!size_ok(W, H) || !dtype_ok(cdt) || !aligned(a, csize(cdt)) || !aligned(b, csize(cdt)) || !aligned(out, 8))
        return EXW_ERR_INVALID_ARG;
    if (!aligned16(ws) || ws_bytes < stats_workspace_bytes()) return EXW_ERR_WORKSPACE;
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
    return launch_color_mse(a, b, cdt, W, H, out, ws, (cudaStream_t)stream) == cudaSuccess ? EXW_OK : EXW_ERR_CUDA;
}

exw_status exw_psnr(const void *a, const void *b, exw_dtype cdt, int W, int H, double *out, void *ws, size_t ws_bytes,
                    exw_stream_t stream) {
    if (!size_ok(W, H) || !dtype_ok(cdt) || !aligned(a, csize(cdt)) || !aligned(b, csize(cdt)) || !aligned(out, 8))
        return EXW_ERR_INVALID_ARG;
    if (!aligned16(ws) || ws_bytes < stats_workspace_bytes()) return EXW_ERR_WORKSPACE;
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
    return from_cuda(launch_color_mse(a, b, cdt, W, H, out, ws, (cudaStream_t)stream, true));
}

exw_status exw_motion_bounds(const float *depth, const float *mv, int W, int H, float *tile_bounds,
                             float *frame_bounds, void *ws, size_t ws_bytes, exw_stream_t stream) {
    if (!size_ok(W, H) || !aligned(depth, 4) || !aligned(mv, 4) || !aligned(frame_bounds, 4) ||
        (tile_bounds && !aligned16(tile_bounds)))
        return EXW_ERR_INVALID_ARG;
    const WsLayout l = ws_layout(W, H, 1, 1, false);
    if (!aligned16(ws) || ws_bytes < l.total) return EXW_ERR_WORKSPACE;
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    char *b = (char *)ws;
    FrameHeader *fh = (FrameHeader *)(b + l.headers);
    float4 *tb = tile_bounds ? (float4 *)tile_bounds : (float4 *)(b + l.tile_bounds);
    cudaError_t e = launch_zero(ws, l.headers + sizeof(FrameHeader), s);
    if (e == cudaSuccess)
        e = launch_bounds(depth, mv, W, H, tb, (float2 *)(b + l.tile_depth), (float4 *)(b + l.region_bounds), fh, s);
    if (e == cudaSuccess) e = launch_bounds_finalize(fh, frame_bounds, s);
    return from_cuda(e);
}

exw_status exw_splat_motion(const float *depth, const float *mv, int W, int H, int k, int denom, uint64_t *keys,
                            exw_stream_t stream) {
    const int L = log2_pow2(denom);
    if (!size_ok(W, H) || L < 0 || k < 0 || k > denom || !aligned(depth, 4) || !aligned(mv, 4) || !aligned(keys, 8))
        return EXW_ERR_INVALID_ARG;
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_clear_keys(keys, (size_t)W * H, s);
    if (e == cudaSuccess) e = launch_splat_global(depth, mv, W, H, k, L, keys, s);
    return from_cuda(e);
}

exw_status exw_warp(const void *color, exw_dtype cdt, const float *depth, const float *mv, const uint64_t *keys,
                    int W, int H, int k, int denom, void *out_color, uint8_t *mask, exw_stream_t stream) {
    const int L = log2_pow2(denom);
    if (!size_ok(W, H) || L < 0 || k < 0 || k > denom || !dtype_ok(cdt) || !aligned(color, csize(cdt)) ||
        !aligned(depth, 4) || !aligned(mv, 4) || !aligned(keys, 8) || !aligned(out_color, csize(cdt)) ||
        !aligned(mask, 1))
        return EXW_ERR_INVALID_ARG;
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
    TileParams p{};
    p.color = color;
    p.depth = depth;
    p.mv = mv;
    p.keys = keys;
    p.W = W;
    p.H = H;
    p.nfrac = 1;
    p.L = L;
    p.k0 = k;
    p.out_color[0] = out_color;
    p.out_mask[0] = mask;
    p.n5x = ceil_div(W, 32);
    p.n5y = ceil_div(H, 32);
    return from_cuda(launch_warp_tiles(p, cdt, (cudaStream_t)stream));
}

exw_status exw_fill_holes(void *color, exw_dtype cdt, const uint8_t *mask, int W, int H, void *ws, size_t ws_bytes,
                          exw_stream_t stream) {
    if (!size_ok(W, H) || !dtype_ok(cdt) || !aligned(color, csize(cdt)) || !aligned(mask, 1))
        return EXW_ERR_INVALID_ARG;
    const WsLayout l = ws_layout(W, H, 1, 1, false);
    if (!aligned16(ws) || ws_bytes < l.total) return EXW_ERR_WORKSPACE;
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    TileParams p = tile_params(l, ws, W, H, 1, 0, 0, 0);
    p.mask_in = mask;
    p.out_color[0] = color;
    cudaError_t e = launch_zero(ws, l.headers + sizeof(FrameHeader), s);
    if (e == cudaSuccess) e = launch_fill_tiles(p, cdt, s);
    if (e == cudaSuccess) e = launch_fixup(p, cdt, s);
    return from_cuda(e);
}

exw_status exw_extrapolate(const exw_frame *frames, int nframes, int nfrac, unsigned flags, exw_frame_out *out,
                           void *ws, size_t ws_bytes, exw_stream_t stream) {
    if (frames == nullptr || out == nullptr || nframes < 1 || nfrac < 1 || nfrac > EXW_MAX_FRAC ||
        (flags & ~(EXW_FLAG_NO_FILL | EXW_FLAG_NO_TMA)) != 0)
        return EXW_ERR_INVALID_ARG;
    const int W = frames[0].W, H = frames[0].H;
    const exw_dtype cdt = frames[0].cdt;
    if (!size_ok(W, H) || !dtype_ok(cdt)) return EXW_ERR_INVALID_ARG;
    for (int f = 0; f < nframes; ++f) {
        const exw_frame &fr = frames[f];
        if (fr.W != W || fr.H != H || fr.cdt != cdt || !aligned(fr.color, csize(cdt)) || !aligned(fr.depth, 4) ||
            !aligned(fr.mv, 4))
            return EXW_ERR_INVALID_ARG;
        for (int j = 0; j < nfrac; ++j) {
            const exw_frame_out &o = out[(size_t)f * nfrac + j];
            if (!aligned(o.color, csize(cdt)) || !aligned(o.mask, 1)) return EXW_ERR_INVALID_ARG;
        }
    }
    std::vector<EngineSpec> specs((size_t)nframes);
    for (int f = 0; f < nframes; ++f) {
        specs[f].src = frames[f];
        for (int j = 0; j < nfrac; ++j) specs[f].out[j] = out[(size_t)f * nfrac + j];
    }
    return engine_run(specs.data(), nframes, nfrac, flags, ws, ws_bytes, nullptr, true, (cudaStream_t)stream);
}

// Host-memory variant: copies in on one stream, the work on the caller's, copies out on another, chunk by chunk.
namespace {
struct HostStreams {
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t start = nullptr, copied = nullptr, done = nullptr, back = nullptr;
};
std::mutex g_host_mu;
HostStreams g_host[16];

bool host_streams(HostStreams *&hs) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return false;
    std::lock_guard<std::mutex> lock(g_host_mu);
    HostStreams &h = g_host[dev];
    if (h.in == nullptr) {
        if (cudaStreamCreateWithFlags(&h.in, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&h.out, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.start, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.copied, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.back, cudaEventDisableTiming) != cudaSuccess) {
            h = HostStreams{};
            return false;
        }
    }
    hs = &h;
    return true;
}

// One copy per run of consecutive items whose source and destination both follow the previous item's.
struct Run {
    char *dst = nullptr;
    const char *src = nullptr;
    size_t bytes = 0;
};
cudaError_t copy_run(Run &r, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s,
                     bool flush) {
    cudaError_t e = cudaSuccess;
    if (r.bytes != 0 && (flush || (char *)dst != r.dst + r.bytes || (const char *)src != r.src + r.bytes)) {
        e = cudaMemcpyAsync(r.dst, r.src, r.bytes, kind, s);
        r = Run{};
    }
    if (flush || e != cudaSuccess) return e;
    if (r.bytes == 0) r = Run{(char *)dst, (const char *)src, 0};
    r.bytes += bytes;
    return cudaSuccess;
}
}  // namespace

exw_status exw_extrapolate_host(const exw_frame *frames_host, const exw_frame *frames_dev, int nframes, int nfrac,
                                unsigned flags, const exw_frame_out *out_host, const exw_frame_out *out_dev, int chunk,
                                void *ws, size_t ws_bytes, exw_stream_t stream) {
    if (frames_host == nullptr || frames_dev == nullptr || out_host == nullptr || nframes < 1 || nfrac < 1 ||
        nfrac > EXW_MAX_FRAC || chunk < 0)
        return EXW_ERR_INVALID_ARG;
    if (chunk == 0) chunk = 8;
    const int W = frames_dev[0].W, H = frames_dev[0].H;
    const exw_dtype cdt = frames_dev[0].cdt;
    if (!size_ok(W, H) || !dtype_ok(cdt)) return EXW_ERR_INVALID_ARG;
    for (int f = 0; f < nframes; ++f) {
        const exw_frame &h = frames_host[f];
        if (h.W != W || h.H != H || h.cdt != cdt || h.color == nullptr || h.depth == nullptr || h.mv == nullptr)
            return EXW_ERR_INVALID_ARG;
        for (int j = 0; j < nfrac; ++j)
            if (out_host[(size_t)f * nfrac + j].color == nullptr || out_host[(size_t)f * nfrac + j].mask == nullptr)
                return EXW_ERR_INVALID_ARG;
    }
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
    // out_dev == NULL: the engine writes every output straight into the (page-locked, device-mapped) host buffers
    std::vector<exw_frame_out> direct;
    if (out_dev == nullptr) {
        direct.resize((size_t)nframes * nfrac);
        for (size_t q = 0; q < direct.size(); ++q) {
            void *c = nullptr, *m = nullptr;
            if (cudaHostGetDevicePointer(&c, out_host[q].color, 0) != cudaSuccess ||
                cudaHostGetDevicePointer(&m, out_host[q].mask, 0) != cudaSuccess) {
                cudaGetLastError();
                return EXW_ERR_INVALID_ARG;
            }
            direct[q] = exw_frame_out{c, (uint8_t *)m};
        }
    }
    HostStreams *hs = nullptr;
    if (!host_streams(hs)) return EXW_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t px = (size_t)W * H, cb = px * 3 * csize(cdt);
    // the copies in start after the work already queued on the caller's stream
    cudaError_t e = cudaEventRecord(hs->start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hs->in, hs->start, 0);
    for (int f0 = 0; f0 < nframes && e == cudaSuccess; f0 += chunk) {
        const int n = nframes - f0 < chunk ? nframes - f0 : chunk;
        Run rc, rd, rm;
        for (int f = f0; f < f0 + n && e == cudaSuccess; ++f) {
            const exw_frame &h = frames_host[f], &d = frames_dev[f];
            // the device descriptors are the staging buffers this call fills
            e = copy_run(rc, const_cast<void *>(d.color), h.color, cb, cudaMemcpyHostToDevice, hs->in, false);
            if (e == cudaSuccess)
                e = copy_run(rd, const_cast<float *>(d.depth), h.depth, px * 4, cudaMemcpyHostToDevice, hs->in, false);
            if (e == cudaSuccess)
                e = copy_run(rm, const_cast<float *>(d.mv), h.mv, px * 8, cudaMemcpyHostToDevice, hs->in, false);
        }
        for (Run *r : {&rc, &rd, &rm})
            if (e == cudaSuccess) e = copy_run(*r, nullptr, nullptr, 0, cudaMemcpyHostToDevice, hs->in, true);
        if (e == cudaSuccess) e = cudaEventRecord(hs->copied, hs->in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, hs->copied, 0);
        if (e != cudaSuccess) break;
        exw_frame_out *od = out_dev != nullptr ? const_cast<exw_frame_out *>(out_dev) : direct.data();
        const exw_status st = exw_extrapolate(frames_dev + f0, n, nfrac, flags, od + (size_t)f0 * nfrac, ws, ws_bytes,
                                              stream);
        if (st != EXW_OK) {  // the copies already queued still finish before the caller's stream does
            if (cudaEventRecord(hs->copied, hs->in) == cudaSuccess) cudaStreamWaitEvent(s, hs->copied, 0);
            if (cudaEventRecord(hs->back, hs->out) == cudaSuccess) cudaStreamWaitEvent(s, hs->back, 0);
            return st;
        }
        if (out_dev == nullptr) continue;
        e = cudaEventRecord(hs->done, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(hs->out, hs->done, 0);
        Run oc, om;
        for (int q = f0 * nfrac; q < (f0 + n) * nfrac && e == cudaSuccess; ++q) {
            e = copy_run(oc, out_host[q].color, out_dev[q].color, cb, cudaMemcpyDeviceToHost, hs->out, false);
            if (e == cudaSuccess)
                e = copy_run(om, out_host[q].mask, out_dev[q].mask, px, cudaMemcpyDeviceToHost, hs->out, false);
        }
        for (Run *r : {&oc, &om})
            if (e == cudaSuccess) e = copy_run(*r, nullptr, nullptr, 0, cudaMemcpyDeviceToHost, hs->out, true);
    }
    // the caller's stream completes once the last outputs are in host memory -- and, after an error, once every
    // copy already queued on the internal streams has finished
    cudaError_t f = cudaEventRecord(hs->copied, hs->in);
    if (f == cudaSuccess) f = cudaStreamWaitEvent(s, hs->copied, 0);
    if (out_dev != nullptr) {
        if (f == cudaSuccess) f = cudaEventRecord(hs->back, hs->out);
        if (f == cudaSuccess) f = cudaStreamWaitEvent(s, hs->back, 0);
    }
    return e == cudaSuccess && f == cudaSuccess ? EXW_OK : EXW_ERR_CUDA;
}

exw_status exw_warp_recursive(const void *color, exw_dtype cdt, const float *depth, const float *mv, int W, int H,
                              int steps, unsigned flags, exw_frame_out *out, void *ws, size_t ws_bytes,
                              exw_stream_t stream) {
    if (!size_ok(W, H) || !dtype_ok(cdt) || steps < 1 || steps > 64 || out == nullptr ||
        (flags & ~EXW_FLAG_NO_FILL) != 0 || !aligned(color, csize(cdt)) || !aligned(depth, 4) || !aligned(mv, 4))
        return EXW_ERR_INVALID_ARG;
    for (int i = 0; i < steps; ++i)
        if (!aligned(out[i].color, csize(cdt)) || !aligned(out[i].mask, 1)) return EXW_ERR_INVALID_ARG;
    const RecursiveLayout r = recursive_layout(W, H);
    if (!aligned16(ws) || ws_bytes < r.total) return EXW_ERR_WORKSPACE;
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    char *b = (char *)ws;
    uint64_t *keys = (uint64_t *)(b + r.keys);
    const WsLayout fl = ws_layout(W, H, 1, 1, false);
    void *fws = b + r.fill;
    const void *c = color;
    const float *d = depth, *m = mv;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < steps && e == cudaSuccess; ++i) {
        // step i: warp the previous frame (the source for i = 0) by a quarter step of the motion it carries
        e = launch_clear_keys(keys, (size_t)W * H, s);
        if (e == cudaSuccess) e = launch_splat_global(d, m, W, H, 1, 2, keys, s);
        TileParams p{};
        p.color = c;
        p.depth = d;
        p.mv = m;
        p.keys = keys;
        p.W = W;
        p.H = H;
        p.nfrac = 1;
        p.L = 2;
        p.k0 = 1;
        p.out_color[0] = out[i].color;
        p.out_mask[0] = out[i].mask;
        p.n5x = ceil_div(W, kFillTileSide);
        p.n5y = ceil_div(H, kFillTileSide);
        if (e == cudaSuccess) e = launch_warp_tiles(p, cdt, s);
        if (e == cudaSuccess && (flags & EXW_FLAG_NO_FILL) == 0) {
            TileParams f = tile_params(fl, fws, W, H, 1, 0, 0, 0);
            f.mask_in = out[i].mask;
            f.out_color[0] = out[i].color;
            e = launch_zero(fws, fl.headers + sizeof(FrameHeader), s);
            if (e == cudaSuccess) e = launch_fill_tiles(f, cdt, s);
            if (e == cudaSuccess) e = launch_fixup(f, cdt, s);
        }
        if (e == cudaSuccess && i + 1 < steps) {  // the warped frame's depth and motion for the next step
            float *dn = (float *)(b + r.depth[i & 1]), *mn = (float *)(b + r.mv[i & 1]);
            e = launch_carry_motion(keys, out[i].mask, d, m, W, H, dn, mn, s);
            d = dn;
            m = mn;
        }
        c = out[i].color;
    }
    return from_cuda(e);
}

exw_status exw_warp_backward(const float *grad_out, const void *color, exw_dtype cdt, const float *depth,
                             const float *mv, const uint64_t *keys, int W, int H, int k, int denom, float *grad_color,
                             float *grad_mv, void *ws, size_t ws_bytes, exw_stream_t stream) {
    const int L = log2_pow2(denom);
    if (!size_ok(W, H) || L < 0 || k < 0 || k > denom || !dtype_ok(cdt) || !aligned(grad_out, 4) ||
        !aligned(color, csize(cdt)) || !aligned(depth, 4) || !aligned(mv, 4) || !aligned(grad_color, 4) ||
        !aligned(grad_mv, 4) || (keys != nullptr && !aligned(keys, 8)))
        return EXW_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t *kp = keys;
    if (kp == nullptr) {
        const WsLayout l = ws_layout(W, H, 1, 1, true);
        if (!aligned16(ws) || ws_bytes < l.total) return EXW_ERR_WORKSPACE;
        if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
        uint64_t *kw = (uint64_t *)((char *)ws + l.keys);
        cudaError_t e = launch_clear_keys(kw, (size_t)W * H, s);
        if (e == cudaSuccess) e = launch_splat_global(depth, mv, W, H, k, L, kw, s);
        if (e != cudaSuccess) return EXW_ERR_CUDA;
        kp = kw;
    } else if (entry_check() != EXW_OK) {
        return EXW_ERR_CUDA;
    }
    return from_cuda(launch_backward(grad_out, color, cdt, depth, mv, kp, W, H, k, L, grad_color, grad_mv, s));
}

exw_status exw_warp_l2_grad(const exw_train_frame *frames, int nframes, int nfrac, double *loss, void *ws,
                            size_t ws_bytes, exw_stream_t stream) {
    if (frames == nullptr || nframes < 1 || nfrac < 1 || nfrac > EXW_MAX_FRAC || !aligned(loss, 8))
        return EXW_ERR_INVALID_ARG;
    const int W = frames[0].src.W, H = frames[0].src.H;
    const exw_dtype cdt = frames[0].src.cdt;
    if (!size_ok(W, H) || !dtype_ok(cdt)) return EXW_ERR_INVALID_ARG;
    for (int f = 0; f < nframes; ++f) {
        const exw_train_frame &t = frames[f];
        if (t.src.W != W || t.src.H != H || t.src.cdt != cdt || !aligned(t.src.color, csize(cdt)) ||
            !aligned(t.src.depth, 4) || !aligned(t.src.mv, 4) || !aligned(t.grad_color, 4) || !aligned(t.grad_mv, 4))
            return EXW_ERR_INVALID_ARG;
        for (int j = 0; j < nfrac; ++j)
            if (!aligned(t.target[j], csize(cdt))) return EXW_ERR_INVALID_ARG;
    }
    if (!aligned16(ws) || ws_bytes < train_workspace_bytes(W, H, nfrac)) return EXW_ERR_WORKSPACE;
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < nframes && e == cudaSuccess; ++f)
        e = launch_train_frame(frames[f], nfrac, loss + f, ws, (cudaStream_t)stream);
    return from_cuda(e);
}

exw_status exw_l2_loss_grad(const void *out, const void *target, exw_dtype cdt, const uint8_t *mask, int W, int H,
                            float *grad_out, float *loss, exw_stream_t stream) {
    if (!size_ok(W, H) || !dtype_ok(cdt) || !aligned(out, csize(cdt)) || !aligned(target, csize(cdt)) ||
        !aligned(mask, 1) || !aligned(grad_out, 4) || !aligned(loss, 4))
        return EXW_ERR_INVALID_ARG;
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
    return from_cuda(launch_l2_loss(out, target, cdt, mask, W, H, grad_out, loss, (cudaStream_t)stream));
}

exw_status exw_device_status(const void *ws, exw_stream_t stream) {
    if (!aligned16(ws)) return EXW_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, ws, sizeof v, cudaMemcpyDeviceToHost, s) != cudaSuccess) return EXW_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return EXW_ERR_CUDA;
    return (exw_status)v;
}

// --- timing --------------------------------------------------------------------------------------------------
void exw_timing_enable(int on) {
    std::lock_guard<std::mutex> g(g_tmu);
    for (auto &t : g_timed) {
        g_event_pool.push_back(t.start);
        g_event_pool.push_back(t.stop);
    }
    g_timed.clear();
    g_timing = on != 0;
}

int exw_timing_query(const char *name, double *total_ms, int *launches) {
    std::lock_guard<std::mutex> g(g_tmu);
    double sum = 0.0;
    int n = 0;
    for (auto &t : g_timed) {
        if (t.name != name) continue;
        if (cudaEventSynchronize(t.stop) != cudaSuccess) return -1;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.start, t.stop) != cudaSuccess) return -1;
        sum += ms;
        ++n;
    }
    if (total_ms) *total_ms = sum;
    if (launches) *launches = n;
    return n > 0 ? 0 : -1;
}

size_t exw_timing_names(char *buf, size_t len) {
    std::lock_guard<std::mutex> g(g_tmu);
    std::vector<std::string> names;
    for (auto &t : g_timed) {
        bool seen = false;
        for (auto &n : names) seen = seen || n == t.name;
        if (!seen) names.push_back(t.name);
    }
    std::string all;
    for (size_t i = 0; i < names.size(); ++i) all += (i ? "," : "") + names[i];
    if (buf && len) {
        const size_t c = all.size() < len - 1 ? all.size() : len - 1;
        std::memcpy(buf, all.data(), c);
        buf[c] = '\0';
    }
    return all.size() + 1;
}

uint64_t exw_launch_count(void) { return g_launches.load(); }

}  // extern "C"
