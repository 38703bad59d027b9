// exw_batched.cu -- host side of the persistent engine: workspace layout, kernel parameters (per-stream tile
// parameters, TMA maps, the diagonal item queue), launches in groups of at most 48 streams, and the autotuner;
// the entry points exw_extrapolate_batched and the tuner API.  exw_extrapolate (exw_api.cu) runs the frames of a
// sequence through the same engine_run, as streams of one size.
//
// Queue: for d = 0, 1, ... the bounds items of stream d, the plan items of stream d - lag, the tile items of
// stream d - 2 lag and the fix-up items of stream d - 3 lag.  A stage's items thus come after every item of the
// previous stage of the same stream, so the producer's wait for them only spins when they have not finished yet.
//
// The autotuner times the schedule choices -- the shape of the staging windows (two per colour type), the queue
// lag and whether two smooth tiles share a slot -- on the caller's streams the first time it sees a set of sizes,
// outside any stream capture, and keeps the fastest.  Global-memory reads instead of TMA windows (EXW_FLAG_NO_TMA)
// stay a flag: they always lose, so they are not timed.
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "exw_engine.cuh"

namespace exw {

cudaError_t launch_engine(const EngineParams &ep, bool fill, int shape, int grid, cudaStream_t s);

constexpr size_t kEngineHeader = 256;  // status word

// Workspace: status block, one 128-byte header per stream (frame), then the sections of min(n, 48) slots; a
// launch uses slots 0.. for its streams.  shared_size: every stream has specs[0]'s size (a sequence), so every
// slot has that layout.
struct EngineLayout {
    size_t headers;
    int nslots;
    size_t base[kMaxStreams];
    WsLayout l[kMaxStreams];
    size_t total;
};

static EngineLayout engine_layout(const EngineSpec *specs, int n, int nfrac, bool shared_size) {
    EngineLayout b{};
    size_t off = kEngineHeader;
    b.headers = off;
    off += align_up((size_t)n * sizeof(FrameHeader));
    b.nslots = n < kMaxStreams ? n : kMaxStreams;
    for (int i = 0; i < b.nslots; ++i) {
        const exw_frame &f = specs[shared_size ? 0 : i].src;
        b.l[i] = ws_layout(f.W, f.H, 1, nfrac, false, true);
        b.base[i] = off;
        off += b.l[i].total;
    }
    b.total = off;
    return b;
}

size_t engine_workspace_bytes(const EngineSpec *specs, int n, int nfrac, bool shared_size) {
    return engine_layout(specs, n, nfrac, shared_size).total;
}

static PFN_cuTensorMapEncodeTiled_v12000 engine_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
    });
    return fn;
}

// A [planes][H][W] array (planes = 1 gives a 2-D map) with box [planes][by][bx].
static bool encode(PFN_cuTensorMapEncodeTiled_v12000 fn, CUtensorMap *m, CUtensorMapDataType t, const void *base,
                   int W, int H, int planes, size_t esize, int bx, int by) {
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)W * esize, (cuuint64_t)W * H * esize};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, t, planes > 1 ? 3 : 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct Schedule {
    int tma;    // 1: TMA windows where a stream allows them; 0: global-memory reads everywhere
    int lag;    // queue distance between consecutive stages of one stream
    int shape;  // staging window shape (WinShape)
    int pair;   // two smooth tiles of a stream that follow each other share one slot
};

// Kernel parameters for streams [first, first + n) of specs, in slots 0 .. n - 1.  The bounds and plans of
// slot 0 -- the head of the pipeline, which nothing else overlaps -- are computed by the bounds and plan kernels
// before the launch, at their full occupancy; the queue starts with slot 0's tiles.
static bool build_params(EngineParams *ep, const EngineSpec *specs, int first, int n, int nfrac, bool fill, char *ws,
                         const EngineLayout &bl, const Schedule &sc, bool inject) {
    std::memset(ep, 0, sizeof(EngineParams));
    FrameHeader *headers = (FrameHeader *)(ws + bl.headers) + first;
    ep->n = n;
    ep->inject = inject ? 1 : 0;
    ep->pair_smooth = sc.pair;
    ep->ahead = 1ull;
    ep->status = (uint32_t *)ws;
    ep->queue = &headers[0].queue;
    PFN_cuTensorMapEncodeTiled_v12000 fn = engine_encode_fn();
    for (int i = 0; i < n; ++i) {
        const EngineSpec &sp = specs[first + i];
        const exw_frame &f = sp.src;
        const WsLayout &l = bl.l[i];
        char *sb = ws + bl.base[i];
        EngineStream &st = ep->st[i];
        TileParams &p = st.p;
        p.color = f.color;
        p.depth = f.depth;
        p.mv = f.mv;
        p.W = f.W;
        p.H = f.H;
        p.nfrac = nfrac;
        p.L = 2;
        p.k0 = 1;
        for (int j = 0; j < nfrac; ++j) {
            p.out_color[j] = sp.out[j].color;
            p.out_mask[j] = sp.out[j].mask;
        }
        p.tile_bounds = (const float4 *)(sb + l.tile_bounds);
        p.tile_depth = (const float2 *)(sb + l.tile_depth);
        p.region_bounds = (const float4 *)(sb + l.region_bounds);
        p.plans = (TilePlan *)(sb + l.plans);
        p.pdesc = (SplatTile *)(sb + l.pdesc);
        p.nbx = l.nbx;
        p.nby = l.nby;
        p.fh = headers + i;
        p.nodes = (float4 *)(sb + l.nodes);
        p.list = (uint32_t *)(sb + l.list);
        p.fillval = (float4 *)(sb + l.fillval);
        p.coarse = (float4 *)(sb + l.coarse);
        p.n5x = l.n5x;
        p.n5y = l.n5y;
        p.ncoarse = l.ncoarse;
        p.status = ep->status;
        st.cdt = (int)f.cdt;
        const int a = f.cdt == EXW_F16 ? 8 : 4;  // TMA: rows and bases 16-byte aligned
        st.tma = sc.tma && fn != nullptr && (f.W % a) == 0 && ((uintptr_t)f.color & 15u) == 0 &&
                 ((uintptr_t)f.depth & 15u) == 0 && ((uintptr_t)f.mv & 15u) == 0;
        if (st.tma) {
            const int bx = win_x(sc.shape, f.cdt), by = win_y(sc.shape, f.cdt);
            const bool ok =
                encode(fn, &ep->maps[i][0],
                       f.cdt == EXW_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, f.color,
                       f.W, f.H, 3, f.cdt == EXW_F16 ? 2 : 4, bx, by) &&
                encode(fn, &ep->maps[i][1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, f.depth, f.W, f.H, 1, 4, bx, by) &&
                encode(fn, &ep->maps[i][2], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, f.mv, f.W, f.H, 2, 4, bx, by);
            if (!ok) st.tma = 0;
        }
        st.nregions = ceil_div(f.W, 32) * ceil_div(f.H, 32);
        st.ntiles = l.n5x * l.n5y;
        st.nfix = fill ? (int)kFixupItems : 0;
    }
    // diagonal queue
    const int lag = sc.lag < 1 ? 1 : sc.lag;
    int nseg = 0, total = 0;
    for (int dd = 0; dd < n + 3 * lag; ++dd) {
        for (int stage = 0; stage < 4; ++stage) {
            const int s = dd - stage * lag;
            if (s < 0 || s >= n) continue;
            const EngineStream &st = ep->st[s];
            if (stage < 2 && ((ep->ahead >> s) & 1ull)) continue;
            const int cnt = stage == 0   ? ceil_div(st.nregions, kRegionsPerItem)
                            : stage == 1 ? ceil_div(st.ntiles, kPlansPerItem)
                            : stage == 2 ? st.ntiles
                                         : st.nfix;
            if (cnt == 0) continue;
            ep->seg[nseg] = EngineSeg{total, (uint16_t)s, (uint16_t)stage};
            ++nseg;
            total += cnt;
        }
    }
    ep->nseg = nseg;
    ep->total = total;
    return nseg > 0;
}

static int num_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

// All streams, in launches of at most 48.  The headers of all streams are zeroed first (one launch).
static cudaError_t run_all(EngineParams *ep, const EngineSpec *specs, int n, int nfrac, bool fill, char *ws,
                           const EngineLayout &bl, const Schedule &sc, bool inject, cudaStream_t s) {
    cudaError_t e = launch_zero(ws, bl.headers + (size_t)n * sizeof(FrameHeader), s);
    const int sms = num_sms();
    for (int first = 0; first < n && e == cudaSuccess; first += kMaxStreams) {
        const int cnt = n - first < kMaxStreams ? n - first : kMaxStreams;
        if (!build_params(ep, specs, first, cnt, nfrac, fill, ws, bl, sc, inject && first == 0))
            return cudaErrorInvalidValue;
        int tiles = 0;
        for (int i = 0; i < cnt; ++i) tiles += ep->st[i].ntiles;
        for (int i = 0; i < cnt && e == cudaSuccess; ++i) {
            if (!((ep->ahead >> i) & 1ull)) continue;
            const TileParams &p = ep->st[i].p;
            e = launch_bounds(p.depth, p.mv, p.W, p.H, const_cast<float4 *>(p.tile_bounds),
                              const_cast<float2 *>(p.tile_depth), const_cast<float4 *>(p.region_bounds), p.fh, s);
            if (e == cudaSuccess) e = launch_plan(p, (exw_dtype)ep->st[i].cdt, sc.shape, s);
        }
        if (e == cudaSuccess) e = launch_engine(*ep, fill, sc.shape, tiles < sms ? tiles : sms, s);
    }
    return e;
}

}  // namespace exw

using namespace exw;

struct exw_tuner {
    std::mutex mu;
    bool fixed = false;  // exw_tuner_fix: every batch runs this schedule, nothing is timed
    Schedule fix{1, 1, 0, 1};
    struct Entry {
        Schedule best;
        std::vector<std::pair<Schedule, float>> trials;
    };
    std::map<std::string, Entry> table;
};

namespace exw {

static std::string batch_key(const EngineSpec *d, int n, int nfrac, unsigned flags) {
    std::string k = std::to_string(n) + "/" + std::to_string(nfrac) + "/" + std::to_string(flags);
    for (int i = 0; i < n; ++i)
        k += ":" + std::to_string(d[i].src.W) + "x" + std::to_string(d[i].src.H) + "c" + std::to_string(d[i].src.cdt);
    return k;
}

exw_status engine_run(const EngineSpec *specs, int n, int nfrac, unsigned flags, void *ws, size_t ws_bytes,
                      exw_tuner *t, bool shared_size, cudaStream_t s) {
    const EngineLayout bl = engine_layout(specs, n, nfrac, shared_size);
    if (ws == nullptr || ((uintptr_t)ws & 15u) || ws_bytes < bl.total) return EXW_ERR_WORKSPACE;
    if (cudaGetLastError() != cudaSuccess) return EXW_ERR_CUDA;
    const bool fill = (flags & EXW_FLAG_NO_FILL) == 0;
    const char *fault = std::getenv("EXW_FAULT");
    const bool inject = fault != nullptr && std::strcmp(fault, "timeout") == 0;
    Schedule sc{(flags & EXW_FLAG_NO_TMA) ? 0 : 1, 1, 0, 1};
    static thread_local EngineParams ep;  // 32 KB: kept off the stack
    char *wsb = (char *)ws;
    if (t != nullptr && !inject) {
        const std::string key = batch_key(specs, n, nfrac, flags);
        std::unique_lock<std::mutex> g(t->mu);
        auto it = t->table.find(key);
        if (t->fixed) {
            sc = Schedule{sc.tma, t->fix.lag, t->fix.shape, t->fix.pair};
        } else if (it != t->table.end()) {
            sc = it->second.best;
        } else {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
                // Time each schedule on these streams (one warm-up, then the best of two runs); keep the fastest.
                exw_tuner::Entry ent;
                float best = 1e30f;
                cudaEvent_t e0, e1;
                if (cudaEventCreate(&e0) != cudaSuccess) return EXW_ERR_CUDA;
                if (cudaEventCreate(&e1) != cudaSuccess) {
                    cudaEventDestroy(e0);
                    return EXW_ERR_CUDA;
                }
                exw_status st = EXW_OK;
                for (int shape = 0; shape < kWinShapes && st == EXW_OK; ++shape) {
                    for (int lag = 1; lag <= 2 && st == EXW_OK; ++lag) {
                        for (int pair = 1; pair >= 0 && st == EXW_OK; --pair) {
                            const Schedule c{sc.tma, lag, shape, pair};
                            float ms = 1e30f;
                            for (int r = 0; r < 3; ++r) {
                                cudaEventRecord(e0, s);
                                if (run_all(&ep, specs, n, nfrac, fill, wsb, bl, c, false, s) != cudaSuccess) {
                                    st = EXW_ERR_CUDA;
                                    break;
                                }
                                cudaEventRecord(e1, s);
                                if (cudaEventSynchronize(e1) != cudaSuccess) {
                                    st = EXW_ERR_CUDA;
                                    break;
                                }
                                float m = 0.f;
                                cudaEventElapsedTime(&m, e0, e1);
                                if (r > 0 && m < ms) ms = m;
                            }
                            ent.trials.push_back({c, ms});
                            if (ms < best) {
                                best = ms;
                                ent.best = c;
                            }
                        }
                    }
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (st != EXW_OK) return st;
                t->table[key] = ent;
                sc = ent.best;
            }
        }
    }
    return run_all(&ep, specs, n, nfrac, fill, wsb, bl, sc, inject, s) == cudaSuccess ? EXW_OK : EXW_ERR_CUDA;
}

}  // namespace exw

namespace exw {
// "FP32 56x48 / FP16 64x56": the staging window of each colour type for a shape.
static std::string shape_name(int shape) {
    char b[64];
    std::snprintf(b, sizeof b, "FP32 %dx%d / FP16 %dx%d", win_x(shape, EXW_F32), win_y(shape, EXW_F32),
                  win_x(shape, EXW_F16), win_y(shape, EXW_F16));
    return b;
}
}  // namespace exw

extern "C" {

exw_tuner *exw_tuner_create(void) { return new exw_tuner(); }

exw_status exw_tuner_fix(exw_tuner *t, int shape, int lag, int pair) {
    if (t == nullptr || shape < 0 || shape >= kWinShapes || lag < 1 || lag > 4 || pair < 0 || pair > 1)
        return EXW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(t->mu);
    t->fixed = true;
    t->fix = Schedule{1, lag, shape, pair};
    return EXW_OK;
}

void exw_tuner_destroy(exw_tuner *t) { delete t; }

size_t exw_tuner_report(const exw_tuner *t, char *buf, size_t len) {
    std::string r;
    if (t != nullptr) {
        exw_tuner *tt = const_cast<exw_tuner *>(t);
        std::lock_guard<std::mutex> g(tt->mu);
        for (auto &kv : tt->table) {
            const Schedule &bs = kv.second.best;
            r += "streams " + kv.first.substr(0, kv.first.find(':')) + ": best window " + shape_name(bs.shape) +
                 " lag=" + std::to_string(bs.lag) + " pair=" + std::to_string(bs.pair) + " (";
            for (size_t i = 0; i < kv.second.trials.size(); ++i) {
                const Schedule &c = kv.second.trials[i].first;
                char tmp[128];
                std::snprintf(tmp, sizeof tmp, "%swindow %s lag %d pair %d: %.3f ms", i ? ", " : "",
                              shape_name(c.shape).c_str(), c.lag, c.pair, kv.second.trials[i].second);
                r += tmp;
            }
            r += ")\n";
        }
    }
    if (buf != nullptr && len > 0) {
        const size_t c = r.size() < len - 1 ? r.size() : len - 1;
        std::memcpy(buf, r.data(), c);
        buf[c] = '\0';
    }
    return r.size() + 1;
}

static void specs_from(const exw_stream_desc *d, int n, std::vector<EngineSpec> &out) {
    out.resize((size_t)n);
    for (int i = 0; i < n; ++i) {
        out[i].src = d[i].src;
        for (int j = 0; j < EXW_MAX_FRAC; ++j) out[i].out[j] = d[i].out[j];
    }
}

size_t exw_batched_workspace_bytes(const exw_stream_desc *d, int n, int nfrac) {
    if (d == nullptr || n < 1 || n > kMaxStreams || nfrac < 1 || nfrac > EXW_MAX_FRAC) return 0;
    for (int i = 0; i < n; ++i)
        if (!size_ok(d[i].src.W, d[i].src.H)) return 0;
    std::vector<EngineSpec> specs;
    specs_from(d, n, specs);
    return engine_workspace_bytes(specs.data(), n, nfrac, false);
}

exw_status exw_extrapolate_batched(const exw_stream_desc *d, int n, int nfrac, unsigned flags, void *ws,
                                   size_t ws_bytes, exw_tuner *t, exw_stream_t stream) {
    if (d == nullptr || n < 1 || nfrac < 1 || nfrac > EXW_MAX_FRAC || (flags & ~(EXW_FLAG_NO_FILL | EXW_FLAG_NO_TMA)))
        return EXW_ERR_INVALID_ARG;
    if (n > kMaxStreams) return EXW_ERR_UNSUPPORTED;
    for (int i = 0; i < n; ++i) {
        const exw_frame &f = d[i].src;
        const uintptr_t cs = f.cdt == EXW_F16 ? 2 : 4;
        if (!size_ok(f.W, f.H) || !dtype_ok(f.cdt) ||
            f.color == nullptr || f.depth == nullptr || f.mv == nullptr || ((uintptr_t)f.color & (cs - 1)) ||
            ((uintptr_t)f.depth & 3u) || ((uintptr_t)f.mv & 3u))
            return EXW_ERR_INVALID_ARG;
        for (int j = 0; j < nfrac; ++j)
            if (d[i].out[j].color == nullptr || d[i].out[j].mask == nullptr ||
                ((uintptr_t)d[i].out[j].color & (cs - 1)))
                return EXW_ERR_INVALID_ARG;
    }
    std::vector<EngineSpec> specs;
    specs_from(d, n, specs);
    return engine_run(specs.data(), n, nfrac, flags, ws, ws_bytes, t, false, (cudaStream_t)stream);
}

}  // extern "C"
