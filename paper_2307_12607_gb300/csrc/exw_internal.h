// exw_internal.h -- workspace layout and kernel launchers shared by the translation units of libexw.
#pragma once

#include <cstddef>
#include <cstdint>
#include <type_traits>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/exw.h"

namespace exw {

// ------------------------------------------------------------------------------------------------------------
// Argument checks shared by every entry point (the rules of include/exw.h)
// ------------------------------------------------------------------------------------------------------------
constexpr int kMaxSide = 16384;     // largest W or H
constexpr int kFillTileSide = 32;  // side of the fill tiles (pyramid levels 1..5 of one tile)
inline bool aligned(const void *p, uintptr_t a) { return p != nullptr && ((uintptr_t)p & (a - 1)) == 0; }
inline bool aligned16(const void *p) { return aligned(p, 16); }
inline uintptr_t csize(exw_dtype d) { return d == EXW_F16 ? 2 : 4; }
inline bool size_ok(int W, int H) { return W >= 1 && H >= 1 && W <= kMaxSide && H <= kMaxSide; }
inline bool dtype_ok(exw_dtype d) { return d == EXW_F32 || d == EXW_F16; }
inline int log2_pow2(int d) {  // log2 of a power of two in [1, 64]; -1 otherwise
    if (d < 1 || d > 64 || (d & (d - 1)) != 0) return -1;
    int l = 0;
    while ((1 << l) != d) ++l;
    return l;
}
inline exw_status from_cuda(cudaError_t e) { return e == cudaSuccess ? EXW_OK : EXW_ERR_CUDA; }
// A sticky error left by earlier work is reported before anything is enqueued.
inline exw_status entry_check() { return cudaGetLastError() == cudaSuccess ? EXW_OK : EXW_ERR_CUDA; }

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Per-frame bookkeeping, zeroed at the start of every call that uses it.
struct FrameHeader {
    uint32_t acc[4];       // ordered-float maxima of -min mv_x, max mv_x, -min mv_y, max mv_y (0 = none)
    uint32_t done;         // tiles finished (the CTA finishing the last one runs the coarse pyramid)
    uint32_t ninvalid[3];  // fill tiles without any valid pixel, per fraction
    uint32_t cready;       // batched path: the coarse values of this frame are written
    uint32_t queue;        // next tile of the persistent kernel
    uint32_t nmode[6];     // tiles done per plan mode (TilePlan::mode)
    uint32_t bdone;        // batched path: bounds regions finished
    uint32_t pdone;        // batched path: plan groups finished
    uint32_t nlazy[2];     // lazy level-5 nodes a coarse pass computed: smooth tiles, others (from their outputs)
    uint32_t pad[12];
};
static_assert(sizeof(FrameHeader) == 128, "FrameHeader is 128 bytes");

// A candidate 8 x 8 source tile of a target tile's splat: the fractions whose landing rectangle meets the tile's
// region and, for a clean tile (one exact motion, every pixel can land, offsets within int8), its whole-pixel
// offsets per fraction.
struct alignas(16) SplatTile {
    uint16_t bx, by;
    uint8_t fm, clean;
    int8_t ox[3], oy[3];
    int8_t pad[2];
};
static_assert(sizeof(SplatTile) == 16, "one load per descriptor");
constexpr int kPlanDesc = 64;  // candidate descriptors the plan stores per target tile (more: none are stored)

// Per target tile, how the fused pass stages its sources (written by the plan kernel).
struct alignas(16) TilePlan {
    int mode;          // 0 uniform motion, 1 one window, 2 one window per fraction, 3 global memory, 4 nothing
                       // lands, 5 uniform motion over smooth valid sources (every pixel a winner, every tap agrees)
    int wx0, wy0;      // window origin (modes 0 and 1)
    int ndesc;         // candidate source tiles stored in the plan's descriptors (0: more than kPlanDesc)
    int rect[3][4];    // per fraction, landing rectangle x0, x1, y0, y1 (source pixels; empty if x1 < x0)
    uint32_t umx, umy; // the one motion of a uniform tile (float bits)
    int pad1[2];
};
static_assert(sizeof(TilePlan) == 80, "TilePlan is 80 bytes");

// Byte offsets of the workspace sections for nframes frames of W x H with nfrac fractions.
struct WsLayout {
    size_t headers, tile_bounds, tile_depth, region_bounds, plans, pdesc, nodes, list, fillval, coarse, keys, total;
    int nbx, nby;       // motion-bounds tiles
    int n5x, n5y;       // fill tiles (level-5 nodes of the pyramid)
    int ncoarse;        // pyramid nodes above level 5, per fraction
};

inline int coarse_nodes(int n5x, int n5y) {
    int total = 0;
    while (n5x > 1 || n5y > 1) {
        n5x = (n5x + 1) / 2;
        n5y = (n5y + 1) / 2;
        total += n5x * n5y;
    }
    return total;
}

inline WsLayout ws_layout(int W, int H, int nframes, int nfrac, bool with_keys, bool with_desc = false) {
    WsLayout l{};
    l.nbx = ceil_div(W, 8);
    l.nby = ceil_div(H, 8);
    l.n5x = ceil_div(W, 32);
    l.n5y = ceil_div(H, 32);
    l.ncoarse = coarse_nodes(l.n5x, l.n5y);
    const size_t n5 = (size_t)l.n5x * l.n5y;
    size_t off = kAlign;  // first 256 bytes: global status word
    l.headers = off;
    off += align_up((size_t)nframes * sizeof(FrameHeader));
    l.tile_bounds = off;
    off += align_up((size_t)l.nbx * l.nby * 16);
    l.tile_depth = off;
    off += align_up((size_t)l.nbx * l.nby * 8);
    l.region_bounds = off;
    off += align_up(n5 * 16);
    l.plans = off;
    off += align_up(n5 * sizeof(TilePlan));
    l.pdesc = off;  // the plans' candidate descriptors (the persistent engine only)
    if (with_desc) off += align_up(n5 * kPlanDesc * sizeof(SplatTile));
    l.nodes = off;
    off += align_up((size_t)nfrac * n5 * 16);
    l.list = off;
    off += align_up((size_t)nfrac * n5 * 4);
    l.fillval = off;
    off += align_up((size_t)nfrac * n5 * 16);
    l.coarse = off;
    off += align_up((size_t)nfrac * (size_t)(l.ncoarse > 0 ? l.ncoarse : 1) * 16);
    l.keys = off;
    if (with_keys) off += align_up((size_t)W * H * 8);
    l.total = off;
    return l;
}

// Parameters of the per-tile passes (stage (b)+(c) on 32 x 32 tiles).
struct alignas(16) TileParams {
    const void *color;          // source colour (fused/warp) or in-out colour (fill)
    const float *depth;
    const float *mv;
    const uint64_t *keys;       // staged warp: global keys
    const uint8_t *mask_in;     // staged fill: input mask
    int W, H, nfrac, L, k0;     // fractions k0 .. k0 + nfrac - 1 of 2^L
    void *out_color[3];
    uint8_t *out_mask[3];
    const float4 *tile_bounds;
    const float2 *tile_depth;   // per 8 x 8 tile: depth range of its pixels, (-1, -1) if one cannot land
    const float4 *region_bounds;  // per 32 x 32 region (fill tile): motion bounds of its 8 x 8 tiles
    TilePlan *plans;            // [n5] staging plan per target tile (persistent TMA kernel)
    SplatTile *pdesc;           // [n5][kPlanDesc] candidate source tiles per target tile, or null
    int nbx, nby;
    FrameHeader *fh;
    float4 *nodes;              // [nfrac][n5]
    uint32_t *list;             // [nfrac][n5]
    float4 *fillval;            // [nfrac][n5]
    float4 *coarse;             // [nfrac][ncoarse]
    int n5x, n5y, ncoarse;
    uint32_t *status;           // workspace status word (EXW_OK, or EXW_ERR_TIMEOUT from a bounded wait)
};

// Shared-memory source windows of the persistent TMA kernel (x extent, y extent): two shapes per colour type, all
// 64,512 bytes (depth, motion and colour planes); the autotuner picks one per batch.  x is a multiple of 16 bytes
// of every plane (TMA) and at most 64 (a half warp covers a row when the depth plane is rewritten).
constexpr int kWinShapes = 2;
template <int SHAPE> struct WinShape;
template <> struct WinShape<0> {  // the default: wider for FP16
    static constexpr int xf32 = 56, yf32 = 48, xf16 = 64, yf16 = 56;
};
template <> struct WinShape<1> {  // wide FP32, tall FP16
    static constexpr int xf32 = 64, yf32 = 42, xf16 = 56, yf16 = 64;
};
inline int win_x(int shape, exw_dtype cdt) {
    return shape == 0 ? (cdt == EXW_F16 ? WinShape<0>::xf16 : WinShape<0>::xf32)
                      : (cdt == EXW_F16 ? WinShape<1>::xf16 : WinShape<1>::xf32);
}
inline int win_y(int shape, exw_dtype cdt) {
    return shape == 0 ? (cdt == EXW_F16 ? WinShape<0>::yf16 : WinShape<0>::yf32)
                      : (cdt == EXW_F16 ? WinShape<1>::yf16 : WinShape<1>::yf32);
}

// Launchers (exw_fwd.cu, exw_aux.cu, exw_bwd.cu).  Each returns the launch error.
cudaError_t launch_clear_keys(uint64_t *keys, size_t n, cudaStream_t s);
cudaError_t launch_zero(void *p, size_t bytes, cudaStream_t s);
cudaError_t launch_carry_motion(const uint64_t *keys, const uint8_t *mask, const float *depth, const float *mv,
                                int W, int H, float *depth_out, float *mv_out, cudaStream_t s);
cudaError_t launch_splat_global(const float *depth, const float *mv, int W, int H, int k, int L, uint64_t *keys,
                                cudaStream_t s);
cudaError_t launch_bounds(const float *depth, const float *mv, int W, int H, float4 *tile_bounds, float2 *tile_depth,
                          float4 *region_bounds, FrameHeader *fh, cudaStream_t s);
cudaError_t launch_bounds_finalize(const FrameHeader *fh, float *frame_bounds, cudaStream_t s);

cudaError_t launch_plan(const TileParams &p, exw_dtype cdt, int shape, cudaStream_t s);

size_t recursive_workspace_bytes(int W, int H);
size_t train_workspace_bytes(int W, int H, int nfrac);
cudaError_t launch_train_frame(const exw_train_frame &f, int nfrac, double *loss, void *ws, cudaStream_t s);

// Frame statistics (exw_stats.cu): FP64 reductions into a small fixed workspace.
size_t stats_workspace_bytes();
cudaError_t launch_mv_variance(const float *mv, int W, int H, double *out, void *ws, cudaStream_t s);
cudaError_t launch_color_mse(const void *a, const void *b, exw_dtype cdt, int W, int H, double *out, void *ws,
                             cudaStream_t s, bool psnr = false);
cudaError_t launch_ssim(const void *a, const void *b, exw_dtype cdt, int W, int H, double *out, void *ws,
                        cudaStream_t s);
cudaError_t launch_warp_tiles(const TileParams &p, exw_dtype cdt, cudaStream_t s);
cudaError_t launch_fill_tiles(const TileParams &p, exw_dtype cdt, cudaStream_t s);
cudaError_t launch_fixup(const TileParams &p, exw_dtype cdt, cudaStream_t s);
cudaError_t launch_l2_loss(const void *out, const void *target, exw_dtype cdt, const uint8_t *mask, int W, int H,
                           float *grad_out, float *loss, cudaStream_t s);
cudaError_t launch_backward(const float *grad_out, const void *color, exw_dtype cdt, const float *depth,
                            const float *mv, const uint64_t *keys, int W, int H, int k, int L, float *grad_color,
                            float *grad_mv, cudaStream_t s);

// The fused forward pass of exw_extrapolate and exw_extrapolate_batched (exw_batched.cu): one engine launch per
// group of at most 48 frames.  specs[i] = (source frame, its nfrac outputs).
struct EngineSpec {
    exw_frame src;
    exw_frame_out out[EXW_MAX_FRAC];
};
size_t engine_workspace_bytes(const EngineSpec *specs, int n, int nfrac, bool shared_size);
exw_status engine_run(const EngineSpec *specs, int n, int nfrac, unsigned flags, void *ws, size_t ws_bytes,
                      struct exw_tuner *tuner, bool shared_size, cudaStream_t s);

// Launch with programmatic stream serialisation: the grid may be scheduled while the kernel before it on the stream
// is still draining, so it must execute grid_dependency_wait() (exw_device.cuh) before it touches any memory.  The
// arguments are passed by address, not copied (the engine's parameter block is 32 KB), so each must have exactly
// its parameter's type.
template <typename... Params, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                    const Args &...args) {
    static_assert(sizeof...(Params) == sizeof...(Args), "one argument per kernel parameter");
    static_assert((std::is_same<typename std::decay<Params>::type, Args>::value && ...),
                  "each argument has its parameter's exact type");
    void *pargs[] = {const_cast<void *>(static_cast<const void *>(&args))...};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, reinterpret_cast<const void *>(kernel), pargs);
}

// Timing hooks (exw_api.cu): bracket a launch with events when timing is enabled.
void timing_begin(const char *name, cudaStream_t s);
void timing_end(const char *name, cudaStream_t s);
void count_launch();

}  // namespace exw
