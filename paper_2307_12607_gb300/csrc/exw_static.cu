// exw_static.cu -- exw_fill_holes_static: the hole fill with its scratch in a fixed device array.
//
// Some callers cannot allocate device memory at the time they fill a frame: a renderer that reserves all of its
// GPU memory up front and forbids allocation inside the frame loop, a plugin that runs inside a host application
// whose allocator it may not call, or code that only receives raw device pointers from elsewhere.  For them the
// fill's scratch (pyramid nodes, the list of tiles without a valid pixel, their fill values, the coarse levels and
// the per-call counters) lives in one file-scope __device__ array of fixed size instead of a caller workspace.
// The array occupies kStaticScratchBytes on every GPU that loads this library, until the process exits.
#include <mutex>

#include "exw_internal.h"

namespace exw {

// Largest frame: at most kStaticMaxTiles fill tiles of 32 x 32 pixels (4096 x 4096, or 8192 x 2048, ...).
constexpr int kStaticMaxTiles = 16384;
constexpr size_t kStaticScratchBytes = 768u * 1024u;

static __device__ __align__(256) unsigned char g_fill_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void *g_static_ptr[64] = {};  // device address of g_fill_scratch, per device ordinal

// The device address of the scratch array on the current device.  In host code g_fill_scratch is only a
// host-side stand-in for the symbol, so the address comes from cudaGetSymbolAddress, once per device.
static cudaError_t static_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_static_mu);
    if (g_static_ptr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fill_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

}  // namespace exw

using namespace exw;

extern "C" exw_status exw_fill_holes_static(void *color, exw_dtype cdt, const uint8_t *mask, int W, int H,
                                            exw_stream_t stream) {
    if (W < 1 || H < 1 || W > 16384 || H > 16384 || (cdt != EXW_F32 && cdt != EXW_F16) || color == nullptr ||
        mask == nullptr || ((uintptr_t)color & (cdt == EXW_F16 ? 1u : 3u)) != 0)
        return EXW_ERR_INVALID_ARG;
    // Fill-only layout: status word, one frame header, then per-tile nodes, invalid-tile list, fill values and the
    // coarse pyramid levels (the motion-bounds tiles of the general workspace are not needed here).
    WsLayout l{};
    l.n5x = ceil_div(W, 32);
    l.n5y = ceil_div(H, 32);
    l.ncoarse = coarse_nodes(l.n5x, l.n5y);
    const size_t n5 = (size_t)l.n5x * l.n5y;
    if (n5 > (size_t)kStaticMaxTiles) return EXW_ERR_WORKSPACE;
    l.headers = kAlign;
    l.tile_bounds = l.headers + kAlign;
    l.nodes = l.tile_bounds;
    l.list = l.nodes + align_up(n5 * 16);
    l.fillval = l.list + align_up(n5 * 4);
    l.coarse = l.fillval + align_up(n5 * 16);
    l.total = l.coarse + align_up((size_t)(l.ncoarse > 0 ? l.ncoarse : 1) * 16);
    if (l.total > kStaticScratchBytes) return EXW_ERR_WORKSPACE;
    if (cudaGetLastError() != cudaSuccess) return EXW_ERR_CUDA;
    void *ws = nullptr;
    if (static_scratch(&ws) != cudaSuccess) return EXW_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    char *b = (char *)ws;
    TileParams p{};
    p.W = W;
    p.H = H;
    p.nfrac = 1;
    p.mask_in = mask;
    p.out_color[0] = color;
    p.fh = (FrameHeader *)(b + l.headers);
    p.nodes = (float4 *)(b + l.nodes);
    p.list = (uint32_t *)(b + l.list);
    p.fillval = (float4 *)(b + l.fillval);
    p.coarse = (float4 *)(b + l.coarse);
    p.n5x = l.n5x;
    p.n5y = l.n5y;
    p.ncoarse = l.ncoarse;
    p.status = (uint32_t *)ws;
    // The array keeps the previous call's contents: the status word and the counters must start at zero.
    cudaError_t e = launch_zero(ws, l.headers + sizeof(FrameHeader), s);
    if (e == cudaSuccess) e = launch_fill_tiles(p, cdt, s);
    if (e == cudaSuccess) e = launch_fixup(p, cdt, s);
    return e == cudaSuccess ? EXW_OK : EXW_ERR_CUDA;
}
