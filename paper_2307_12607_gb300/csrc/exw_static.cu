// exw_static.cu -- exw_fill_holes_static: the hole fill with its scratch in a fixed device array.
//
// Some callers cannot allocate device memory at the time they fill a frame: a renderer that reserves all of its
// GPU memory up front and forbids allocation inside the frame loop, a plugin that runs inside a host application
// whose allocator it may not call, or code that only receives raw device pointers from elsewhere.  For them the
// fill's scratch (pyramid nodes, the list of tiles without a valid pixel, their fill values, the coarse levels and
// the per-call counters) lives in one file-scope __device__ array of fixed size instead of a caller workspace.
// The array occupies kStaticScratchBytes on every GPU that loads this library, until the process exits.
#include "exw_internal.h"

namespace exw {

// Largest frame: at most kStaticMaxTiles fill tiles of 32 x 32 pixels (4096 x 4096, or 8192 x 2048, ...).
constexpr int kStaticMaxTiles = 16384;
constexpr size_t kStaticScratchBytes = 768u * 1024u;

static __device__ __align__(256) unsigned char g_fill_scratch[kStaticScratchBytes];

// The device address of the scratch array on the current device.  In host code g_fill_scratch is only a
// host-side stand-in for the symbol, so the address comes from cudaGetSymbolAddress.  It is looked up on every
// call (cheap once the module is loaded), so it stays right after cudaDeviceReset or in a new context, where the
// array may sit elsewhere.  The first call on a device loads the module: make it before any stream capture.
static cudaError_t static_scratch(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_fill_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace exw

using namespace exw;

extern "C" exw_status exw_fill_holes_static(void *color, exw_dtype cdt, const uint8_t *mask, int W, int H,
                                            exw_stream_t stream) {
    // the argument rules of exw_fill_holes (shared helpers), then the size limit of the built-in array
    if (!size_ok(W, H) || !dtype_ok(cdt) || !aligned(color, csize(cdt)) || !aligned(mask, 1))
        return EXW_ERR_INVALID_ARG;
    // Fill-only layout: status word, one frame header, then per-tile nodes, invalid-tile list, fill values and the
    // coarse pyramid levels (the motion-bounds tiles of the general workspace are not needed here).
    WsLayout l{};
    l.n5x = ceil_div(W, kFillTileSide);
    l.n5y = ceil_div(H, kFillTileSide);
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
    if (entry_check() != EXW_OK) return EXW_ERR_CUDA;
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
    return from_cuda(e);
}
