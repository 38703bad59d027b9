// exw_fwd.cu -- the staged kernels (exw_warp's gather, exw_fill_holes' fill) and the coarse fix-up; the fused
// forward pass is the persistent engine (exw_engine.cu).
#include "exw_items.cuh"

namespace exw {

// Plans: one warp per target tile (the first stream of an engine launch is planned ahead of the launch).
template <typename CT, int WX, int WY>
__global__ void __launch_bounds__(kThreads) plan_kernel(TileParams p) {
    grid_dependency_wait();  // the bounds kernel before
    grid_dependents_launch();
    const int tile = blockIdx.x * kWarps + (threadIdx.x >> 5);
    if (tile < p.n5x * p.n5y) plan_tile<CT, WX, WY>(p, tile);
}

// ------------------------------------------------------------------------------------------------------------
// Staged stage (b): keys from global memory (exw_splat_motion), one fraction, no fill.
// ------------------------------------------------------------------------------------------------------------
template <typename CT>
__global__ void __launch_bounds__(kThreads) warp_tiles_kernel(TileParams p) {
    __shared__ __align__(16) TileSmem s;
    const int tid = threadIdx.x;
    const int X0 = blockIdx.x * kFillTile, Y0 = blockIdx.y * kFillTile;
    const uint32_t npix = (uint32_t)p.W * (uint32_t)p.H;
    for (int i = tid; i < kRegionN; i += kThreads) {
        const int ry = i / kRegion, rx = i - ry * kRegion;
        const int gx = X0 - 1 + rx, gy = Y0 - 1 + ry;
        uint64_t kv = kKeyEmpty;
        if (gx >= 0 && gx < p.W && gy >= 0 && gy < p.H) {
            const uint64_t g = __ldg((const unsigned long long *)p.keys + (size_t)gy * p.W + gx);
            const uint32_t idx = (uint32_t)g;
            if (g != kKeyEmpty && idx < npix) {  // a malformed key reads as empty instead of faulting
                const uint32_t py = idx / (uint32_t)p.W, px = idx - py * (uint32_t)p.W;
                kv = pack_key_local(key_dbits(g), (int)px, (int)py);
            }
        }
        s.key[0][i] = kv;
    }
    __syncthreads();
    const GlobalAcc<CT> a{(const CT *)p.color, p.depth, p.mv, p.W, (size_t)p.W * p.H};
    finish_fraction<CT, false>(s, a, key_source(s, 0), p, 0, X0, Y0, 0);
}

// ------------------------------------------------------------------------------------------------------------
// Staged stage (c): pull-push of an existing colour + mask, in place.
// ------------------------------------------------------------------------------------------------------------
template <typename CT>
__global__ void __launch_bounds__(kThreads) fill_tiles_kernel(TileParams p) {
    __shared__ __align__(16) TilePyr pyr;
    __shared__ int last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int X0 = blockIdx.x * kFillTile, Y0 = blockIdx.y * kFillTile;
    const size_t plane = (size_t)p.W * p.H;
    const int gx = X0 + lane;
    const CT *oc = (const CT *)p.out_color[0];
    float4 c[2];
    uint8_t m[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int gy = Y0 + 2 * wid + j;
        const bool in = gx < p.W && gy < p.H;
        c[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        m[j] = 1;
        if (in) {
            const size_t q = (size_t)gy * p.W + gx;
            m[j] = __ldg(p.mask_in + q);
            c[j] = make_float4(load_c<CT>(oc + q), load_c<CT>(oc + plane + q), load_c<CT>(oc + 2 * plane + q),
                               m[j] == 0 ? 1.0f : 0.0f);
        }
    }
    fill_store<CT>(p, pyr, c, m, 0, X0, Y0, blockIdx.y * p.n5x + blockIdx.x, false, false);
    tile_done(p, &last);
}

// Fix-up: every tile without a valid pixel takes the coarse value chosen for it.
template <typename CT>
__global__ void __launch_bounds__(kThreads) fixup_kernel(TileParams p) {
    fixup_slice<CT>(p, blockIdx.x, gridDim.x, (int)threadIdx.x, (int)blockDim.x);
}

// ------------------------------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------------------------------
static dim3 tile_grid(const TileParams &p) { return dim3((unsigned)p.n5x, (unsigned)p.n5y, 1); }

cudaError_t launch_plan(const TileParams &p, exw_dtype cdt, int shape, cudaStream_t s) {
    const int ntiles = p.n5x * p.n5y;
    const unsigned g = (unsigned)((ntiles + kWarps - 1) / kWarps);
    timing_begin("exw_plan", s);
    using S0 = WinShape<0>;
    using S1 = WinShape<1>;
    void (*k)(TileParams) = shape == 0 ? (cdt == EXW_F32 ? plan_kernel<float, S0::xf32, S0::yf32>
                                                          : plan_kernel<__half, S0::xf16, S0::yf16>)
                                       : (cdt == EXW_F32 ? plan_kernel<float, S1::xf32, S1::yf32>
                                                          : plan_kernel<__half, S1::xf16, S1::yf16>);
    const cudaError_t e = launch_dependent(k, dim3(g), dim3(kThreads), 0, s, p);
    count_launch();
    timing_end("exw_plan", s);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_warp_tiles(const TileParams &p, exw_dtype cdt, cudaStream_t s) {
    const dim3 g = tile_grid(p);
    timing_begin("exw_warp_tiles", s);
    if (cdt == EXW_F32) warp_tiles_kernel<float><<<g, kThreads, 0, s>>>(p);
    else warp_tiles_kernel<__half><<<g, kThreads, 0, s>>>(p);
    count_launch();
    timing_end("exw_warp_tiles", s);
    return cudaGetLastError();
}

cudaError_t launch_fill_tiles(const TileParams &p, exw_dtype cdt, cudaStream_t s) {
    const dim3 g = tile_grid(p);
    timing_begin("exw_fill_tiles", s);
    if (cdt == EXW_F32) fill_tiles_kernel<float><<<g, kThreads, 0, s>>>(p);
    else fill_tiles_kernel<__half><<<g, kThreads, 0, s>>>(p);
    count_launch();
    timing_end("exw_fill_tiles", s);
    return cudaGetLastError();
}

cudaError_t launch_fixup(const TileParams &p, exw_dtype cdt, cudaStream_t s) {
    const int n5 = p.n5x * p.n5y;
    const unsigned g = (unsigned)(n5 < 304 ? n5 : 304);
    timing_begin("exw_fixup", s);
    if (cdt == EXW_F32) fixup_kernel<float><<<g, kThreads, 0, s>>>(p);
    else fixup_kernel<__half><<<g, kThreads, 0, s>>>(p);
    count_launch();
    timing_end("exw_fixup", s);
    return cudaGetLastError();
}

}  // namespace exw
