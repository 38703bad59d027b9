// exw_fwd.cu -- forward tile kernels: fused splat+gather+fill (persistent TMA and plain), staged gather, staged
// fill, coarse fix-up.
//
// The persistent TMA kernel runs 2 CTAs of 512 threads per SM (about 100 KB of shared memory each).  Each CTA takes 32 x 32 target
// tiles from a queue.  Per tile it scans the 8 x 8 motion bounds for the source rectangles that can land in the
// tile (plus its one-pixel ring), then stages the source depth, motion and colour of that rectangle grown by one
// pixel (the bilinear taps) into shared memory with three TMA loads (cp.async.bulk.tensor, mbarrier completion):
//   uniform: every candidate source tile carries one and the same motion, so each fraction is a pure translation
//            and the winners are read off the window directly -- no splat, no atomics;
//   mode A:  one window covers the rectangles of all fractions -> one load, splat all fractions, gather each;
//   mode B:  per fraction, a window for that fraction's rectangle;
//   mode C:  a rectangle too large for a window -> the tile is processed from global memory.
// While one CTA of an SM waits for its TMA load, the other computes.  Tiles without a valid pixel after the fill
// are finished from the coarse pyramid levels, which the CTA finishing the frame's last tile builds (a done
// counter in the workspace; no grid-wide barrier and no spin on other CTAs).
#include "exw_tile.cuh"
#include "exw_tma.cuh"

namespace exw {

// ------------------------------------------------------------------------------------------------------------
// Plain fused kernel: one tile per CTA, source read from global memory (any frame width).
// ------------------------------------------------------------------------------------------------------------
template <typename CT, bool FILL>
__global__ void __launch_bounds__(kThreads) fused_kernel(TileParams p) {
    __shared__ __align__(16) TileSmem s;
    const int tile = blockIdx.y * p.n5x + blockIdx.x;
    const int X0 = blockIdx.x * kFillTile, Y0 = blockIdx.y * kFillTile;
    init_keys(s, p.nfrac);
    __syncthreads();
    splat_global(s, p, X0 - 1, Y0 - 1);
    __syncthreads();
    const GlobalAcc<CT> a{(const CT *)p.color, p.depth, p.mv, p.W, (size_t)p.W * p.H};
    for (int kk = 0; kk < p.nfrac; ++kk) finish_fraction<CT, FILL>(s, a, key_source(s, kk), p, kk, X0, Y0, tile);
    if (FILL) tile_done(p, &s.last);
}

// ------------------------------------------------------------------------------------------------------------
// Persistent fused kernel with TMA-staged source windows.
// ------------------------------------------------------------------------------------------------------------
constexpr uint32_t kWaitLimit = 1u << 22;  // iterations of the bounded mbarrier wait (each >= 128 ns)

template <typename CT, int WX, int WY>
struct TmaSmem {
    Window<CT, WX, WY> win;  // first: 128-byte aligned TMA destinations
    TileSmem t;
};

template <typename CT, int WX, int WY>
__device__ __forceinline__ Rect window_rect(Rect U) {  // window origin/extent for rectangle U grown by 1
    constexpr int kAlign = sizeof(CT) == 2 ? 8 : 4;  // x * element size must be a multiple of 16 bytes
    Rect w;
    w.x0 = (U.x0 - 1) & ~(kAlign - 1);
    w.y0 = U.y0 - 1;
    w.x1 = w.x0 + WX - 1;
    w.y1 = w.y0 + WY - 1;
    return w;
}

template <typename CT, int WX, int WY>
__device__ __forceinline__ bool window_fits(Rect U) {
    const Rect w = window_rect<CT, WX, WY>(U);
    return U.x1 + 1 <= w.x1 && U.y1 + 1 <= w.y1;
}

// ------------------------------------------------------------------------------------------------------------
// Plan kernel: one warp per target tile scans the 8 x 8 motion bounds that can reach the tile's region and
// records the landing rectangle of every fraction, whether all candidate sources share one motion, and the
// staging mode and window the fused kernel will use.
// ------------------------------------------------------------------------------------------------------------
template <typename CT, int WX, int WY>
__global__ void __launch_bounds__(kThreads) plan_kernel(TileParams p) {
    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (tile >= p.n5x * p.n5y) return;
    const int X0 = (tile % p.n5x) * kFillTile, Y0 = (tile / p.n5x) * kFillTile;
    const int RX0 = X0 - 1, RY0 = Y0 - 1;
    int r[kMaxFrac][4];
#pragma unroll
    for (int kk = 0; kk < kMaxFrac; ++kk) {
        r[kk][0] = r[kk][2] = 1 << 30;
        r[kk][1] = r[kk][3] = -(1 << 30);
    }
    bool uni = true, has = false;
    uint32_t mx = 0u, my = 0u;
    int bx0, bx1, by0, by1;
    if (frame_window(p, RX0, RY0, bx0, bx1, by0, by1)) {
        const int nbxr = bx1 - bx0 + 1;
        const int total = nbxr * (by1 - by0 + 1);
        for (int idx = lane; idx < total; idx += 32) {
            const int by = by0 + idx / nbxr, bx = bx0 + idx % nbxr;
            const float4 b = __ldcg(p.tile_bounds + (size_t)by * p.nbx + bx);
            if (!(b.x <= b.y)) continue;
            bool cand = false;
#pragma unroll
            for (int kk = 0; kk < kMaxFrac; ++kk) {
                if (kk >= p.nfrac) break;
                int ox0, ox1, oy0, oy1;
                tile_offsets(b, p.k0 + kk, p.L, ox0, ox1, oy0, oy1);
                const int lx0 = max(8 * bx, RX0 - ox1), lx1 = min(min(8 * bx + 7, p.W - 1), RX0 + kRegion - 1 - ox0);
                const int ly0 = max(8 * by, RY0 - oy1), ly1 = min(min(8 * by + 7, p.H - 1), RY0 + kRegion - 1 - oy0);
                if (lx0 > lx1 || ly0 > ly1) continue;
                cand = true;
                r[kk][0] = min(r[kk][0], lx0);
                r[kk][1] = max(r[kk][1], lx1);
                r[kk][2] = min(r[kk][2], ly0);
                r[kk][3] = max(r[kk][3], ly1);
            }
            if (cand) {
                const uint32_t bxb = __float_as_uint(b.x), byb = __float_as_uint(b.z);
                if (b.x != b.y || b.z != b.w) uni = false;
                else if (!has) { has = true; mx = bxb; my = byb; }
                else if (mx != bxb || my != byb) uni = false;
            }
        }
    }
#pragma unroll
    for (int kk = 0; kk < kMaxFrac; ++kk) {
        r[kk][0] = __reduce_min_sync(0xFFFFFFFFu, r[kk][0]);
        r[kk][1] = __reduce_max_sync(0xFFFFFFFFu, r[kk][1]);
        r[kk][2] = __reduce_min_sync(0xFFFFFFFFu, r[kk][2]);
        r[kk][3] = __reduce_max_sync(0xFFFFFFFFu, r[kk][3]);
    }
    const unsigned hasm = __ballot_sync(0xFFFFFFFFu, has);
    uni = __all_sync(0xFFFFFFFFu, uni) != 0;
    if (hasm) {
        const int src = __ffs(hasm) - 1;
        const uint32_t m0 = __shfl_sync(0xFFFFFFFFu, mx, src), m1 = __shfl_sync(0xFFFFFFFFu, my, src);
        uni = uni && __all_sync(0xFFFFFFFFu, !has || (mx == m0 && my == m1)) != 0;
        mx = m0;
        my = m1;
    }
    if (lane != 0) return;
    TilePlan pl{};
    Rect U{1 << 30, -(1 << 30), 1 << 30, -(1 << 30)};
    bool all_fit = true;
    for (int kk = 0; kk < p.nfrac; ++kk) {
        const Rect R{r[kk][0], r[kk][1], r[kk][2], r[kk][3]};
        pl.rect[kk][0] = R.x0;
        pl.rect[kk][1] = R.x1;
        pl.rect[kk][2] = R.y0;
        pl.rect[kk][3] = R.y1;
        if (R.empty()) continue;
        U.x0 = min(U.x0, R.x0);
        U.x1 = max(U.x1, R.x1);
        U.y0 = min(U.y0, R.y0);
        U.y1 = max(U.y1, R.y1);
        all_fit = all_fit && window_fits<CT, WX, WY>(R);
    }
    constexpr int kAlign = sizeof(CT) == 2 ? 8 : 4;
    pl.mode = -1;
    pl.umx = mx;
    pl.umy = my;
    if (U.empty()) {
        pl.mode = 4;
    } else if (uni && hasm) {
        // uniform: fraction kk's sources are R - o_kk; stage their union grown by one pixel (the taps)
        Rect N{1 << 30, -(1 << 30), 1 << 30, -(1 << 30)};
        for (int kk = 0; kk < p.nfrac; ++kk) {
            const int ox = axis_off_of(mx, p.k0 + kk, p.L), oy = axis_off_of(my, p.k0 + kk, p.L);
            N.x0 = min(N.x0, RX0 - ox - 1);
            N.x1 = max(N.x1, RX0 + kRegion - ox);
            N.y0 = min(N.y0, RY0 - oy - 1);
            N.y1 = max(N.y1, RY0 + kRegion - oy);
        }
        N.x0 = max(N.x0, 0);
        N.y0 = max(N.y0, 0);
        N.x1 = min(N.x1, p.W - 1);
        N.y1 = min(N.y1, p.H - 1);
        if (!N.empty() && N.x1 < (N.x0 & ~(kAlign - 1)) + WX && N.y1 < N.y0 + WY) {
            pl.mode = 0;
            pl.wx0 = N.x0 & ~(kAlign - 1);
            pl.wy0 = N.y0;
        }
    }
    if (pl.mode < 0) {
        if (window_fits<CT, WX, WY>(U)) {
            const Rect w = window_rect<CT, WX, WY>(U);
            pl.mode = 1;
            pl.wx0 = w.x0;
            pl.wy0 = w.y0;
        } else {
            pl.mode = all_fit ? 2 : 3;
        }
    }
    p.plans[tile] = pl;
}

__device__ __forceinline__ Rect union_rect(const TilePlan &pl, int nfrac) {
    Rect U{1 << 30, -(1 << 30), 1 << 30, -(1 << 30)};
    for (int kk = 0; kk < nfrac; ++kk) {
        const Rect R{__ldcg(&pl.rect[kk][0]), __ldcg(&pl.rect[kk][1]), __ldcg(&pl.rect[kk][2]),
                     __ldcg(&pl.rect[kk][3])};
        if (R.empty()) continue;
        U.x0 = min(U.x0, R.x0);
        U.x1 = max(U.x1, R.x1);
        U.y0 = min(U.y0, R.y0);
        U.y1 = max(U.y1, R.y1);
    }
    return U;
}

// Stage the window at (x0, y0) and wait for it.  Returns false (with the status word set) if the bounded wait ran
// out; every thread returns the same value.  The leading barrier makes every thread finish with the previous
// contents of the window before the copy overwrites them.
template <typename CT, int WX, int WY>
__device__ bool load_window(TmaSmem<CT, WX, WY> &s, const TileParams &p, const CUtensorMap *tcol,
                            const CUtensorMap *tdep, const CUtensorMap *tmv, int x0, int y0, uint32_t &phase) {
    constexpr uint32_t kBytes = WX * WY * (4 + 8 + 3 * (uint32_t)sizeof(CT));
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&s.t.mbar, kBytes);
        tma_load_2d(s.win.depth, tdep, x0, y0, &s.t.mbar);
        tma_load_3d(&s.win.mv[0][0], tmv, x0, y0, 0, &s.t.mbar);
        tma_load_3d(&s.win.col[0][0], tcol, x0, y0, 0, &s.t.mbar);
    }
    const bool ok = mbar_wait_bounded(&s.t.mbar, phase, kWaitLimit);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicExch(p.status, (uint32_t)EXW_ERR_TIMEOUT);
        mbar_wait_bounded(&s.t.mbar, phase ^ 1u, kWaitLimit);  // let the copy in flight land before leaving
        return false;
    }
    return true;
}

template <typename CT, int WX, int WY, bool FILL>
__global__ void __launch_bounds__(kThreads, 2)
    fused_tma_kernel(TileParams p, const __grid_constant__ CUtensorMap tcol, const __grid_constant__ CUtensorMap tdep,
                     const __grid_constant__ CUtensorMap tmv) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TmaSmem<CT, WX, WY> &s = *reinterpret_cast<TmaSmem<CT, WX, WY> *>(smem_raw);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&s.t.mbar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    const int ntiles = p.n5x * p.n5y;
    const GlobalAcc<CT> ga{(const CT *)p.color, p.depth, p.mv, p.W, (size_t)p.W * p.H};
    for (;;) {
        if (tid == 0) s.t.tile = (int)atomicAdd(&p.fh->queue, 1u);
        __syncthreads();
        const int tile = s.t.tile;
        if (tile >= ntiles) break;
        const int X0 = (tile % p.n5x) * kFillTile, Y0 = (tile / p.n5x) * kFillTile;
        const int RX0 = X0 - 1, RY0 = Y0 - 1;
        const TilePlan &pl = p.plans[tile];
        const int mode = __ldcg(&pl.mode);
        if (tid == 0) atomicAdd(&p.fh->nmode[mode < 4 ? mode : 1], 1u);
        if (mode == 0) {
            const int x0 = __ldcg(&pl.wx0), y0 = __ldcg(&pl.wy0);
            const uint32_t umx = __ldcg(&pl.umx), umy = __ldcg(&pl.umy);
            if (!load_window(s, p, &tcol, &tdep, &tmv, x0, y0, phase)) return;
            const WinAcc<CT, WX, WY> wa{&s.win, x0, y0};
            uint32_t *dw = reinterpret_cast<uint32_t *>(&s.t.key[0][0]);
            for (int kk = 0; kk < p.nfrac; ++kk)
                uniform_words(dw + kk * kRegionN, p, wa, axis_off_of(umx, p.k0 + kk, p.L),
                              axis_off_of(umy, p.k0 + kk, p.L), __uint_as_float(umx), __uint_as_float(umy), RX0, RY0);
            __syncthreads();
            for (int kk = 0; kk < p.nfrac; ++kk)
                finish_fraction<CT, FILL>(s.t, wa,
                                          UniformSource{dw + kk * kRegionN, __uint_as_float(umx),
                                                        __uint_as_float(umy), axis_off_of(umx, p.k0 + kk, p.L),
                                                        axis_off_of(umy, p.k0 + kk, p.L)},
                                          p, kk, X0, Y0, tile);
        } else if (mode == 1) {
            const int x0 = __ldcg(&pl.wx0), y0 = __ldcg(&pl.wy0);
            const Rect U = union_rect(pl, p.nfrac);
            init_keys(s.t, p.nfrac);
            if (!load_window(s, p, &tcol, &tdep, &tmv, x0, y0, phase)) return;
            const WinAcc<CT, WX, WY> wa{&s.win, x0, y0};
            splat_window(s.t, p, wa, U, (1u << p.nfrac) - 1u, RX0, RY0);
            __syncthreads();
            for (int kk = 0; kk < p.nfrac; ++kk)
                finish_fraction<CT, FILL>(s.t, wa, key_source(s.t, kk), p, kk, X0, Y0, tile);
        } else if (mode == 2) {
            init_keys(s.t, p.nfrac);
            for (int kk = 0; kk < p.nfrac; ++kk) {
                const Rect R{__ldcg(&pl.rect[kk][0]), __ldcg(&pl.rect[kk][1]), __ldcg(&pl.rect[kk][2]),
                             __ldcg(&pl.rect[kk][3])};
                if (R.empty()) {
                    __syncthreads();
                    finish_fraction<CT, FILL>(s.t, ga, key_source(s.t, kk), p, kk, X0, Y0, tile);
                    continue;
                }
                const Rect w = window_rect<CT, WX, WY>(R);
                if (!load_window(s, p, &tcol, &tdep, &tmv, w.x0, w.y0, phase)) return;
                const WinAcc<CT, WX, WY> wa{&s.win, w.x0, w.y0};
                splat_window(s.t, p, wa, R, 1u << kk, RX0, RY0);
                __syncthreads();
                finish_fraction<CT, FILL>(s.t, wa, key_source(s.t, kk), p, kk, X0, Y0, tile);
            }
        } else {  // 3: too wide for a window; 4: nothing lands (every key stays empty)
            init_keys(s.t, p.nfrac);
            __syncthreads();
            if (mode == 3) {
                splat_global(s.t, p, RX0, RY0);
                __syncthreads();
            }
            for (int kk = 0; kk < p.nfrac; ++kk)
                finish_fraction<CT, FILL>(s.t, ga, key_source(s.t, kk), p, kk, X0, Y0, tile);
        }
        if (FILL) tile_done(p, &s.t.last);
    }
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

// ------------------------------------------------------------------------------------------------------------
// Fix-up: every tile without a valid pixel takes the coarse value chosen for it.
// ------------------------------------------------------------------------------------------------------------
template <typename CT>
__global__ void __launch_bounds__(kThreads) fixup_kernel(TileParams p) {
    const int n5 = p.n5x * p.n5y;
    const size_t plane = (size_t)p.W * p.H;
    for (int kk = 0; kk < p.nfrac; ++kk) {
        const uint32_t cnt = p.fh->ninvalid[kk];
        CT *oc = (CT *)p.out_color[kk];
        for (uint32_t e = blockIdx.x; e < cnt; e += gridDim.x) {
            const uint32_t tile = p.list[(size_t)kk * n5 + e];
            const float4 v = p.fillval[(size_t)kk * n5 + e];
            const int X0 = (int)(tile % (uint32_t)p.n5x) * kFillTile, Y0 = (int)(tile / (uint32_t)p.n5x) * kFillTile;
            const CT c0 = to_storage<CT>(v.x), c1 = to_storage<CT>(v.y), c2 = to_storage<CT>(v.z);
            for (int i = threadIdx.x; i < kFillTile * kFillTile; i += kThreads) {
                const int gx = X0 + (i & 31), gy = Y0 + (i >> 5);
                if (gx >= p.W || gy >= p.H) continue;
                const size_t q = (size_t)gy * p.W + gx;
                oc[q] = c0;
                oc[plane + q] = c1;
                oc[2 * plane + q] = c2;
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------------------------------
static dim3 tile_grid(const TileParams &p) { return dim3((unsigned)p.n5x, (unsigned)p.n5y, 1); }

cudaError_t launch_fused(const TileParams &p, exw_dtype cdt, bool fill, cudaStream_t s) {
    const dim3 g = tile_grid(p);
    timing_begin("exw_fused", s);
    if (cdt == EXW_F32) {
        if (fill) fused_kernel<float, true><<<g, kThreads, 0, s>>>(p);
        else fused_kernel<float, false><<<g, kThreads, 0, s>>>(p);
    } else {
        if (fill) fused_kernel<__half, true><<<g, kThreads, 0, s>>>(p);
        else fused_kernel<__half, false><<<g, kThreads, 0, s>>>(p);
    }
    count_launch();
    timing_end("exw_fused", s);
    return cudaGetLastError();
}

template <typename CT, int WX, int WY, bool FILL>
static cudaError_t launch_tma_t(const TileParams &p, const TmaMaps &m, int grid, cudaStream_t s) {
    constexpr size_t kSmem = sizeof(TmaSmem<CT, WX, WY>);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(fused_tma_kernel<CT, WX, WY, FILL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    fused_tma_kernel<CT, WX, WY, FILL><<<grid, kThreads, kSmem, s>>>(p, m.col, m.depth, m.mv);
    return cudaGetLastError();
}

cudaError_t launch_fused_tma(const TileParams &p, const TmaMaps &m, exw_dtype cdt, bool fill, int grid,
                             cudaStream_t s) {
    timing_begin("exw_fused_tma", s);
    cudaError_t e;
    if (cdt == EXW_F32)
        e = fill ? launch_tma_t<float, kWinXF32, kWinYF32, true>(p, m, grid, s)
                 : launch_tma_t<float, kWinXF32, kWinYF32, false>(p, m, grid, s);
    else
        e = fill ? launch_tma_t<__half, kWinXF16, kWinYF16, true>(p, m, grid, s)
                 : launch_tma_t<__half, kWinXF16, kWinYF16, false>(p, m, grid, s);
    count_launch();
    timing_end("exw_fused_tma", s);
    return e;
}

cudaError_t launch_plan(const TileParams &p, exw_dtype cdt, cudaStream_t s) {
    const int ntiles = p.n5x * p.n5y;
    const unsigned g = (unsigned)((ntiles + kThreads / 32 - 1) / (kThreads / 32));
    timing_begin("exw_plan", s);
    if (cdt == EXW_F32) plan_kernel<float, kWinXF32, kWinYF32><<<g, kThreads, 0, s>>>(p);
    else plan_kernel<__half, kWinXF16, kWinYF16><<<g, kThreads, 0, s>>>(p);
    count_launch();
    timing_end("exw_plan", s);
    return cudaGetLastError();
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
