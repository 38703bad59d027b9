// exw_items.cuh -- the work items of the forward pass as device functions of a whole CTA (or warp): a bounds
// region, a tile plan, a fused tile (TMA windows or global memory), a fix-up slice.  The per-frame kernels launch
// them one item per CTA or in a persistent loop; the batched kernel takes them from a work queue.
#pragma once

#include "exw_tile.cuh"
#include "exw_tma.cuh"

namespace exw {

constexpr uint32_t kWaitLimit = 1u << 22;  // iterations of the bounded mbarrier wait (each >= 128 ns)

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
// Plan of one target tile (one warp): scans the 8 x 8 motion bounds that can reach the tile's region and
// records the landing rectangle of every fraction, whether all candidate sources share one motion, and the
// staging mode and window the fused kernel will use.
// ------------------------------------------------------------------------------------------------------------
template <typename CT, int WX, int WY>
__device__ inline void plan_tile(const TileParams &p, int tile) {  // called by one whole warp
    const int lane = threadIdx.x & 31;
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
    // One 8 x 8 bounds tile (bx, by): does it reach R, and with which landing rectangles and motion?  Returns its
    // splat descriptor (fm = 0 when it does not reach R).
    auto visit = [&](int bx, int by) -> SplatTile {
        SplatTile st{};
        const float4 b = __ldcg(p.tile_bounds + (size_t)by * p.nbx + bx);
        const float2 dr = __ldcg(p.tile_depth + (size_t)by * p.nbx + bx);  // issued with the bounds
        if (!(b.x <= b.y)) return st;
        uint32_t fm = 0u;
        bool small = true;
        const BoundsDec bd = bounds_dec(b, p.L);
#pragma unroll
        for (int kk = 0; kk < kMaxFrac; ++kk) {
            int ox0, ox1, oy0, oy1;
            bounds_offsets(bd, p.k0 + kk, ox0, ox1, oy0, oy1);
            const int lx0 = max(8 * bx, RX0 - ox1), lx1 = min(min(8 * bx + 7, p.W - 1), RX0 + kRegion - 1 - ox0);
            const int ly0 = max(8 * by, RY0 - oy1), ly1 = min(min(8 * by + 7, p.H - 1), RY0 + kRegion - 1 - oy0);
            const bool hit = kk < p.nfrac && lx0 <= lx1 && ly0 <= ly1;
            fm |= hit ? 1u << kk : 0u;
            r[kk][0] = hit ? min(r[kk][0], lx0) : r[kk][0];
            r[kk][1] = hit ? max(r[kk][1], lx1) : r[kk][1];
            r[kk][2] = hit ? min(r[kk][2], ly0) : r[kk][2];
            r[kk][3] = hit ? max(r[kk][3], ly1) : r[kk][3];
            small = small && ox0 >= -128 && ox0 <= 127 && oy0 >= -128 && oy0 <= 127;
            st.ox[kk] = (int8_t)max(-128, min(127, ox0));
            st.oy[kk] = (int8_t)max(-128, min(127, oy0));
        }
        if (fm) {
            const uint32_t bxb = __float_as_uint(b.x), byb = __float_as_uint(b.z);
            if (b.x != b.y || b.z != b.w) uni = false;
            else if (!has) { has = true; mx = bxb; my = byb; }
            else if (mx != bxb || my != byb) uni = false;
            st.bx = (uint16_t)bx;
            st.by = (uint16_t)by;
            st.fm = (uint8_t)fm;
            st.clean = b.x == b.y && b.z == b.w && dr.x > 0.0f && small ? 1 : 0;
        }
        return st;
    };
    // the candidates, compacted in visiting order into the plan's descriptors (none when there are too many)
    SplatTile *desc = p.pdesc != nullptr ? p.pdesc + (size_t)tile * kPlanDesc : nullptr;
    int ndesc = 0;
    // Two levels: the 32 x 32 regions within the frame-wide motion range whose bounds can reach R (one per lane),
    // then the 16 bounds tiles of each such region (two regions per pass, 16 lanes each).  A region's bounds
    // contain its tiles' bounds and the offsets are monotone in the motion, so no tile that reaches R is skipped.
    int bx0, bx1, by0, by1;
    if (frame_window(p, RX0, RY0, bx0, bx1, by0, by1)) {
        const int rx0 = bx0 >> 2, ry0 = by0 >> 2, nrr = (bx1 >> 2) - rx0 + 1;
        const int nreg = nrr * ((by1 >> 2) - ry0 + 1);
        for (int base = 0; base < nreg; base += 32) {
            const int idx = base + lane;
            int rxl = 0, ryl = 0;
            bool reach = false;
            if (idx < nreg) {
                ryl = ry0 + idx / nrr;
                rxl = rx0 + idx % nrr;
                const float4 rb = __ldcg(p.region_bounds + (size_t)ryl * p.n5x + rxl);
                if (rb.x <= rb.y) {
                    const BoundsDec rd = bounds_dec(rb, p.L);
                    for (int kk = 0; kk < p.nfrac && !reach; ++kk) {
                        int ox0, ox1, oy0, oy1;
                        bounds_offsets(rd, p.k0 + kk, ox0, ox1, oy0, oy1);
                        reach = 32 * rxl + 31 + ox1 >= RX0 && 32 * rxl + ox0 <= RX0 + kRegion - 1 &&
                                32 * ryl + 31 + oy1 >= RY0 && 32 * ryl + oy0 <= RY0 + kRegion - 1;
                    }
                }
            }
            unsigned m = __ballot_sync(0xFFFFFFFFu, reach);
            while (m) {
                const int l0 = __ffs(m) - 1;
                m &= m - 1u;
                int l1 = -1;
                if (m) {
                    l1 = __ffs(m) - 1;
                    m &= m - 1u;
                }
                const int src = lane < 16 ? l0 : l1;
                const int qx = __shfl_sync(0xFFFFFFFFu, rxl, src < 0 ? 0 : src);
                const int qy = __shfl_sync(0xFFFFFFFFu, ryl, src < 0 ? 0 : src);
                SplatTile st{};
                if (src >= 0) {
                    const int bx = 4 * qx + (lane & 3), by = 4 * qy + ((lane >> 2) & 3);
                    if (bx < p.nbx && by < p.nby) st = visit(bx, by);
                }
                const unsigned hm = __ballot_sync(0xFFFFFFFFu, st.fm != 0);
                const int slot = ndesc + __popc(hm & ((1u << lane) - 1u));
                if (desc != nullptr && st.fm != 0 && slot < kPlanDesc) desc[slot] = st;
                ndesc += __popc(hm);
            }
        }
    }
    __syncwarp();  // every lane's descriptors before lane 0 publishes the plan
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
    // Smooth uniform tile: every pixel of the source rectangle Nu (the union over fractions of R - o_k grown by one)
    // lies in the frame, can land, moves by (mx, my) (its 8 x 8 tile's bounds are exactly that motion), and the
    // depths of Nu lie within a factor 1 + 1/32 of their minimum.  Then every target of the tile has a winner,
    // no target is a crack (a nearer neighbour would differ by more than D/32) and every tap agrees: the
    // fractions are pure bilinear resamplings.  Exact: |Dt - Dp| <= Dmax - Dmin <= Dmin / 32 <= Dp / 32.
    bool smooth = false;
    if (uni && hasm && RX0 >= 0 && RY0 >= 0 && RX0 + kRegion <= p.W && RY0 + kRegion <= p.H) {
        Rect Nu{1 << 30, -(1 << 30), 1 << 30, -(1 << 30)};
        for (int kk = 0; kk < p.nfrac; ++kk) {
            const int ox = axis_off_of(mx, p.k0 + kk, p.L), oy = axis_off_of(my, p.k0 + kk, p.L);
            Nu.x0 = min(Nu.x0, RX0 - ox - 1);
            Nu.x1 = max(Nu.x1, RX0 + kRegion - ox);
            Nu.y0 = min(Nu.y0, RY0 - oy - 1);
            Nu.y1 = max(Nu.y1, RY0 + kRegion - oy);
        }
        if (Nu.x0 >= 0 && Nu.y0 >= 0 && Nu.x1 < p.W && Nu.y1 < p.H) {
            const int tx0 = Nu.x0 >> 3, ty0 = Nu.y0 >> 3, ntx = (Nu.x1 >> 3) - tx0 + 1;
            const int nt = ntx * ((Nu.y1 >> 3) - ty0 + 1);
            bool ok = true;
            float dmin = __int_as_float(0x7F800000), dmax = 0.0f;
            for (int idx = lane; idx < nt; idx += 32) {
                const size_t t = (size_t)(ty0 + idx / ntx) * p.nbx + (tx0 + idx % ntx);
                const float4 b = __ldcg(p.tile_bounds + t);
                const float2 d = __ldcg(p.tile_depth + t);
                ok = ok && __float_as_uint(b.x) == mx && __float_as_uint(b.y) == mx && __float_as_uint(b.z) == my &&
                     __float_as_uint(b.w) == my && d.x > 0.0f;
                dmin = fminf(dmin, d.x);
                dmax = fmaxf(dmax, d.y);
            }
            ok = __all_sync(0xFFFFFFFFu, ok) != 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                dmin = fminf(dmin, __shfl_xor_sync(0xFFFFFFFFu, dmin, o));
                dmax = fmaxf(dmax, __shfl_xor_sync(0xFFFFFFFFu, dmax, o));
            }
            smooth = ok && 32.0f * (dmax - dmin) <= dmin;
        }
    }
    if (lane != 0) return;
    TilePlan pl{};
    Rect U{1 << 30, -(1 << 30), 1 << 30, -(1 << 30)};
    bool all_fit = true;
#pragma unroll
    for (int kk = 0; kk < kMaxFrac; ++kk) {  // static indices: r and pl stay in registers
        const Rect R{r[kk][0], r[kk][1], r[kk][2], r[kk][3]};
        pl.rect[kk][0] = R.x0;
        pl.rect[kk][1] = R.x1;
        pl.rect[kk][2] = R.y0;
        pl.rect[kk][3] = R.y1;
        if (kk >= p.nfrac || R.empty()) continue;
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
    pl.ndesc = desc != nullptr && ndesc <= kPlanDesc ? ndesc : 0;
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
            pl.mode = smooth ? 5 : 0;
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

// Fix-up of the tiles without a valid pixel: the calling threads (tid of nt) take list entries first,
// first + stride, ...
template <typename CT>
__device__ __noinline__ void fixup_slice(const TileParams &p, uint32_t first, uint32_t stride, int tid, int nt) {
    const int n5 = p.n5x * p.n5y;
    const size_t plane = (size_t)p.W * p.H;
    for (int kk = 0; kk < p.nfrac; ++kk) {
        const uint32_t cnt = __ldcg(&p.fh->ninvalid[kk]);
        CT *oc = (CT *)p.out_color[kk];
        for (uint32_t e = first; e < cnt; e += stride) {
            const uint32_t tile = __ldcg(p.list + (size_t)kk * n5 + e);
            const float4 v = __ldcg(p.fillval + (size_t)kk * n5 + e);
            const int X0 = (int)(tile % (uint32_t)p.n5x) * kFillTile, Y0 = (int)(tile / (uint32_t)p.n5x) * kFillTile;
            const CT c0 = to_storage<CT>(v.x), c1 = to_storage<CT>(v.y), c2 = to_storage<CT>(v.z);
            for (int i = tid; i < kFillTile * kFillTile; i += nt) {
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

// Stage (a0) for one 32 x 32 source region (all threads of the CTA, any multiple of 128 threads up to 1024):
// per 8 x 8 tile the min/max of each motion component over pixels that can land, clamped to [-65536, 65536] (for
// k/4 fractions |d| >= 16384 beyond that: no landing in any frame) and -0 read as +0; frame-wide maxima in fh.
// Also per tile the depth range of its pixels in the frame, or (-1, -1) when one of them cannot land (the plan
// uses it to find smooth sources).  Warp w covers the rows w*rpw .. w*rpw + rpw - 1 of the region (rpw = 32 /
// warps), lane = column.  part: 8 float4 per warp of shared memory.
// The region's bounds go to region_bounds[ry * ceil(W / 32) + rx]; with frame_atomics the frame-wide maxima are
// raised here, else the caller raises them from the returned bounds (valid in warp 0).
// NW warps take part (4, 8 or 16), thread index tid in [0, 32 NW); bar() is a barrier over exactly them.
struct CtaBarrier {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
template <int NW, class Bar>
__device__ inline float4 bounds_region(const float *__restrict__ depth, const float *__restrict__ mv, int W, int H,
                                float4 *tile_bounds, float2 *tile_depth, float4 *region_bounds, FrameHeader *fh,
                                int rx, int ry, float4 *part, bool frame_atomics, int tid, Bar bar) {
    constexpr int nw = NW, rpw = 32 / NW;
    const int lane = tid & 31, w = tid >> 5;
    const int X0 = rx * 32, Y0 = ry * 32;
    const size_t plane = (size_t)W * H;
    float mnx = __int_as_float(0x7F800000), mxx = -mnx, mny = mnx, mxy = -mnx;
    const int x = X0 + lane;
    // the frame-wide maxima as they stand, read with the data (any earlier value is a valid lower bound: a stale one
    // only costs an atomic that does not raise anything)
    uint32_t seen = 0xFFFFFFFFu;
    if (frame_atomics && tid < 4) seen = reinterpret_cast<volatile uint32_t *>(fh->acc)[tid];
    float fx[rpw], fy[rpw];
    uint32_t db[rpw];
#pragma unroll
    for (int r = 0; r < rpw; ++r) {  // issue every load of the thread before using any
        db[r] = 0u;
        fx[r] = fy[r] = 0.0f;
        const int y = Y0 + w * rpw + r;
        if (r < rpw && x < W && y < H) {
            const size_t i = (size_t)y * W + x;
            db[r] = __float_as_uint(__ldg(depth + i));
            fx[r] = __ldg(mv + i);
            fy[r] = __ldg(mv + plane + i);
        }
    }
    float dmn = __int_as_float(0x7F800000), dmx = 0.0f, bad = 0.0f;
#pragma unroll
    for (int r = 0; r < rpw; ++r) {
        if (depth_ok(db[r]) && finite_bits(__float_as_uint(fx[r])) && finite_bits(__float_as_uint(fy[r]))) {
            const float cx = fminf(fmaxf(fx[r], -65536.0f), 65536.0f) + 0.0f;
            const float cy = fminf(fmaxf(fy[r], -65536.0f), 65536.0f) + 0.0f;
            mnx = fminf(mnx, cx);
            mxx = fmaxf(mxx, cx);
            mny = fminf(mny, cy);
            mxy = fmaxf(mxy, cy);
            dmn = fminf(dmn, __uint_as_float(db[r]));
            dmx = fmaxf(dmx, __uint_as_float(db[r]));
        } else if (r < rpw && x < W && Y0 + w * rpw + r < H) {
            bad = 1.0f;
        }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        mnx = fminf(mnx, __shfl_xor_sync(0xFFFFFFFFu, mnx, o));
        mxx = fmaxf(mxx, __shfl_xor_sync(0xFFFFFFFFu, mxx, o));
        mny = fminf(mny, __shfl_xor_sync(0xFFFFFFFFu, mny, o));
        mxy = fmaxf(mxy, __shfl_xor_sync(0xFFFFFFFFu, mxy, o));
        dmn = fminf(dmn, __shfl_xor_sync(0xFFFFFFFFu, dmn, o));
        dmx = fmaxf(dmx, __shfl_xor_sync(0xFFFFFFFFu, dmx, o));
        bad = fmaxf(bad, __shfl_xor_sync(0xFFFFFFFFu, bad, o));
    }
    if ((lane & 7) == 0) {
        part[w * 4 + (lane >> 3)] = make_float4(mnx, mxx, mny, mxy);
        part[4 * nw + w * 4 + (lane >> 3)] = make_float4(dmn, dmx, bad, 0.0f);
    }
    bar();
    if (tid < 32) {
        const int t = tid;
        float4 b = make_float4(__int_as_float(0x7F800000), __int_as_float(0xFF800000), __int_as_float(0x7F800000),
                               __int_as_float(0xFF800000));
        if (t < 16) {
            const int bxl = t & 3, byl = t >> 2, per = nw / 4;  // warps per 8-row band
            float4 dr = make_float4(__int_as_float(0x7F800000), 0.0f, 0.0f, 0.0f);
            for (int i = 0; i < per; ++i) {
                const float4 u = part[(byl * per + i) * 4 + bxl];
                b = make_float4(fminf(b.x, u.x), fmaxf(b.y, u.y), fminf(b.z, u.z), fmaxf(b.w, u.w));
                const float4 v = part[4 * nw + (byl * per + i) * 4 + bxl];
                dr = make_float4(fminf(dr.x, v.x), fmaxf(dr.y, v.y), fmaxf(dr.z, v.z), 0.0f);
            }
            const int gbx = X0 / 8 + bxl, gby = Y0 / 8 + byl;
            const int nbx = (W + 7) / 8, nby = (H + 7) / 8;
            if (gbx < nbx && gby < nby) {
                tile_bounds[(size_t)gby * nbx + gbx] = b;
                tile_depth[(size_t)gby * nbx + gbx] = dr.z != 0.0f ? make_float2(-1.0f, -1.0f) : make_float2(dr.x, dr.y);
            }
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            b.x = fminf(b.x, __shfl_xor_sync(0xFFFFFFFFu, b.x, o));
            b.y = fmaxf(b.y, __shfl_xor_sync(0xFFFFFFFFu, b.y, o));
            b.z = fminf(b.z, __shfl_xor_sync(0xFFFFFFFFu, b.z, o));
            b.w = fmaxf(b.w, __shfl_xor_sync(0xFFFFFFFFu, b.w, o));
        }
        if (t == 0) region_bounds[(size_t)ry * ((W + 31) / 32) + rx] = b;
        if (frame_atomics && t < 4 && b.x <= b.y) {
            // Frame-wide maxima: an atomic only when this region's value exceeds what was there when the region began
            const float v = t == 0 ? -b.x : t == 1 ? b.y : t == 2 ? -b.z : b.w;
            const uint32_t code = float_order(v);
            if (code > seen) atomicMax(&fh->acc[t], code);
        }
        return b;
    }
    return make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace exw
