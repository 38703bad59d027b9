// exw_tile.cuh -- per-tile passes shared by the forward kernels (one 32 x 32 target tile Q per CTA iteration).
//
// A tile's keys cover Q plus a one-pixel ring R (the crack rule reads 4-neighbours).  The splat takes every
// source pixel that can land in R -- found from the 8 x 8 motion bounds -- either from a TMA-staged shared-memory
// window or from global memory; the gather reads through the matching accessor.  Per fraction the tile is then
// gathered, hole-marked, filled from pyramid levels 1..5 and stored with lane = x (one 128-byte row per warp
// access).
#pragma once

#include "exw_device.cuh"
#include "exw_internal.h"

namespace exw {

constexpr int kThreads = 256;

struct TileSmem {
    uint64_t key[kMaxFrac][kRegionN];
    FillSmem fill;
    uint32_t cand[kThreads];
    int urect[kMaxFrac][4];  // landing rectangle per fraction: x0, x1, y0, y1 (source pixels)
    uint32_t ncand;
    int tile, last, flag;
    uint64_t mbar;
};

struct Rect {
    int x0, x1, y0, y1;
    __device__ __forceinline__ bool empty() const { return x1 < x0 || y1 < y0; }
};

__device__ __forceinline__ void init_keys(TileSmem &s, int nfrac) {
    for (int i = threadIdx.x; i < nfrac * kRegionN; i += blockDim.x) (&s.key[0][0])[i] = kKeyEmpty;
}

// The block range that can reach region R (RX0, RY0 .. +33) under the frame-wide motion bounds, for fractions
// k0 .. k0+nfrac-1.  Returns false when nothing can land anywhere.
__device__ __forceinline__ bool frame_window(const TileParams &p, int RX0, int RY0, int &bx0, int &bx1, int &by0,
                                             int &by1) {
    const uint32_t a0 = __ldcg(&p.fh->acc[0]), a1 = __ldcg(&p.fh->acc[1]);
    const uint32_t a2 = __ldcg(&p.fh->acc[2]), a3 = __ldcg(&p.fh->acc[3]);
    if (a1 == 0u) return false;
    const AxisDec fx0 = axis_dec(__float_as_uint(-float_unorder(a0)), p.L);
    const AxisDec fx1 = axis_dec(__float_as_uint(float_unorder(a1)), p.L);
    const AxisDec fy0 = axis_dec(__float_as_uint(-float_unorder(a2)), p.L);
    const AxisDec fy1 = axis_dec(__float_as_uint(float_unorder(a3)), p.L);
    int xlo = 1 << 30, xhi = -(1 << 30), ylo = 1 << 30, yhi = -(1 << 30);
    for (int kk = 0; kk < p.nfrac; ++kk) {
        const int k = p.k0 + kk;
        int ox0, ox1, oy0, oy1;
        axis_off(fx0, k, ox0);
        axis_off(fx1, k, ox1);
        axis_off(fy0, k, oy0);
        axis_off(fy1, k, oy1);
        xlo = min(xlo, RX0 - ox1);
        xhi = max(xhi, RX0 + kRegion - 1 - ox0);
        ylo = min(ylo, RY0 - oy1);
        yhi = max(yhi, RY0 + kRegion - 1 - oy0);
    }
    bx0 = max(0, xlo >> 3);
    bx1 = min(p.nbx - 1, xhi >> 3);
    by0 = max(0, ylo >> 3);
    by1 = min(p.nby - 1, yhi >> 3);
    return bx0 <= bx1 && by0 <= by1;
}

// Offsets of one bounds tile for fraction k: [ox0, ox1] x [oy0, oy1].
__device__ __forceinline__ void tile_offsets(const float4 &b, int k, int L, int &ox0, int &ox1, int &oy0, int &oy1) {
    ox0 = axis_off_of(__float_as_uint(b.x), k, L);
    ox1 = axis_off_of(__float_as_uint(b.y), k, L);
    oy0 = axis_off_of(__float_as_uint(b.z), k, L);
    oy1 = axis_off_of(__float_as_uint(b.w), k, L);
}

// Landing rectangles: per fraction, the bounding box of the source pixels whose tile's motion bounds allow them
// to land in R.  Every pixel that does land lies inside (the winners' taps lie inside it grown by one pixel).
__device__ void scan_landing(TileSmem &s, const TileParams &p, int RX0, int RY0) {
    const int tid = threadIdx.x;
    if (tid < kMaxFrac * 4) (&s.urect[0][0])[tid] = (tid & 1) ? -(1 << 30) : (1 << 30);
    __syncthreads();
    int bx0, bx1, by0, by1;
    if (!frame_window(p, RX0, RY0, bx0, bx1, by0, by1)) return;
    const int nbxr = bx1 - bx0 + 1;
    const int total = nbxr * (by1 - by0 + 1);
    for (int idx = tid; idx < total; idx += kThreads) {
        const int by = by0 + idx / nbxr, bx = bx0 + idx % nbxr;
        const float4 b = __ldcg(p.tile_bounds + (size_t)by * p.nbx + bx);
        if (!(b.x <= b.y)) continue;
        for (int kk = 0; kk < p.nfrac; ++kk) {
            int ox0, ox1, oy0, oy1;
            tile_offsets(b, p.k0 + kk, p.L, ox0, ox1, oy0, oy1);
            const int lx0 = max(8 * bx, RX0 - ox1), lx1 = min(min(8 * bx + 7, p.W - 1), RX0 + kRegion - 1 - ox0);
            const int ly0 = max(8 * by, RY0 - oy1), ly1 = min(min(8 * by + 7, p.H - 1), RY0 + kRegion - 1 - oy0);
            if (lx0 > lx1 || ly0 > ly1) continue;
            atomicMin(&s.urect[kk][0], lx0);
            atomicMax(&s.urect[kk][1], lx1);
            atomicMin(&s.urect[kk][2], ly0);
            atomicMax(&s.urect[kk][3], ly1);
        }
    }
}

// Splat one source pixel (x, y) for the fractions in fm into the region keys.
__device__ __forceinline__ void splat_pixel(TileSmem &s, const TileParams &p, int x, int y, uint32_t db, uint32_t ux,
                                            uint32_t uy, uint32_t fm, int RX0, int RY0) {
    if (!depth_ok(db) || !finite_bits(ux) || !finite_bits(uy)) return;
    const AxisDec dx = axis_dec(ux, p.L), dy = axis_dec(uy, p.L);
    const uint64_t key = pack_key_local(db, x, y);
    for (int kk = 0; kk < p.nfrac; ++kk) {
        if (!(fm & (1u << kk))) continue;
        const int k = p.k0 + kk;
        int ox, oy;
        if (!axis_off(dx, k, ox) || !axis_off(dy, k, oy)) continue;
        const int gx = x + ox, gy = y + oy;
        if ((unsigned)gx >= (unsigned)p.W || (unsigned)gy >= (unsigned)p.H) continue;
        const int rx = gx - RX0, ry = gy - RY0;
        if ((unsigned)rx < (unsigned)kRegion && (unsigned)ry < (unsigned)kRegion)
            atomicMin((unsigned long long *)&s.key[kk][ry * kRegion + rx], (unsigned long long)key);
    }
}

// Splat from a staged window: every pixel of rectangle U (inside the window) for the fractions in fm.
template <typename CT, int WX, int WY>
__device__ __forceinline__ void splat_window(TileSmem &s, const TileParams &p, const WinAcc<CT, WX, WY> &a, Rect U,
                                             uint32_t fm, int RX0, int RY0) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int y = U.y0 + wid; y <= U.y1; y += kThreads / 32) {
        for (int x = U.x0 + lane; x <= U.x1; x += 32) {
            const int i = a.at(x, y);
            splat_pixel(s, p, x, y, __float_as_uint(a.w->depth[i]), __float_as_uint(a.w->mv[0][i]),
                        __float_as_uint(a.w->mv[1][i]), fm, RX0, RY0);
        }
    }
}

// Splat from global memory: candidate 8 x 8 tiles (those whose bounds reach R), 64 threads per candidate.
__device__ void splat_global(TileSmem &s, const TileParams &p, int RX0, int RY0) {
    const int tid = threadIdx.x;
    int bx0, bx1, by0, by1;
    if (!frame_window(p, RX0, RY0, bx0, bx1, by0, by1)) return;
    const int nbxr = bx1 - bx0 + 1;
    const int total = nbxr * (by1 - by0 + 1);
    const size_t plane = (size_t)p.W * p.H;
    for (int base = 0; base < total; base += kThreads) {
        if (tid == 0) s.ncand = 0u;
        __syncthreads();
        const int idx = base + tid;
        if (idx < total) {
            const int by = by0 + idx / nbxr, bx = bx0 + idx % nbxr;
            const float4 b = __ldcg(p.tile_bounds + (size_t)by * p.nbx + bx);
            if (b.x <= b.y) {
                uint32_t fm = 0;
                for (int kk = 0; kk < p.nfrac; ++kk) {
                    int ox0, ox1, oy0, oy1;
                    tile_offsets(b, p.k0 + kk, p.L, ox0, ox1, oy0, oy1);
                    const int tx0 = 8 * bx + ox0, tx1 = 8 * bx + 7 + ox1;
                    const int ty0 = 8 * by + oy0, ty1 = 8 * by + 7 + oy1;
                    if (tx1 >= RX0 && tx0 < RX0 + kRegion && ty1 >= RY0 && ty0 < RY0 + kRegion) fm |= 1u << kk;
                }
                if (fm) {
                    const uint32_t slot = atomicAdd(&s.ncand, 1u);
                    s.cand[slot] = (uint32_t)bx | ((uint32_t)by << 12) | (fm << 24);
                }
            }
        }
        __syncthreads();
        const int nc = (int)s.ncand;
        for (int c0 = 0; c0 < nc; c0 += kThreads / 64) {
            const int ci = c0 + (tid >> 6);
            if (ci < nc) {
                const uint32_t e = s.cand[ci];
                const int bx = (int)(e & 0xFFFu), by = (int)((e >> 12) & 0xFFFu);
                const int x = 8 * bx + (tid & 7), y = 8 * by + ((tid >> 3) & 7);
                if (x < p.W && y < p.H) {
                    const size_t i = (size_t)y * p.W + x;
                    splat_pixel(s, p, x, y, __float_as_uint(__ldg(p.depth + i)), __float_as_uint(__ldg(p.mv + i)),
                                __float_as_uint(__ldg(p.mv + plane + i)), e >> 24, RX0, RY0);
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------------------------
// Coarse levels and bookkeeping of the fill
// ------------------------------------------------------------------------------------------------------------

// Coarse levels of the pyramid (above level 5) for every fraction with invalid tiles, and the value each invalid
// tile receives (its first valid ancestor; 0 when the frame has no valid pixel).  Run by one CTA.
__device__ void coarse_pass(const TileParams &p) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int n5 = p.n5x * p.n5y;
    for (int kk = 0; kk < p.nfrac; ++kk) {
        const uint32_t cnt = __ldcg(&p.fh->ninvalid[kk]);
        if (cnt == 0u) continue;
        const float4 *child = p.nodes + (size_t)kk * n5;
        float4 *cz = p.coarse + (size_t)kk * p.ncoarse;
        int cw = p.n5x, ch = p.n5y, off = 0;
        while (cw > 1 || ch > 1) {
            const int pw = (cw + 1) / 2, ph = (ch + 1) / 2;
            float4 *par = cz + off;
            for (int node = tid; node < pw * ph; node += nt) {
                const int i = node / pw, j = node - i * pw;
                float4 c[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int ci = 2 * i + (q >> 1), cj = 2 * j + (q & 1);
                    c[q] = (ci < ch && cj < cw) ? __ldcg(child + ci * cw + cj) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                par[node] = mean4(c[0], c[1], c[2], c[3]);
            }
            __syncthreads();
            child = par;
            off += pw * ph;
            cw = pw;
            ch = ph;
        }
        for (uint32_t e = tid; e < cnt; e += nt) {
            const uint32_t tile = __ldcg(p.list + (size_t)kk * n5 + e);
            int ax = (int)(tile % (uint32_t)p.n5x), ay = (int)(tile / (uint32_t)p.n5x);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            int w = p.n5x, h = p.n5y, o = 0;
            while (w > 1 || h > 1) {
                const int pw = (w + 1) / 2, ph = (h + 1) / 2;
                ax >>= 1;
                ay >>= 1;
                const float4 c = __ldcg(cz + o + ay * pw + ax);
                if (c.w != 0.0f) {
                    v = c;
                    break;
                }
                o += pw * ph;
                w = pw;
                h = ph;
            }
            p.fillval[(size_t)kk * n5 + e] = make_float4(v.x, v.y, v.z, 1.0f);
        }
        __syncthreads();
    }
}

// Write the level-5 node of a tile for fraction kk; list the tile if it has no valid pixel.
__device__ __forceinline__ void publish_node(const TileParams &p, const FillSmem &fs, int kk, int tile) {
    const float4 node = fs.lv[340];
    const int n5 = p.n5x * p.n5y;
    p.nodes[(size_t)kk * n5 + tile] = node;
    if (node.w == 0.0f) {
        const uint32_t slot = atomicAdd(&p.fh->ninvalid[kk], 1u);
        p.list[(size_t)kk * n5 + slot] = (uint32_t)tile;
    }
}

// Count a finished tile; the CTA that finishes the last tile of the frame runs the coarse pass.
__device__ __forceinline__ void tile_done(const TileParams &p, int *last) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *last = atomicAdd(&p.fh->done, 1u) == (uint32_t)(p.n5x * p.n5y) - 1u;
    __syncthreads();
    if (*last) {
        __threadfence();
        coarse_pass(p);
    }
}

// ------------------------------------------------------------------------------------------------------------
// Stage (b) + (c) of one fraction of a tile, from region keys, through accessor a.  Contains barriers.
// ------------------------------------------------------------------------------------------------------------
template <typename CT, bool FILL, class Acc>
__device__ void finish_fraction(TileSmem &s, const Acc &a, const TileParams &p, int kk, int X0, int Y0, int tile) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k = p.k0 + kk;
    const uint64_t *sk = s.key[kk];
    const uint32_t *sw = reinterpret_cast<const uint32_t *>(sk);  // word 2i+1 = depth bits of key i
    const size_t plane = (size_t)p.W * p.H;
    const int gx = X0 + lane;
    CT *oc = (CT *)p.out_color[kk];
    uint8_t *om = p.out_mask[kk];
    uint8_t mreg[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int y = wid + 8 * j, gy = Y0 + y;
        const bool in = gx < p.W && gy < p.H;
        float c[3] = {0.f, 0.f, 0.f};
        uint8_t m = 0;
        if (in) {
            const int r = (y + 1) * kRegion + (lane + 1);
            const uint64_t kq = sk[r];
            if (kq == kKeyEmpty) {
                m = (uint8_t)EXW_MASK_EMPTY;
            } else if (is_crack(key_dbits(kq), sw[2 * (r - 1) + 1], sw[2 * (r + 1) + 1], sw[2 * (r - kRegion) + 1],
                                sw[2 * (r + kRegion) + 1])) {
                m = (uint8_t)EXW_MASK_CRACK;
            } else {
                const uint32_t lo = (uint32_t)kq;
                float v[3];
                gather_at(a, key_dbits(kq), (int)(lo & 0x3FFFu), (int)(lo >> 14), gx, gy, k, p.L, p.W, p.H, v);
                c[0] = storage_round<CT>(v[0]);
                c[1] = storage_round<CT>(v[1]);
                c[2] = storage_round<CT>(v[2]);
            }
        }
        mreg[j] = m;
        if (FILL) {
            s.fill.v0[0][y][lane] = c[0];
            s.fill.v0[1][y][lane] = c[1];
            s.fill.v0[2][y][lane] = c[2];
            s.fill.m0[y][lane] = in && m == 0;
        } else if (in) {
            const size_t q = (size_t)gy * p.W + gx;
            oc[q] = to_storage<CT>(c[0]);
            oc[plane + q] = to_storage<CT>(c[1]);
            oc[2 * plane + q] = to_storage<CT>(c[2]);
            om[q] = m;
        }
    }
    if (FILL) {
        __syncthreads();
        pull_tile(s.fill);
        const bool tile_valid = s.fill.lv[340].w != 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int y = wid + 8 * j, gy = Y0 + y;
            if (gx >= p.W || gy >= p.H) continue;
            const size_t q = (size_t)gy * p.W + gx;
            om[q] = mreg[j];
            if (!tile_valid) continue;  // every pixel is a hole; the coarse fix-up writes them
            float c0 = s.fill.v0[0][y][lane], c1 = s.fill.v0[1][y][lane], c2 = s.fill.v0[2][y][lane];
            if (mreg[j]) {
                const float4 v = push_value(s.fill, y, lane);
                c0 = v.x;
                c1 = v.y;
                c2 = v.z;
            }
            oc[q] = to_storage<CT>(c0);
            oc[plane + q] = to_storage<CT>(c1);
            oc[2 * plane + q] = to_storage<CT>(c2);
        }
        if (threadIdx.x == 0) publish_node(p, s.fill, kk, tile);
    }
    __syncthreads();
}

}  // namespace exw
