// exw_tile.cuh -- per-tile passes shared by the forward kernels (one 32 x 32 target tile Q per CTA iteration).
//
// A tile's keys cover Q plus a one-pixel ring R (the crack rule reads 4-neighbours).  The splat takes every
// source pixel that can land in R -- found from the 8 x 8 motion bounds -- either from a TMA-staged shared-memory
// window or from global memory; the gather reads through the matching accessor.  Per fraction the tile is then
// gathered, hole-marked, filled from pyramid levels 1..5 and stored.  A CTA has 16 warps; warp w handles tile rows
// 2w and 2w+1 with lane = column, so each row access is one 128-byte line.
#pragma once

#include "exw_device.cuh"
#include "exw_internal.h"

namespace exw {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;

struct TileSmem {
    uint64_t key[kMaxFrac][kRegionN];  // region keys; in uniform tiles reused as depth words (uint32 per cell)
    TilePyr pyr;                       // pyramid levels 1..5 of the fraction being filled
    uint32_t cand[kThreads];
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
        const int ox0 = axis_off(fx0, k), ox1 = axis_off(fx1, k);
        const int oy0 = axis_off(fy0, k), oy1 = axis_off(fy1, k);
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

// The four motion bounds of a tile decoded once (axis_dec); each fraction's offsets [ox0, ox1] x [oy0, oy1] then
// cost four shift-adds (axis_off of the decoded bounds: the offset is monotone in the motion).
struct BoundsDec {
    AxisDec x0, x1, y0, y1;
};
__device__ __forceinline__ BoundsDec bounds_dec(const float4 &b, int L) {
    return BoundsDec{axis_dec(__float_as_uint(b.x), L), axis_dec(__float_as_uint(b.y), L),
                     axis_dec(__float_as_uint(b.z), L), axis_dec(__float_as_uint(b.w), L)};
}
__device__ __forceinline__ void bounds_offsets(const BoundsDec &d, int k, int &ox0, int &ox1, int &oy0, int &oy1) {
    ox0 = axis_off(d.x0, k);
    ox1 = axis_off(d.x1, k);
    oy0 = axis_off(d.y0, k);
    oy1 = axis_off(d.y1, k);
}

// Splat one source pixel (x, y) for the fractions in fm into the region keys.
__device__ __forceinline__ void splat_pixel(TileSmem &s, const TileParams &p, int x, int y, uint32_t db, uint32_t ux,
                                            uint32_t uy, uint32_t fm, int RX0, int RY0) {
    if (!depth_ok(db) || !finite_bits(ux) || !finite_bits(uy)) return;
    const AxisDec dx = axis_dec(ux, p.L), dy = axis_dec(uy, p.L);
    if (!dx.land || !dy.land) return;
    const uint64_t key = pack_key_local(db, x, y);
    for (int kk = 0; kk < p.nfrac; ++kk) {
        if (!(fm & (1u << kk))) continue;
        const int k = p.k0 + kk;
        const int gx = x + axis_off(dx, k), gy = y + axis_off(dy, k);
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
    for (int y = U.y0 + wid; y <= U.y1; y += kWarps) {
        for (int x = U.x0 + lane; x <= U.x1; x += 32) {
            const int i = a.at(x, y);
            splat_pixel(s, p, x, y, __float_as_uint(a.w->depth[i]), __float_as_uint(a.w->mv[0][i]),
                        __float_as_uint(a.w->mv[1][i]), fm, RX0, RY0);
        }
    }
}

// Splat from global memory: candidate 8 x 8 tiles (those whose bounds reach R), 64 threads per candidate.
__device__ inline void splat_global(TileSmem &s, const TileParams &p, int RX0, int RY0) {
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
                const BoundsDec bd = bounds_dec(b, p.L);
                for (int kk = 0; kk < p.nfrac; ++kk) {
                    int ox0, ox1, oy0, oy1;
                    bounds_offsets(bd, p.k0 + kk, ox0, ox1, oy0, oy1);
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

// Uniform tile: every source pixel that can land in R moves by one motion (mx, my), so for fraction kk the target
// q can only receive the source q - o, and does when that pixel has a valid depth and exactly that motion (a pixel
// there with another motion sits in a tile whose bounds cannot reach R, so it lands elsewhere).  Writes its depth
// word, or all ones for an empty target, for every cell of R: the key words the splat would produce.
template <typename CT, int WX, int WY>
__device__ __forceinline__ void uniform_words(uint32_t *dw, const TileParams &p, const WinAcc<CT, WX, WY> &a, int ox,
                                             int oy, float mx, float my, int RX0, int RY0) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 6; ++i) {  // 34 x 34 cells: rows wid + 16 (i >> 1), columns lane + 32 (i & 1)
        const int ry = wid + kWarps * (i >> 1), rx = lane + 32 * (i & 1);
        if (ry >= kRegion || rx >= kRegion) continue;
        const int qx = RX0 + rx, qy = RY0 + ry;
        const int px = qx - ox, py = qy - oy;
        uint32_t w = 0xFFFFFFFFu;
        if ((unsigned)qx < (unsigned)p.W && (unsigned)qy < (unsigned)p.H && (unsigned)px < (unsigned)p.W &&
            (unsigned)py < (unsigned)p.H) {
            const int ai = a.at(px, py);
            const uint32_t db = __float_as_uint(a.w->depth[ai]);
            if (depth_ok(db) && a.w->mv[0][ai] == mx && a.w->mv[1][ai] == my) w = db;
        }
        dw[ry * kRegion + rx] = w;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Coarse levels and bookkeeping of the fill
// ------------------------------------------------------------------------------------------------------------

// Coarse levels of the pyramid (above level 5) for every fraction with invalid tiles, and the value each invalid
// tile receives (its first valid ancestor; 0 when the frame has no valid pixel).  Run by one CTA.
__device__ inline void coarse_pass(const TileParams &p) {
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

// Write the level-5 node of a tile for fraction kk; list the tile if it has no valid pixel.  Thread 0 only.
__device__ __forceinline__ void publish_node(const TileParams &p, float4 node, int kk, int tile) {
    const int n5 = p.n5x * p.n5y;
    p.nodes[(size_t)kk * n5 + tile] = node;
    if (node.w == 0.0f) {
        const uint32_t slot = atomicAdd(&p.fh->ninvalid[kk], 1u);
        p.list[(size_t)kk * n5 + slot] = (uint32_t)tile;
    }
}

// Count a finished tile; the CTA that finishes the last tile of the frame runs the coarse pass.  Only thread 0
// wrote the tile's nodes and list entries, so only it needs the fence before counting.
__device__ __forceinline__ void tile_done(const TileParams &p, int *last) {
    if (threadIdx.x == 0) {
        __threadfence();
        *last = atomicAdd(&p.fh->done, 1u) == (uint32_t)(p.n5x * p.n5y) - 1u;
    }
    __syncthreads();
    if (*last) {
        __threadfence();
        coarse_pass(p);
    }
}

// ------------------------------------------------------------------------------------------------------------
// Fill and store one fraction of a tile: c[j] (.w = validity) are this thread's two pixels (tile rows 2w + j,
// column lane), m[j] their mask bytes (for pixels in the frame).  write_valid: store valid pixels too (fused pass)
// or only the filled holes (in-place fill); write_mask: store the mask.  Contains two block barriers.
// ------------------------------------------------------------------------------------------------------------
template <typename CT>
__device__ __forceinline__ void fill_store(const TileParams &p, TilePyr &pyr, const float4 c[2], const uint8_t m[2],
                                           int kk, int X0, int Y0, int tile, bool write_valid, bool write_mask) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t plane = (size_t)p.W * p.H;
    const int gx = X0 + lane;
    CT *oc = (CT *)p.out_color[kk];
    const float4 n1 = build_pyramid(pyr, c[0], c[1]);
    const bool tile_valid = pyr.l5.w != 0.0f;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int gy = Y0 + 2 * wid + j;
        if (gx >= p.W || gy >= p.H) continue;
        const size_t q = (size_t)gy * p.W + gx;
        if (write_mask) p.out_mask[kk][q] = m[j];
        if (!tile_valid) continue;  // every pixel is a hole; the coarse fix-up writes them
        const bool hole = m[j] != 0;
        if (!hole && !write_valid) continue;
        const float4 v = hole ? push_value(pyr, n1) : c[j];
        oc[q] = to_storage<CT>(v.x);
        oc[plane + q] = to_storage<CT>(v.y);
        oc[2 * plane + q] = to_storage<CT>(v.z);
    }
    if (threadIdx.x == 0) publish_node(p, pyr.l5, kk, tile);
}

// ------------------------------------------------------------------------------------------------------------
// Winner sources of a region cell r: the splat keys, or (uniform tiles) depth words plus one whole-pixel offset.
// ------------------------------------------------------------------------------------------------------------
struct KeySource {
    static constexpr bool kUniform = false;
    const uint32_t *w;  // the keys as 32-bit words: 2r = (y << 14) | x, 2r + 1 = depth bits
    float mx, my;       // unused
    int ox, oy;         // unused
    __device__ __forceinline__ uint32_t dword(int r) const { return w[2 * r + 1]; }
    __device__ __forceinline__ void winner(int r, int, int, int &px, int &py) const {
        const uint32_t lo = w[2 * r];
        px = (int)(lo & 0x3FFFu);
        py = (int)(lo >> 14);
    }
};
struct UniformSource {
    static constexpr bool kUniform = true;
    const uint32_t *w;  // depth word per cell
    float mx, my;       // the tile's one motion
    int ox, oy;         // whole-pixel offset of the fraction
    __device__ __forceinline__ uint32_t dword(int r) const { return w[r]; }
    __device__ __forceinline__ void winner(int, int gx, int gy, int &px, int &py) const {
        px = gx - ox;
        py = gy - oy;
    }
};

// ------------------------------------------------------------------------------------------------------------
// Stage (b) + (c) of one fraction of a tile, from the winners of the region, through accessor a.  With FILL,
// contains the two barriers of the pyramid.
// ------------------------------------------------------------------------------------------------------------
template <typename CT, bool FILL, class Acc, class Src>
__device__ void finish_fraction(TileSmem &s, const Acc &a, const Src &src, const TileParams &p, int kk, int X0, int Y0,
                                int tile) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k = p.k0 + kk;
    const size_t plane = (size_t)p.W * p.H;
    const int gx = X0 + lane;
    float4 c[2];
    uint8_t m[2];
    // The two pixels of this thread go through each step together, so their loads overlap.  Pixels without a
    // winner (empty, crack, outside the frame) gather at a safe position and their result is discarded.
    uint32_t dq[2];
    int px[2], py[2];
    bool ok[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int y = 2 * wid + j, gy = Y0 + y;
        const bool in = gx < p.W && gy < p.H;
        const int r = (y + 1) * kRegion + (lane + 1);
        dq[j] = src.dword(r);
        const bool empty = dq[j] == 0xFFFFFFFFu;
        const bool crack = !empty && is_crack(dq[j], src.dword(r - 1), src.dword(r + 1), src.dword(r - kRegion),
                                              src.dword(r + kRegion));
        m[j] = !in ? (uint8_t)0 : empty ? (uint8_t)EXW_MASK_EMPTY : crack ? (uint8_t)EXW_MASK_CRACK : (uint8_t)0;
        ok[j] = in && !empty && !crack;
        src.winner(r, gx, gy, px[j], py[j]);
        if (!ok[j]) {
            px[j] = a.safe_x();
            py[j] = a.safe_y();
        }
    }
    // Residuals: one per fraction in a uniform tile, else from each winner's motion.
    int usx = 0, usy = 0;
    float urx = 0.0f, ury = 0.0f;
    if (Src::kUniform) {
        urx = residual(src.mx, k, p.L, src.ox, usx);
        ury = residual(src.my, k, p.L, src.oy, usy);
    }
    decltype(a.at(0, 0)) i00[2], i10[2], i01[2], i11[2];
    float wx0[2], wx1[2], wy0[2], wy1[2];
    bool ex[2], ey[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        i00[j] = a.at(px[j], py[j]);
        int sx = usx, sy = usy;
        float rx = urx, ry = ury;
        if (!Src::kUniform) {
            rx = residual(a.mx(i00[j]), k, p.L, gx - px[j], sx);
            ry = residual(a.my(i00[j]), k, p.L, Y0 + 2 * wid + j - py[j], sy);
        }
        wx1[j] = fabsf(rx);
        wy1[j] = fabsf(ry);
        wx0[j] = 1.0f - wx1[j];
        wy0[j] = 1.0f - wy1[j];
        ex[j] = sx != 0 && (unsigned)(px[j] + sx) < (unsigned)p.W;
        ey[j] = sy != 0 && (unsigned)(py[j] + sy) < (unsigned)p.H;
        i10[j] = ex[j] ? i00[j] + sx : i00[j];
        const auto ir = sy > 0 ? i00[j] + a.stride() : i00[j] - a.stride();
        i01[j] = ey[j] ? ir : i00[j];
        i11[j] = (ex[j] && ey[j]) ? ir + sx : i00[j];
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float Dp = __uint_as_float(dq[j]);
        const bool a10 = ex[j] && tap_agrees(a.d(i10[j]), Dp);
        const bool a01 = ey[j] && tap_agrees(a.d(i01[j]), Dp);
        const bool a11 = ex[j] && ey[j] && tap_agrees(a.d(i11[j]), Dp);
        const float w00 = __fmul_rn(wx0[j], wy0[j]);
        const float w10 = a10 ? __fmul_rn(wx1[j], wy0[j]) : 0.0f;
        const float w01 = a01 ? __fmul_rn(wx0[j], wy1[j]) : 0.0f;
        const float w11 = a11 ? __fmul_rn(wx1[j], wy1[j]) : 0.0f;
        const float den = weight_sum(w00, w10, w01, w11);
        float v[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float n = __fmul_rn(w00, a.c(ch, i00[j]));
            const float c10 = a.c(ch, i10[j]), c01 = a.c(ch, i01[j]), c11 = a.c(ch, i11[j]);
            n = a10 ? fmaf(w10, c10, n) : n;
            n = a01 ? fmaf(w01, c01, n) : n;
            n = a11 ? fmaf(w11, c11, n) : n;
            v[ch] = n;
        }
        const float inv = __frcp_rn(den);
        const bool okj = ok[j];
        c[j] = make_float4(okj ? storage_round<CT>(__fmul_rn(v[0], inv)) : 0.0f,
                           okj ? storage_round<CT>(__fmul_rn(v[1], inv)) : 0.0f,
                           okj ? storage_round<CT>(__fmul_rn(v[2], inv)) : 0.0f, okj ? 1.0f : 0.0f);
    }
    if (!FILL) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int gy = Y0 + 2 * wid + j;
            if (gx >= p.W || gy >= p.H) continue;
            const size_t q = (size_t)gy * p.W + gx;
            CT *oc = (CT *)p.out_color[kk];
            oc[q] = to_storage<CT>(c[j].x);
            oc[plane + q] = to_storage<CT>(c[j].y);
            oc[2 * plane + q] = to_storage<CT>(c[j].z);
            p.out_mask[kk][q] = m[j];
        }
    } else {
        fill_store<CT>(p, s.pyr, c, m, kk, X0, Y0, tile, true, true);
    }
}

// The splat keys of fraction kk as a winner source.
__device__ __forceinline__ KeySource key_source(const TileSmem &s, int kk) {
    return KeySource{reinterpret_cast<const uint32_t *>(s.key[kk]), 0.0f, 0.0f, 0, 0};
}

}  // namespace exw
