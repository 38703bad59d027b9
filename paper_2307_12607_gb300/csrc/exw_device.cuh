// exw_device.cuh -- device-side building blocks of the warping fast path (sm_103a).
//
// Everything a kernel needs per pixel lives here so that the staged kernels (exw_splat_motion, exw_warp,
// exw_fill_holes), the fused kernels and the batched kernel run literally the same arithmetic and agree bit for
// bit.  Source data is read through an accessor (global memory or a shared-memory window staged by TMA).
#pragma once

#include <cstdint>
#include <cuda_fp16.h>

namespace exw {

constexpr uint64_t kKeyEmpty = ~0ull;
constexpr int kFillTile = 32;          // fill tile side: pyramid levels 1..5 live in shared memory
constexpr int kRegion = kFillTile + 2; // fill tile plus a one-pixel ring (the crack rule reads 4-neighbours)
constexpr int kRegionN = kRegion * kRegion;
constexpr int kBoundsBlock = 8;        // side of the motion-bounds tiles
constexpr int kMaxFrac = 3;

// ------------------------------------------------------------------------------------------------------------
// Validity of source pixels
// ------------------------------------------------------------------------------------------------------------

// Positive finite depth (subnormals included): bits in [1, 0x7F7FFFFF].
__device__ __forceinline__ bool depth_ok(uint32_t dbits) { return (dbits - 1u) < 0x7F7FFFFFu; }
__device__ __forceinline__ bool finite_bits(uint32_t b) { return (b & 0x7F800000u) != 0x7F800000u; }

__device__ __forceinline__ float pow2_neg(int n) {  // 2^-n for n in [-126, 126]
    return __int_as_float((127 - n) << 23);
}

// ------------------------------------------------------------------------------------------------------------
// Exact target offset off = floor(1/2 + k * mv / 2^L).
//
// A finite float mv is sM * 2^(e - 150) with |sM| < 2^24, so k*mv/2^L = k*sM * 2^-n with n = 150 + L - e.  For
// k <= 64, |k*sM| < 2^30, and rounding half up is an arithmetic shift: off = (k*sM + 2^(n-1)) >> n.  n >= 32 means
// |d| < 1/4 (off = 0); n <= 0 means |d| >= 2^23 (cannot land in any frame).  The decomposition is shared by all
// fractions, so each extra fraction costs one multiply-add and one shift.
// ------------------------------------------------------------------------------------------------------------
struct AxisDec {
    int sM;  // signed significand
    int n;   // right-shift amount
};

__device__ __forceinline__ AxisDec axis_dec(uint32_t u, int L) {
    const uint32_t E = (u >> 23) & 0xFFu;
    const int M = (int)((u & 0x7FFFFFu) | (E ? 0x800000u : 0u));
    AxisDec d;
    d.sM = (u >> 31) ? -M : M;
    d.n = 150 + L - (E ? (int)E : 1);
    return d;
}

// Returns false when the offset cannot land in any frame (|offset| >= 2^23).
__device__ __forceinline__ bool axis_off(const AxisDec &d, int k, int &off) {
    if (d.n >= 32 || d.sM == 0 || k == 0) {
        off = 0;
        return true;
    }
    if (d.n <= 0) return false;
    off = (k * d.sM + (1 << (d.n - 1))) >> d.n;
    return true;
}

__device__ __forceinline__ int axis_off_of(uint32_t bits, int k, int L) {  // for clamped bounds (always lands)
    int off = 0;
    axis_off(axis_dec(bits, L), k, off);
    return off;
}

// Residual rho = t - k*mv/2^L for a winner displaced by the whole-pixel offset t (|rho| <= 1/2).  One fused
// multiply-add computes the exact value rounded once, i.e. the correctly rounded residual.  Its sign is exact
// except when |rho| < 2^-150 rounds to zero, which needs t = 0 and a subnormal mv; then rho = -d has the sign of
// -mv.  sgn is -1, 0 or +1.
__device__ __forceinline__ float residual(float mv, int k, int L, int t, int &sgn) {
    const float r = fmaf(-(float)k * pow2_neg(L), mv, (float)t);
    sgn = (r > 0.0f) - (r < 0.0f);
    if (sgn == 0 && t == 0 && k != 0 && mv != 0.0f) sgn = mv > 0.0f ? -1 : 1;
    return r;
}

// Key packings.  In global memory: (depth bits << 32) | (y * W + x).  In shared memory the low word is
// (y << 14) | x, which orders exactly like y * W + x for x < 2^14 and needs no division to unpack.
__device__ __forceinline__ uint64_t pack_key_local(uint32_t dbits, int x, int y) {
    return ((uint64_t)dbits << 32) | (uint32_t)((y << 14) | x);
}
__device__ __forceinline__ uint64_t pack_key_global(uint32_t dbits, uint32_t idx) {
    return ((uint64_t)dbits << 32) | idx;
}
__device__ __forceinline__ uint32_t key_dbits(uint64_t key) { return (uint32_t)(key >> 32); }

// ------------------------------------------------------------------------------------------------------------
// Colour types
// ------------------------------------------------------------------------------------------------------------
template <typename CT> __device__ __forceinline__ float to_f(CT v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

template <typename CT> __device__ __forceinline__ float load_c(const CT *p) { return to_f<CT>(__ldg(p)); }

template <typename CT> __device__ __forceinline__ CT to_storage(float v);
template <> __device__ __forceinline__ float to_storage<float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_storage<__half>(float v) { return __float2half_rn(v); }

template <typename CT> __device__ __forceinline__ float storage_round(float v) { return v; }
template <> __device__ __forceinline__ float storage_round<__half>(float v) {
    return __half2float(__float2half_rn(v));
}

// ------------------------------------------------------------------------------------------------------------
// Source accessors: global memory, or a shared-memory window [x0, x0 + WX) x [y0, y0 + WY) staged by TMA.
// ------------------------------------------------------------------------------------------------------------
template <typename CT>
struct GlobalAcc {
    const CT *col;
    const float *depth;
    const float *mv;
    int W;
    size_t plane;
    __device__ __forceinline__ size_t at(int x, int y) const { return (size_t)y * W + x; }
    __device__ __forceinline__ float d(int x, int y) const { return __ldg(depth + at(x, y)); }
    __device__ __forceinline__ float mx(int x, int y) const { return __ldg(mv + at(x, y)); }
    __device__ __forceinline__ float my(int x, int y) const { return __ldg(mv + plane + at(x, y)); }
    __device__ __forceinline__ float c(int ch, int x, int y) const { return load_c<CT>(col + ch * plane + at(x, y)); }
};

template <typename CT, int WX, int WY>
struct Window {  // TMA destinations: [y][x] per plane
    float depth[WY * WX];
    float mv[2][WY * WX];
    CT col[3][WY * WX];
};

template <typename CT, int WX, int WY>
struct WinAcc {
    const Window<CT, WX, WY> *w;
    int x0, y0;
    __device__ __forceinline__ int at(int x, int y) const { return (y - y0) * WX + (x - x0); }
    __device__ __forceinline__ float d(int x, int y) const { return w->depth[at(x, y)]; }
    __device__ __forceinline__ float mx(int x, int y) const { return w->mv[0][at(x, y)]; }
    __device__ __forceinline__ float my(int x, int y) const { return w->mv[1][at(x, y)]; }
    __device__ __forceinline__ float c(int ch, int x, int y) const { return to_f<CT>(w->col[ch][at(x, y)]); }
};

// ------------------------------------------------------------------------------------------------------------
// Stage (b) for one target pixel
// ------------------------------------------------------------------------------------------------------------

// Crack rule: at least 3 non-empty 4-neighbours nearer than the target by more than D_q / 32.  Only the depth
// words of the keys matter: an empty key's word (all ones) is a NaN and never counts.  32 * (Dq - Dn) > Dq is
// exact in float: within a factor of 2 the difference is exact (Sterbenz), outside it both sides are far from
// the threshold.
__device__ __forceinline__ bool is_crack(uint32_t dq, uint32_t d0, uint32_t d1, uint32_t d2, uint32_t d3) {
    const float Dq = __uint_as_float(dq);
    int c = 0;
    c += (32.0f * (Dq - __uint_as_float(d0)) > Dq);
    c += (32.0f * (Dq - __uint_as_float(d1)) > Dq);
    c += (32.0f * (Dq - __uint_as_float(d2)) > Dq);
    c += (32.0f * (Dq - __uint_as_float(d3)) > Dq);
    return c >= 3;
}

// Tap agreement |D(t) - D(p)| <= D(p) / 32, exact in float by the same argument.  A NaN, infinite or
// non-positive tap depth fails it.
__device__ __forceinline__ bool tap_agrees(float Dt, float Dp) { return 32.0f * fabsf(Dt - Dp) <= Dp; }

// Bilinear gather for target (qx, qy) at its winner (px, py): taps p, p+sx, p+sy, p+sx+sy (in this order),
// renormalised over the participating ones.  Returns the colour in out[3].
template <class Acc>
__device__ __forceinline__ void gather_at(const Acc &a, uint32_t dbits, int px, int py, int qx, int qy, int k, int L,
                                          int W, int H, float out[3]) {
    int sx, sy;
    const float rx = residual(a.mx(px, py), k, L, qx - px, sx);
    const float ry = residual(a.my(px, py), k, L, qy - py, sy);
    const float Dp = __uint_as_float(dbits);
    const float ax = fabsf(rx), ay = fabsf(ry);
    const float wx0 = 1.0f - ax, wy0 = 1.0f - ay;
    const int tx = px + sx, ty = py + sy;
    const bool inx = sx != 0 && (unsigned)tx < (unsigned)W;
    const bool iny = sy != 0 && (unsigned)ty < (unsigned)H;
    float w = wx0 * wy0;
    float den = w;
    float n0 = w * a.c(0, px, py), n1 = w * a.c(1, px, py), n2 = w * a.c(2, px, py);
    if (inx && tap_agrees(a.d(tx, py), Dp)) {
        w = ax * wy0;
        den += w;
        n0 += w * a.c(0, tx, py);
        n1 += w * a.c(1, tx, py);
        n2 += w * a.c(2, tx, py);
    }
    if (iny) {
        if (tap_agrees(a.d(px, ty), Dp)) {
            w = wx0 * ay;
            den += w;
            n0 += w * a.c(0, px, ty);
            n1 += w * a.c(1, px, ty);
            n2 += w * a.c(2, px, ty);
        }
        if (inx && tap_agrees(a.d(tx, ty), Dp)) {
            w = ax * ay;
            den += w;
            n0 += w * a.c(0, tx, ty);
            n1 += w * a.c(1, tx, ty);
            n2 += w * a.c(2, tx, ty);
        }
    }
    const float inv = __frcp_rn(den);
    out[0] = n0 * inv;
    out[1] = n1 * inv;
    out[2] = n2 * inv;
}

// ------------------------------------------------------------------------------------------------------------
// Pull-push inside one 32 x 32 fill tile (levels 1..5 of the frame's pyramid: tiles are aligned to 32, so every
// ancestor up to level 5 of a tile pixel is computed from that tile alone; out-of-frame pixels are invalid,
// which reproduces the ceil-halving level sizes).
// ------------------------------------------------------------------------------------------------------------
struct FillSmem {
    float v0[3][kFillTile][kFillTile];  // level 0 colour (already rounded to the storage type)
    uint8_t m0[kFillTile][kFillTile];   // level 0 validity
    float4 lv[341];                     // levels 1..5: 16x16, 8x8, 4x4, 2x2, 1x1 (rgb, validity)
};
__device__ __forceinline__ int lv_offset(int l) {  // l in 1..5
    return l == 1 ? 0 : l == 2 ? 256 : l == 3 ? 320 : l == 4 ? 336 : 340;
}

// Mean of the valid children, taken in the order (0,0),(0,1),(1,0),(1,1) (row, column).
__device__ __forceinline__ float4 mean4(float4 c0, float4 c1, float4 c2, float4 c3) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    int cnt = 0;
    if (c0.w != 0.0f) { a0 += c0.x; a1 += c0.y; a2 += c0.z; ++cnt; }
    if (c1.w != 0.0f) { a0 += c1.x; a1 += c1.y; a2 += c1.z; ++cnt; }
    if (c2.w != 0.0f) { a0 += c2.x; a1 += c2.y; a2 += c2.z; ++cnt; }
    if (c3.w != 0.0f) { a0 += c3.x; a1 += c3.y; a2 += c3.z; ++cnt; }
    if (cnt == 0) return make_float4(0.f, 0.f, 0.f, 0.f);
    const float fc = (float)cnt;
    return make_float4(a0 / fc, a1 / fc, a2 / fc, 1.0f);
}

// Build levels 1..5 from v0/m0.  Must be called by all threads of the block (contains barriers); v0/m0 must be
// complete on entry.
__device__ __forceinline__ void pull_tile(FillSmem &s) {
    const int t = threadIdx.x;
    const int nt = blockDim.x;
    for (int node = t; node < 256; node += nt) {
        const int i = node >> 4, j = node & 15;
        const int y = 2 * i, x = 2 * j;
        float4 c[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int yy = y + (q >> 1), xx = x + (q & 1);
            c[q] = s.m0[yy][xx] ? make_float4(s.v0[0][yy][xx], s.v0[1][yy][xx], s.v0[2][yy][xx], 1.0f)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        s.lv[node] = mean4(c[0], c[1], c[2], c[3]);
    }
    __syncthreads();
#pragma unroll 1
    for (int l = 2; l <= 5; ++l) {
        const int lg = 5 - l;                 // log2 of this level's side
        const int side = 1 << lg, cside = side * 2;
        const int po = lv_offset(l), co = lv_offset(l - 1);
        for (int node = t; node < side * side; node += nt) {
            const int i = node >> lg, j = node & (side - 1);
            const float4 *c = s.lv + co + (2 * i) * cside + 2 * j;
            s.lv[po + node] = mean4(c[0], c[1], c[cside], c[cside + 1]);
        }
        __syncthreads();
    }
}

// Value pushed down to tile pixel (y, x): its first valid ancestor among levels 1..5; .w = 0 when the whole
// tile is invalid (the coarse levels decide).
__device__ __forceinline__ float4 push_value(const FillSmem &s, int y, int x) {
#pragma unroll
    for (int l = 1; l <= 5; ++l) {
        const int side = kFillTile >> l;
        const float4 v = s.lv[lv_offset(l) + (y >> l) * side + (x >> l)];
        if (v.w != 0.0f) return v;
    }
    return make_float4(0.f, 0.f, 0.f, 0.f);
}

// Ordered encoding of a non-NaN float for unsigned atomicMax: larger float <-> larger code, and 0 is below every
// code (the "nothing seen" value).
__device__ __forceinline__ uint32_t float_order(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_unorder(uint32_t c) {
    return __uint_as_float((c & 0x80000000u) ? (c & 0x7FFFFFFFu) : ~c);
}

}  // namespace exw
