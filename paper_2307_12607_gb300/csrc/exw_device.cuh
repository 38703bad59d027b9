// exw_device.cuh -- device-side building blocks of the warping fast path (sm_103a).
//
// Everything a kernel needs per pixel lives here so that the staged kernels (exw_splat_motion, exw_warp,
// exw_fill_holes) and the fused/batched kernels run literally the same arithmetic and agree bit for bit.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>

namespace exw {

constexpr uint64_t kKeyEmpty = ~0ull;
constexpr int kFillTile = 32;          // fill tile side: pyramid levels 1..5 live in shared memory
constexpr int kRegion = kFillTile + 2; // fill tile plus a one-pixel ring (the crack rule reads 4-neighbours)
constexpr int kBoundsBlock = 8;        // side of the motion-bounds tiles
constexpr int kMaxFrac = 3;

// ------------------------------------------------------------------------------------------------------------
// Validity of source pixels
// ------------------------------------------------------------------------------------------------------------

// Positive finite depth (subnormals included): bits in [1, 0x7F7FFFFF].
__device__ __forceinline__ bool depth_ok(uint32_t dbits) { return (dbits - 1u) < 0x7F7FFFFFu; }
__device__ __forceinline__ bool finite_bits(uint32_t b) { return (b & 0x7F800000u) != 0x7F800000u; }

// ------------------------------------------------------------------------------------------------------------
// Exact target offset: off = floor(1/2 + k * mv / 2^L) and the residual rho = off - k * mv / 2^L.
//
// A float mv is (+-)M * 2^(e - 150) with M < 2^24, so k*mv/2^L = (+-)K * 2^-n with K = k*M < 2^30 (k <= 64) and
// n = 150 + L - e.  Rounding half up is then an arithmetic shift: off = (sK + 2^(n-1)) >> n, and the remainder r
// of that shift gives rho * 2^n = 2^(n-1) - r exactly in 32 bits.  n >= 32 means |d| < 1/4 (off = 0); n <= 0
// means |d| >= 2^23, which cannot land in any frame.  All integer, so every thread agrees with exact arithmetic.
// ------------------------------------------------------------------------------------------------------------
struct AxisStep {
    int off;    // the whole-pixel offset (meaningful when ok)
    float rho;  // residual rounded to float; its sign is exact
    int sgn;    // sign of the exact residual: -1, 0 or +1
    bool ok;    // false when |offset| >= 2^23 (cannot land)
};

__device__ __forceinline__ float pow2_neg(int n) {  // 2^-n for n in [-126, 126]
    return __int_as_float((127 - n) << 23);
}

__device__ __forceinline__ AxisStep axis_step(uint32_t u, int k, int L) {
    AxisStep r;
    const uint32_t E = (u >> 23) & 0xFFu;
    const uint32_t m = u & 0x7FFFFFu;
    const uint32_t M = E ? (m | 0x800000u) : m;
    const int e = E ? (int)E : 1;
    const uint32_t K = (uint32_t)k * M;
    const bool neg = (u >> 31) != 0u;
    r.off = 0;
    r.rho = 0.0f;
    r.sgn = 0;
    r.ok = true;
    if (K == 0u) return r;
    const int n = 150 + L - e;
    if (n <= 0) {
        r.ok = false;
        return r;
    }
    if (n >= 32) {  // |d| < 1/4: off = 0 and rho = -d
        float mag = __uint2float_rn(K) * 0x1p-64f;
        mag = mag * pow2_neg(n - 64);
        r.rho = neg ? mag : -mag;
        r.sgn = neg ? 1 : -1;
        return r;
    }
    const int sK = neg ? -(int)K : (int)K;
    const int half = 1 << (n - 1);
    const int a = sK + half;
    r.off = a >> n;
    const uint32_t rem = (uint32_t)a & ((1u << n) - 1u);
    const int num = half - (int)rem;
    r.sgn = (num > 0) - (num < 0);
    r.rho = __int2float_rn(num) * pow2_neg(n);
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
// Colour access
// ------------------------------------------------------------------------------------------------------------
template <typename CT> __device__ __forceinline__ float load_c(const CT *p);
template <> __device__ __forceinline__ float load_c<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_c<__half>(const __half *p) { return __half2float(__ldg(p)); }

template <typename CT> __device__ __forceinline__ CT to_storage(float v);
template <> __device__ __forceinline__ float to_storage<float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_storage<__half>(float v) { return __float2half_rn(v); }

template <typename CT> __device__ __forceinline__ float storage_round(float v) { return v; }
template <> __device__ __forceinline__ float storage_round<__half>(float v) {
    return __half2float(__float2half_rn(v));
}

// ------------------------------------------------------------------------------------------------------------
// Stage (b) for one target pixel
// ------------------------------------------------------------------------------------------------------------

// Crack rule: at least 3 non-empty 4-neighbours nearer than the target by more than D_q / 32.
// 32 * (Dq - Dn) > Dq is exact in float: within a factor of 2 the difference is exact (Sterbenz), and outside it
// both sides are far from the threshold.  Empty neighbours (all-ones key, NaN depth bits) never count.
__device__ __forceinline__ bool is_crack(uint64_t kq, uint64_t k0, uint64_t k1, uint64_t k2, uint64_t k3) {
    const float Dq = __uint_as_float(key_dbits(kq));
    int c = 0;
    c += (k0 != kKeyEmpty) && (32.0f * (Dq - __uint_as_float(key_dbits(k0))) > Dq);
    c += (k1 != kKeyEmpty) && (32.0f * (Dq - __uint_as_float(key_dbits(k1))) > Dq);
    c += (k2 != kKeyEmpty) && (32.0f * (Dq - __uint_as_float(key_dbits(k2))) > Dq);
    c += (k3 != kKeyEmpty) && (32.0f * (Dq - __uint_as_float(key_dbits(k3))) > Dq);
    return c >= 3;
}

// Tap agreement |D(t) - D(p)| <= D(p) / 32, exact in float by the same argument.  A NaN, infinite or
// non-positive tap depth fails it.
__device__ __forceinline__ bool tap_agrees(float Dt, float Dp) { return 32.0f * fabsf(Dt - Dp) <= Dp; }

// Bilinear gather at the winner (px, py) of target q: taps p, p+sx, p+sy, p+sx+sy (in this order), renormalised
// over the participating ones.  Returns the colour in out[3].
template <typename CT>
__device__ __forceinline__ void gather_pixel(uint32_t dbits, int px, int py, int k, int L, const CT *__restrict__ col,
                                             const float *__restrict__ depth, const float *__restrict__ mv, int W,
                                             int H, size_t plane, float out[3]) {
    const size_t p = (size_t)py * W + px;
    const AxisStep ax = axis_step(__float_as_uint(__ldg(mv + p)), k, L);
    const AxisStep ay = axis_step(__float_as_uint(__ldg(mv + plane + p)), k, L);
    const float Dp = __uint_as_float(dbits);
    float wx0 = 1.0f, wx1 = 0.0f, wy0 = 1.0f, wy1 = 0.0f;
    if (ax.sgn) { const float a = fabsf(ax.rho); wx0 = 1.0f - a; wx1 = a; }
    if (ay.sgn) { const float a = fabsf(ay.rho); wy0 = 1.0f - a; wy1 = a; }
    const int tx = px + ax.sgn, ty = py + ay.sgn;
    const bool inx = ax.sgn != 0 && tx >= 0 && tx < W;
    const bool iny = ay.sgn != 0 && ty >= 0 && ty < H;
    float w = wx0 * wy0;
    float den = w;
    float n0 = w * load_c<CT>(col + p);
    float n1 = w * load_c<CT>(col + plane + p);
    float n2 = w * load_c<CT>(col + 2 * plane + p);
    if (inx) {
        const size_t t = (size_t)py * W + tx;
        if (tap_agrees(__ldg(depth + t), Dp)) {
            w = wx1 * wy0;
            den += w;
            n0 += w * load_c<CT>(col + t);
            n1 += w * load_c<CT>(col + plane + t);
            n2 += w * load_c<CT>(col + 2 * plane + t);
        }
    }
    if (iny) {
        const size_t t = (size_t)ty * W + px;
        if (tap_agrees(__ldg(depth + t), Dp)) {
            w = wx0 * wy1;
            den += w;
            n0 += w * load_c<CT>(col + t);
            n1 += w * load_c<CT>(col + plane + t);
            n2 += w * load_c<CT>(col + 2 * plane + t);
        }
        if (inx) {
            const size_t t2 = (size_t)ty * W + tx;
            if (tap_agrees(__ldg(depth + t2), Dp)) {
                w = wx1 * wy1;
                den += w;
                n0 += w * load_c<CT>(col + t2);
                n1 += w * load_c<CT>(col + plane + t2);
                n2 += w * load_c<CT>(col + 2 * plane + t2);
            }
        }
    }
    out[0] = n0 / den;
    out[1] = n1 / den;
    out[2] = n2 / den;
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

// Build levels 1..5 from v0/m0.  Children are averaged in the order (0,0),(0,1),(1,0),(1,1) (row, column).
// Must be called by all threads of the block (contains barriers); v0/m0 must be complete on entry.
__device__ __forceinline__ void pull_tile(FillSmem &s) {
    const int t = threadIdx.x;
    const int nt = blockDim.x;
    for (int node = t; node < 256; node += nt) {
        const int i = node >> 4, j = node & 15;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        int cnt = 0;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int y = 2 * i + a, x = 2 * j + b;
                if (s.m0[y][x]) {
                    a0 += s.v0[0][y][x];
                    a1 += s.v0[1][y][x];
                    a2 += s.v0[2][y][x];
                    ++cnt;
                }
            }
        }
        const float fc = (float)cnt;
        s.lv[node] = cnt ? make_float4(a0 / fc, a1 / fc, a2 / fc, 1.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 1
    for (int l = 2; l <= 5; ++l) {
        const int side = kFillTile >> l, cside = side * 2;
        const int po = lv_offset(l), co = lv_offset(l - 1);
        for (int node = t; node < side * side; node += nt) {
            const int i = node / side, j = node % side;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
            int cnt = 0;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const float4 c = s.lv[co + (2 * i + a) * cside + (2 * j + b)];
                    if (c.w != 0.0f) {
                        a0 += c.x;
                        a1 += c.y;
                        a2 += c.z;
                        ++cnt;
                    }
                }
            }
            const float fc = (float)cnt;
            s.lv[po + node] = cnt ? make_float4(a0 / fc, a1 / fc, a2 / fc, 1.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
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
