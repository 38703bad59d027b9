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

// Grids launched by launch_dependent: wait until the grids before this one on the stream have completed and their
// writes are visible (at once for a grid launched without programmatic serialisation), and let the next grid be
// scheduled (it waits in turn before touching memory).
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

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
// k <= 64, |k*sM| < 2^30, and rounding half up is an arithmetic shift: off = (k*sM + 2^(n-1)) >> n.  For n >= 32
// (|d| < 1/4) the same expression with n clamped to 31 gives 0, since |k*sM| < 2^30; n <= 0 means |d| >= 2^23,
// which cannot land in any frame.  The decomposition is shared by all fractions, so each fraction costs one
// multiply-add and one shift, without branches.
// ------------------------------------------------------------------------------------------------------------
struct AxisDec {
    int sM;     // signed significand
    int n;      // right-shift amount, clamped to [1, 31]
    int half;   // 2^(n-1)
    bool land;  // false when the motion is too large to land in any frame
};

__device__ __forceinline__ AxisDec axis_dec(uint32_t u, int L) {
    const uint32_t E = (u >> 23) & 0xFFu;
    const int M = (int)((u & 0x7FFFFFu) | (E ? 0x800000u : 0u));
    const int n = 150 + L - (E ? (int)E : 1);
    AxisDec d;
    d.sM = (u >> 31) ? -M : M;
    d.land = n > 0;
    d.n = min(max(n, 1), 31);
    d.half = 1 << (d.n - 1);
    return d;
}

__device__ __forceinline__ int axis_off(const AxisDec &d, int k) { return (k * d.sM + d.half) >> d.n; }

__device__ __forceinline__ int axis_off_of(uint32_t bits, int k, int L) {  // for clamped bounds (always lands)
    return axis_off(axis_dec(bits, L), k);
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
    __device__ __forceinline__ size_t stride() const { return (size_t)W; }
    __device__ __forceinline__ int safe_x() const { return 0; }  // a pixel every access may use
    __device__ __forceinline__ int safe_y() const { return 0; }
    __device__ __forceinline__ float d(size_t i) const { return __ldg(depth + i); }
    __device__ __forceinline__ float mx(size_t i) const { return __ldg(mv + i); }
    __device__ __forceinline__ float my(size_t i) const { return __ldg(mv + plane + i); }
    __device__ __forceinline__ float c(int ch, size_t i) const { return load_c<CT>(col + ch * plane + i); }
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
    __device__ __forceinline__ int stride() const { return WX; }
    __device__ __forceinline__ int safe_x() const { return x0 + 1; }  // its taps stay inside the window
    __device__ __forceinline__ int safe_y() const { return y0 + 1; }
    __device__ __forceinline__ float d(int i) const { return w->depth[i]; }
    __device__ __forceinline__ float mx(int i) const { return w->mv[0][i]; }
    __device__ __forceinline__ float my(int i) const { return w->mv[1][i]; }
    __device__ __forceinline__ float c(int ch, int i) const { return to_f<CT>(w->col[ch][i]); }
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

// The products and sums of the gather are written with explicit round-to-nearest intrinsics (never fused into an
// FMA by the compiler), so every path that computes a gather -- the per-tile passes, the engine's window, uniform
// and smooth tiles, the recomputation in the fused training pass -- gets the same bits in any context.
// Sum of the bilinear weights of the participating taps (0 for the others), in the order 00, 10, 01, 11.
__device__ __forceinline__ float weight_sum(float w00, float w10, float w01, float w11) {
    return __fadd_rn(__fadd_rn(__fadd_rn(w00, w10), w01), w11);
}

// ------------------------------------------------------------------------------------------------------------
// Pull-push inside one 32 x 32 fill tile.  Tiles are aligned to 32, so every ancestor up to level 5 of a tile pixel
// is computed from that tile alone; out-of-frame pixels are invalid, which reproduces the ceil-halving level sizes.
// Warp w of 16 owns tile rows 2w and 2w+1 (lane = column).
// ------------------------------------------------------------------------------------------------------------

// Mean of the valid children, taken in the order (0,0),(0,1),(1,0),(1,1) (row, column); .w = validity.
__device__ __forceinline__ float4 mean4(float4 c0, float4 c1, float4 c2, float4 c3) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    int cnt = 0;
    if (c0.w != 0.0f) { a0 += c0.x; a1 += c0.y; a2 += c0.z; ++cnt; }
    if (c1.w != 0.0f) { a0 += c1.x; a1 += c1.y; a2 += c1.z; ++cnt; }
    if (c2.w != 0.0f) { a0 += c2.x; a1 += c2.y; a2 += c2.z; ++cnt; }
    if (c3.w != 0.0f) { a0 += c3.x; a1 += c3.y; a2 += c3.z; ++cnt; }
    if (cnt == 0) return make_float4(0.f, 0.f, 0.f, 0.f);
    const float inv = cnt == 1 ? 1.0f : cnt == 2 ? 0.5f : cnt == 3 ? (1.0f / 3.0f) : 0.25f;
    return make_float4(__fmul_rn(a0, inv), __fmul_rn(a1, inv), __fmul_rn(a2, inv), 1.0f);
}

__device__ __forceinline__ float4 shfl4_xor(float4 v, int m) {
    return make_float4(__shfl_xor_sync(0xFFFFFFFFu, v.x, m), __shfl_xor_sync(0xFFFFFFFFu, v.y, m),
                       __shfl_xor_sync(0xFFFFFFFFu, v.z, m), __shfl_xor_sync(0xFFFFFFFFu, v.w, m));
}

__device__ __forceinline__ float4 shfl4_idx(float4 v, int src) {
    return make_float4(__shfl_sync(0xFFFFFFFFu, v.x, src), __shfl_sync(0xFFFFFFFFu, v.y, src),
                       __shfl_sync(0xFFFFFFFFu, v.z, src), __shfl_sync(0xFFFFFFFFu, v.w, src));
}

// Pyramid levels 1..5 of one 32 x 32 tile in shared memory: 16x16, 8x8, 4x4, 2x2, 1x1 nodes.
struct TilePyr {
    float4 l1[256];
    float4 l2[64];
    float4 l3[16];
    float4 l4[4];
    float4 l5;
};

// Build the pyramid from this thread's two pixels (tile rows 2w and 2w+1 of column lane; .w = validity) with
// 16 warps per CTA.  Level 1 is formed in registers (warp shuffle with the neighbouring column), levels 2..5 by
// warp 0.  Contains two block barriers, which every thread must reach.  Returns this thread's level-1 node.
__device__ __forceinline__ float4 build_pyramid(TilePyr &t, float4 top, float4 bot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float4 ptop = shfl4_xor(top, 1), pbot = shfl4_xor(bot, 1);
    const float4 n1 = (lane & 1) ? mean4(ptop, top, pbot, bot) : mean4(top, ptop, bot, pbot);
    if ((lane & 1) == 0) t.l1[wid * 16 + (lane >> 1)] = n1;
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int node = lane + 32 * h, i = node >> 3, j = node & 7;
            const float4 *c = t.l1 + (2 * i) * 16 + 2 * j;
            t.l2[node] = mean4(c[0], c[1], c[16], c[17]);
        }
        __syncwarp();
        if (lane < 16) {
            const int i = lane >> 2, j = lane & 3;
            const float4 *c = t.l2 + (2 * i) * 8 + 2 * j;
            t.l3[lane] = mean4(c[0], c[1], c[8], c[9]);
        }
        __syncwarp();
        if (lane < 4) {
            const int i = lane >> 1, j = lane & 1;
            const float4 *c = t.l3 + (2 * i) * 4 + 2 * j;
            t.l4[lane] = mean4(c[0], c[1], c[4], c[5]);
        }
        __syncwarp();
        if (lane == 0) t.l5 = mean4(t.l4[0], t.l4[1], t.l4[2], t.l4[3]);
    }
    __syncthreads();
    return n1;
}

// Value pushed down to a pixel of this thread (tile row 2w or 2w+1, column lane): its first valid ancestor; .w = 0
// when the whole tile is invalid.  n1 is the thread's level-1 node.
__device__ __forceinline__ float4 push_value(const TilePyr &t, float4 n1) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (n1.w != 0.0f) return n1;
    const float4 v2 = t.l2[(wid >> 1) * 8 + (lane >> 2)];
    if (v2.w != 0.0f) return v2;
    const float4 v3 = t.l3[(wid >> 2) * 4 + (lane >> 3)];
    if (v3.w != 0.0f) return v3;
    const float4 v4 = t.l4[(wid >> 3) * 2 + (lane >> 4)];
    if (v4.w != 0.0f) return v4;
    return t.l5;
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
