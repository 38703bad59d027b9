// exw_bwd.cu -- adjoint of stage (b) with respect to source colour and motion.
//
// A CTA owns a 32 x 32 SOURCE tile S.  Phase 1 visits every source pixel p of S plus a one-pixel ring: if p won
// its target q = T(p) and q is not a hole, it stores the normalised weights w_t / sum w of its four taps and the
// upstream gradient g(q) in shared memory, and (for p inside S) writes dL/d mv(p) -- p wins at most one target,
// so that sum has one term and needs no atomics.  Phase 2 gives each source pixel s of S the contributions of
// the (at most 9) winners p = s - (dx, dy) that use s as a tap, in a fixed order, so dL/d colour(s) is summed by
// one thread deterministically.
#include "exw_device.cuh"
#include "exw_internal.h"

namespace exw {

constexpr int kBwdThreads = 256;
constexpr int kBwdRegionN = kRegionN;

template <typename CT>
__global__ void __launch_bounds__(kBwdThreads) backward_kernel(const float *__restrict__ grad_out,
                                                               const CT *__restrict__ col,
                                                               const float *__restrict__ depth,
                                                               const float *__restrict__ mv,
                                                               const unsigned long long *__restrict__ keys, int W, int H,
                                                               int k, int L, float *grad_color, float *grad_mv) {
    __shared__ float4 recw[kBwdRegionN];  // w_t / S for taps (p), (p+sx), (p+sy), (p+sx+sy)
    __shared__ float4 recg[kBwdRegionN];  // g(q) rgb, .w = flags: bit0 active, bits1-2 sx+1, bits3-4 sy+1
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int X0 = blockIdx.x * kFillTile, Y0 = blockIdx.y * kFillTile;
    const size_t plane = (size_t)W * H;
    const float scale = -(float)k * pow2_neg(L);
    for (int r = tid; r < kBwdRegionN; r += kBwdThreads) {
        const int ry = r / kRegion, rx = r - ry * kRegion;
        const int px = X0 - 1 + rx, py = Y0 - 1 + ry;
        float4 wv = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (px >= 0 && px < W && py >= 0 && py < H) {
            const size_t i = (size_t)py * W + px;
            const uint32_t db = __float_as_uint(__ldg(depth + i));
            const uint32_t ux = __float_as_uint(__ldg(mv + i)), uy = __float_as_uint(__ldg(mv + plane + i));
            if (depth_ok(db) && finite_bits(ux) && finite_bits(uy)) {
                const AxisDec dx = axis_dec(ux, L), dy = axis_dec(uy, L);
                const bool lands = dx.land && dy.land;
                const int ox = axis_off(dx, k), oy = axis_off(dy, k);
                const int qx = px + ox, qy = py + oy;
                if (lands && qx >= 0 && qx < W && qy >= 0 && qy < H) {
                    const size_t q = (size_t)qy * W + qx;
                    const unsigned long long kq = __ldg(keys + q);
                    if (kq == pack_key_global(db, (uint32_t)i)) {
                        const unsigned long long k0 = qx > 0 ? __ldg(keys + q - 1) : kKeyEmpty;
                        const unsigned long long k1 = qx < W - 1 ? __ldg(keys + q + 1) : kKeyEmpty;
                        const unsigned long long k2 = qy > 0 ? __ldg(keys + q - W) : kKeyEmpty;
                        const unsigned long long k3 = qy < H - 1 ? __ldg(keys + q + W) : kKeyEmpty;
                        if (!is_crack(key_dbits(kq), key_dbits(k0), key_dbits(k1), key_dbits(k2), key_dbits(k3))) {
                            const float Dp = __uint_as_float(db);
                            int sx, sy;
                            const float rhox = residual(__uint_as_float(ux), k, L, ox, sx);
                            const float rhoy = residual(__uint_as_float(uy), k, L, oy, sy);
                            const float wx1 = fabsf(rhox), wy1 = fabsf(rhoy);
                            const float wx0 = 1.f - wx1, wy0 = 1.f - wy1;
                            const int tx = px + sx, ty = py + sy;
                            const bool inx = sx != 0 && tx >= 0 && tx < W;
                            const bool iny = sy != 0 && ty >= 0 && ty < H;
                            const size_t t10 = (size_t)py * W + tx, t01 = (size_t)ty * W + px;
                            const size_t t11 = (size_t)ty * W + tx;
                            const bool a10 = inx && tap_agrees(__ldg(depth + t10), Dp);
                            const bool a01 = iny && tap_agrees(__ldg(depth + t01), Dp);
                            const bool a11 = inx && iny && tap_agrees(__ldg(depth + t11), Dp);
                            const float w00 = wx0 * wy0, w10 = a10 ? wx1 * wy0 : 0.f;
                            const float w01 = a01 ? wx0 * wy1 : 0.f, w11 = a11 ? wx1 * wy1 : 0.f;
                            const float S = ((w00 + w10) + w01) + w11;
                            const float inv = 1.0f / S;
                            wv = make_float4(w00 * inv, w10 * inv, w01 * inv, w11 * inv);
                            const float g0 = __ldg(grad_out + q), g1 = __ldg(grad_out + plane + q);
                            const float g2 = __ldg(grad_out + 2 * plane + q);
                            const uint32_t flags = 1u | ((uint32_t)(sx + 1) << 1) | ((uint32_t)(sy + 1) << 3);
                            gv = make_float4(g0, g1, g2, __uint_as_float(flags));
                            if (rx >= 1 && rx <= kFillTile && ry >= 1 && ry <= kFillTile) {
                                // dL/d mv(p) = -(k/denom) sum_c g_c sum_t (dw_t/drho)(C_c(t) - out_c) / S
                                const float dx00 = -sx * wy0, dx10 = a10 ? sx * wy0 : 0.f;
                                const float dx01 = a01 ? -sx * wy1 : 0.f, dx11 = a11 ? sx * wy1 : 0.f;
                                const float dy00 = -sy * wx0, dy10 = a10 ? -sy * wx1 : 0.f;
                                const float dy01 = a01 ? sy * wx0 : 0.f, dy11 = a11 ? sy * wx1 : 0.f;
                                const float g[3] = {g0, g1, g2};
                                float gx = 0.f, gy = 0.f;
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    const CT *cp = col + c * plane;
                                    const float C00 = load_c<CT>(cp + i);
                                    const float C10 = a10 ? load_c<CT>(cp + t10) : 0.f;
                                    const float C01 = a01 ? load_c<CT>(cp + t01) : 0.f;
                                    const float C11 = a11 ? load_c<CT>(cp + t11) : 0.f;
                                    const float o = (((w00 * C00 + w10 * C10) + w01 * C01) + w11 * C11) * inv;
                                    const float ddx = dx00 * (C00 - o) + dx10 * (C10 - o) + dx01 * (C01 - o) +
                                                      dx11 * (C11 - o);
                                    const float ddy = dy00 * (C00 - o) + dy10 * (C10 - o) + dy01 * (C01 - o) +
                                                      dy11 * (C11 - o);
                                    gx += g[c] * ddx;
                                    gy += g[c] * ddy;
                                }
                                grad_mv[i] += scale * gx * inv;
                                grad_mv[plane + i] += scale * gy * inv;
                            }
                        }
                    }
                }
            }
        }
        recw[r] = wv;
        recg[r] = gv;
    }
    __syncthreads();
    const int sxg = X0 + lane;
    if (sxg >= W) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int y = wid + 8 * j, syg = Y0 + y;
        if (syg >= H) continue;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int r = (y + 1 - dy) * kRegion + (lane + 1 - dx);
                const float4 gv = recg[r];
                const uint32_t flags = __float_as_uint(gv.w);
                if (!(flags & 1u)) continue;
                const int psx = (int)((flags >> 1) & 3u) - 1, psy = (int)((flags >> 3) & 3u) - 1;
                const int xp = dx == 0 ? 0 : (dx == psx ? 1 : -1);
                const int yp = dy == 0 ? 0 : (dy == psy ? 1 : -1);
                if (xp < 0 || yp < 0) continue;
                const float4 wv = recw[r];
                const int t = xp + 2 * yp;
                const float w = t == 0 ? wv.x : t == 1 ? wv.y : t == 2 ? wv.z : wv.w;
                a0 += gv.x * w;
                a1 += gv.y * w;
                a2 += gv.z * w;
            }
        }
        const size_t s = (size_t)syg * W + sxg;
        grad_color[s] += a0;
        grad_color[plane + s] += a1;
        grad_color[2 * plane + s] += a2;
    }
}

cudaError_t launch_backward(const float *grad_out, const void *color, exw_dtype cdt, const float *depth,
                            const float *mv, const uint64_t *keys, int W, int H, int k, int L, float *grad_color,
                            float *grad_mv, cudaStream_t s) {
    const dim3 g((unsigned)ceil_div(W, kFillTile), (unsigned)ceil_div(H, kFillTile), 1);
    timing_begin("exw_backward", s);
    if (cdt == EXW_F32)
        backward_kernel<float><<<g, kBwdThreads, 0, s>>>(grad_out, (const float *)color, depth, mv,
                                                         (const unsigned long long *)keys, W, H, k, L, grad_color,
                                                         grad_mv);
    else
        backward_kernel<__half><<<g, kBwdThreads, 0, s>>>(grad_out, (const __half *)color, depth, mv,
                                                          (const unsigned long long *)keys, W, H, k, L, grad_color,
                                                          grad_mv);
    count_launch();
    timing_end("exw_backward", s);
    return cudaGetLastError();
}

}  // namespace exw
