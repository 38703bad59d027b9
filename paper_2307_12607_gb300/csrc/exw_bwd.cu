// exw_bwd.cu -- adjoint of stage (b) with respect to source colour and motion, and the fused training pass.
//
// A CTA owns a 32 x 32 SOURCE tile S and runs the fractions of its call one after another.  Per fraction, phase 1
// visits every source pixel p of S plus a one-pixel ring: if p won its target q = T(p) and q is not a hole, it
// stores the normalised weights w_t / sum w of its four taps and the upstream gradient g(q) in shared memory, and
// (for p inside S) adds dL/d mv(p) -- p wins at most one target per fraction, so each fraction adds one term and
// needs no atomics.  Phase 2 gives each source pixel s of S the contributions of the (at most 9) winners
// p = s - (dx, dy) that use s as a tap, in a fixed order, so dL/d colour(s) is summed by one thread
// deterministically.  The accumulators are read once, updated per fraction in fraction order and written once:
// a call over nfrac fractions equals nfrac one-fraction calls bit for bit.
//
// g(q) comes from grad_out (exw_warp_backward) or, in the fused training pass (exw_warp_l2_grad), from the
// forward value itself: q's colour is recomputed at its winner p with the arithmetic of stage (b) (same taps,
// weights and operation order, rounded to the storage type), g = 2 (out(q) - target(q)), and (out - target)^2 is
// added to the loss at q's winner, i.e. once per non-hole target.  The loss is summed in a fixed order: in FP32 by
// each thread over its few terms, then in FP64 across threads and CTAs (the FP64 pipe of this part issues about one
// operation per SM clock, so no FP64 arithmetic runs per pixel).
#include "exw_device.cuh"
#include "exw_internal.h"

namespace exw {

constexpr int kBwdThreads = 256;
constexpr int kStage = kFillTile + 4;  // S plus a two-pixel ring: the ring's winners and their taps
constexpr int kStageN = kStage * kStage;

// Shared memory of a CTA: the staged source depth (read once, used by every fraction for the taps' agreement; the
// motion and colour are read through L1), the per-fraction records of phase 1 and the motion accumulators of S.
template <typename CT>
struct BwdSmem {
    float4 recw[kRegionN];  // w_t / S for taps (p), (p+sx), (p+sy), (p+sx+sy)
    float4 recg[kRegionN];  // g(q) rgb, .w = flags: bit0 active, bits1-2 sx+1, bits3-4 sy+1
    float2 gms[kFillTile * kFillTile];
    float depth[kStageN];   // NaN outside the frame (never lands, never agrees)
    double red[kBwdThreads / 32];
    int last;
};

struct BwdArgs {
    const void *color;
    const float *depth;
    const float *mv;
    const unsigned long long *keys;  // [nfrac][H][W]: fraction k0 + kk's keys at keys + kk W H
    const float *grad_out;           // [3][H][W] (one fraction) unless fused
    const void *target[kMaxFrac];    // fused: [3][H][W] per fraction
    int W, H, nfrac, k0, L;
    float *grad_color;               // [3][H][W], accumulated
    float *grad_mv;                  // [2][H][W], accumulated
    double *partial;                 // fused: one loss partial per CTA
    unsigned int *arrived;           // fused: CTAs finished (the last one sums the partials)
    double *loss;                    // fused: the frame's loss
};

template <typename CT, bool FUSED>
__global__ void __launch_bounds__(kBwdThreads, 4) bwd_tile_kernel(const BwdArgs a) {
    extern __shared__ __align__(16) unsigned char bwd_smem_raw[];
    BwdSmem<CT> &sm = *reinterpret_cast<BwdSmem<CT> *>(bwd_smem_raw);
    float4 *recw = sm.recw, *recg = sm.recg;
    float2 *gms = sm.gms;
    double *red = sm.red;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int W = a.W, H = a.H;
    const int X0 = blockIdx.x * kFillTile, Y0 = blockIdx.y * kFillTile;
    const size_t plane = (size_t)W * H;
    const CT *col = (const CT *)a.color;
    // this thread's source pixels of phase 2 (rows wid + 8 j, column lane) and their colour accumulators
    const int sxg = X0 + lane;
    float gc[4][3];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int syg = Y0 + wid + 8 * j;
        const bool in = sxg < W && syg < H;
        const size_t s = (size_t)syg * W + sxg;
#pragma unroll
        for (int c = 0; c < 3; ++c) gc[j][c] = in ? a.grad_color[c * plane + s] : 0.0f;
    }
    // the motion accumulators of S, in shared memory for the whole call
    for (int c = tid; c < kFillTile * kFillTile; c += kBwdThreads) {
        const int x = X0 + (c & (kFillTile - 1)), y = Y0 + c / kFillTile;
        const size_t i = (size_t)y * W + x;
        gms[c] = (x < W && y < H) ? make_float2(a.grad_mv[i], a.grad_mv[plane + i]) : make_float2(0.f, 0.f);
    }
    // the source of S and its two-pixel ring, once for every fraction
    for (int c = tid; c < kStageN; c += kBwdThreads) {
        const int x = X0 - 2 + c % kStage, y = Y0 - 2 + c / kStage;
        const bool in = x >= 0 && x < W && y >= 0 && y < H;
        const size_t i = in ? (size_t)y * W + x : 0;
        sm.depth[c] = in ? __ldg(a.depth + i) : __int_as_float(0x7FC00000);
    }
    __syncthreads();  // phase 1 reads the stage and updates cells another thread loaded
    float lacc = 0.0f;  // this thread's loss terms (at most 5 cells x 3 fractions x 3 channels), then FP64
    for (int kk = 0; kk < a.nfrac; ++kk) {
        const int k = a.k0 + kk, L = a.L;
        const float scale = -(float)k * pow2_neg(L);
        const unsigned long long *keys = a.keys + (size_t)kk * plane;
        const CT *tgt = FUSED ? (const CT *)(kk == 0 ? a.target[0] : kk == 1 ? a.target[1] : a.target[2]) : nullptr;
#pragma unroll 1
        for (int r = tid; r < kRegionN; r += kBwdThreads) {  // a cell belongs to the same thread in every fraction
            const int ry = r / kRegion, rx = r - ry * kRegion;
            const int px = X0 - 1 + rx, py = Y0 - 1 + ry;
            const bool inside = rx >= 1 && rx <= kFillTile && ry >= 1 && ry <= kFillTile;
            float4 wv = make_float4(0.f, 0.f, 0.f, 0.f);
            float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
            const int e = (ry + 1) * kStage + (rx + 1);  // p in the stage
            if (px >= 0 && px < W && py >= 0 && py < H) {
                const size_t i = (size_t)py * W + px;
                const uint32_t db = __float_as_uint(sm.depth[e]);
                const uint32_t ux = __float_as_uint(__ldg(a.mv + i)), uy = __float_as_uint(__ldg(a.mv + plane + i));
                if (depth_ok(db) && finite_bits(ux) && finite_bits(uy)) {
                    const AxisDec dx = axis_dec(ux, L), dy = axis_dec(uy, L);
                    const bool lands = dx.land && dy.land;
                    const int ox = axis_off(dx, k), oy = axis_off(dy, k);
                    const int qx = px + ox, qy = py + oy;
                    if (lands && qx >= 0 && qx < W && qy >= 0 && qy < H) {
                        const size_t q = (size_t)qy * W + qx;
                        // every global load of the cell at once: the keys of q and its 4-neighbours, g's inputs
                        const unsigned long long kq = __ldg(keys + q);
                        const unsigned long long k0 = qx > 0 ? __ldg(keys + q - 1) : kKeyEmpty;
                        const unsigned long long k1 = qx < W - 1 ? __ldg(keys + q + 1) : kKeyEmpty;
                        const unsigned long long k2 = qy > 0 ? __ldg(keys + q - W) : kKeyEmpty;
                        const unsigned long long k3 = qy < H - 1 ? __ldg(keys + q + W) : kKeyEmpty;
                        float gin[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            gin[c] = FUSED ? load_c<CT>(tgt + c * plane + q) : __ldg(a.grad_out + c * plane + q);
                        if (kq == pack_key_global(db, (uint32_t)i)) {
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
                                const int e10 = e + sx, e01 = e + sy * kStage, e11 = e01 + sx;  // taps in the stage
                                const bool a10 = inx && tap_agrees(sm.depth[e10], Dp);
                                const bool a01 = iny && tap_agrees(sm.depth[e01], Dp);
                                const bool a11 = inx && iny && tap_agrees(sm.depth[e11], Dp);
                                const float w00 = __fmul_rn(wx0, wy0), w10 = a10 ? __fmul_rn(wx1, wy0) : 0.f;
                                const float w01 = a01 ? __fmul_rn(wx0, wy1) : 0.f;
                                const float w11 = a11 ? __fmul_rn(wx1, wy1) : 0.f;
                                const float S = weight_sum(w00, w10, w01, w11);
                                const float inv = __fdiv_rn(1.0f, S);
                                wv = make_float4(__fmul_rn(w00, inv), __fmul_rn(w10, inv), __fmul_rn(w01, inv),
                                                 __fmul_rn(w11, inv));
                                float C[3][4];  // tap colours (0 for taps that do not take part)
                                if (FUSED || inside) {
                                    const size_t t10 = i + sx, t01 = sy > 0 ? i + W : i - W, t11 = t01 + sx;
#pragma unroll
                                    for (int c = 0; c < 3; ++c) {
                                        const CT *cp = col + c * plane;
                                        C[c][0] = load_c<CT>(cp + i);
                                        C[c][1] = a10 ? load_c<CT>(cp + t10) : 0.f;
                                        C[c][2] = a01 ? load_c<CT>(cp + t01) : 0.f;
                                        C[c][3] = a11 ? load_c<CT>(cp + t11) : 0.f;
                                    }
                                }
                                float g[3];
                                if (FUSED) {
                                    // q's colour as stage (b) computes it, then the loss and its gradient
                                    const float rcp = __frcp_rn(S);
#pragma unroll
                                    for (int c = 0; c < 3; ++c) {
                                        float n = __fmul_rn(w00, C[c][0]);
                                        n = a10 ? fmaf(w10, C[c][1], n) : n;
                                        n = a01 ? fmaf(w01, C[c][2], n) : n;
                                        n = a11 ? fmaf(w11, C[c][3], n) : n;
                                        const float d = __fsub_rn(storage_round<CT>(__fmul_rn(n, rcp)), gin[c]);
                                        g[c] = __fmul_rn(2.0f, d);
                                        if (inside) lacc = fmaf(d, d, lacc);
                                    }
                                } else {
#pragma unroll
                                    for (int c = 0; c < 3; ++c) g[c] = gin[c];
                                }
                                const uint32_t flags = 1u | ((uint32_t)(sx + 1) << 1) | ((uint32_t)(sy + 1) << 3);
                                gv = make_float4(g[0], g[1], g[2], __uint_as_float(flags));
                                if (inside) {
                                    // dL/d mv(p) = -(k/denom) sum_c g_c sum_t (dw_t/drho)(C_c(t) - out_c) / S
                                    // d w_t / d rho: +-(the other axis' weight), signs from the tap side
                                    const float fsx = (float)sx, fsy = (float)sy;
                                    const float dx00 = -fsx * wy0, dx10 = a10 ? fsx * wy0 : 0.f;
                                    const float dx01 = a01 ? -fsx * wy1 : 0.f, dx11 = a11 ? fsx * wy1 : 0.f;
                                    const float dy00 = -fsy * wx0, dy10 = a10 ? -fsy * wx1 : 0.f;
                                    const float dy01 = a01 ? fsy * wx0 : 0.f, dy11 = a11 ? fsy * wx1 : 0.f;
                                    float gx = 0.f, gy = 0.f;
#pragma unroll
                                    for (int c = 0; c < 3; ++c) {
                                        const float C00 = C[c][0], C10 = C[c][1], C01 = C[c][2], C11 = C[c][3];
                                        float t = __fmul_rn(w00, C00);
                                        t = fmaf(w10, C10, t);
                                        t = fmaf(w01, C01, t);
                                        t = fmaf(w11, C11, t);
                                        const float o = __fmul_rn(t, inv);
                                        float ddx = __fmul_rn(dx00, __fsub_rn(C00, o));
                                        ddx = fmaf(dx10, __fsub_rn(C10, o), ddx);
                                        ddx = fmaf(dx01, __fsub_rn(C01, o), ddx);
                                        ddx = fmaf(dx11, __fsub_rn(C11, o), ddx);
                                        float ddy = __fmul_rn(dy00, __fsub_rn(C00, o));
                                        ddy = fmaf(dy10, __fsub_rn(C10, o), ddy);
                                        ddy = fmaf(dy01, __fsub_rn(C01, o), ddy);
                                        ddy = fmaf(dy11, __fsub_rn(C11, o), ddy);
                                        gx = fmaf(g[c], ddx, gx);
                                        gy = fmaf(g[c], ddy, gy);
                                    }
                                    float2 &gm = gms[(ry - 1) * kFillTile + (rx - 1)];
                                    gm.x = fmaf(__fmul_rn(scale, gx), inv, gm.x);
                                    gm.y = fmaf(__fmul_rn(scale, gy), inv, gm.y);
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
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int y = wid + 8 * j;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
            for (int ddy = -1; ddy <= 1; ++ddy) {
#pragma unroll
                for (int ddx = -1; ddx <= 1; ++ddx) {
                    const int r = (y + 1 - ddy) * kRegion + (lane + 1 - ddx);
                    const float4 gv = recg[r];
                    const uint32_t flags = __float_as_uint(gv.w);
                    if (!(flags & 1u)) continue;
                    const int psx = (int)((flags >> 1) & 3u) - 1, psy = (int)((flags >> 3) & 3u) - 1;
                    const int xp = ddx == 0 ? 0 : (ddx == psx ? 1 : -1);
                    const int yp = ddy == 0 ? 0 : (ddy == psy ? 1 : -1);
                    if (xp < 0 || yp < 0) continue;
                    const float4 wv = recw[r];
                    const int t = xp + 2 * yp;
                    const float w = t == 0 ? wv.x : t == 1 ? wv.y : t == 2 ? wv.z : wv.w;
                    a0 = fmaf(gv.x, w, a0);
                    a1 = fmaf(gv.y, w, a1);
                    a2 = fmaf(gv.z, w, a2);
                }
            }
            gc[j][0] = __fadd_rn(gc[j][0], a0);
            gc[j][1] = __fadd_rn(gc[j][1], a1);
            gc[j][2] = __fadd_rn(gc[j][2], a2);
        }
        __syncthreads();  // recw / recg are rewritten by the next fraction
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int syg = Y0 + wid + 8 * j;
        if (sxg >= W || syg >= H) continue;
        const size_t s = (size_t)syg * W + sxg;
#pragma unroll
        for (int c = 0; c < 3; ++c) a.grad_color[c * plane + s] = gc[j][c];
    }
    for (int c = tid; c < kFillTile * kFillTile; c += kBwdThreads) {  // (the last barrier ordered every update)
        const int x = X0 + (c & (kFillTile - 1)), y = Y0 + c / kFillTile;
        if (x >= W || y >= H) continue;
        const size_t i = (size_t)y * W + x;
        const float2 gm = gms[c];
        a.grad_mv[i] = gm.x;
        a.grad_mv[plane + i] = gm.y;
    }
    if constexpr (FUSED) {
        // the loss: per CTA a fixed tree over its threads, then the CTAs in a fixed order by the last one to finish
        double lsum = (double)lacc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xFFFFFFFFu, lsum, o);
        if (lane == 0) red[wid] = lsum;
        __syncthreads();
        const unsigned int nblocks = gridDim.x * gridDim.y, bid = blockIdx.y * gridDim.x + blockIdx.x;
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < kBwdThreads / 32; ++w) t += red[w];
            a.partial[bid] = t;
            __threadfence();
            sm.last = atomicAdd(a.arrived, 1u) == nblocks - 1u ? 1 : 0;
        }
        __syncthreads();
        if (!sm.last) return;
        __threadfence();
        double t = 0.0;
        for (unsigned int b = tid; b < nblocks; b += kBwdThreads) t += __ldcg(a.partial + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
        __syncthreads();
        if (lane == 0) red[wid] = t;
        __syncthreads();
        if (tid == 0) {
            double v = 0.0;
            for (int w = 0; w < kBwdThreads / 32; ++w) v += red[w];
            *a.loss = v;
            *a.arrived = 0u;
        }
    }
}

// Stage (a) for fractions k0 .. k0 + nfrac - 1 in one pass: each source pixel is read once and takes the 64-bit
// atomic minimum at its target in each fraction's key plane (keys + kk W H, cleared beforehand).
__global__ void __launch_bounds__(256) splat_multi_kernel(const float *__restrict__ depth,
                                                          const float *__restrict__ mv, int W, int H, int k0,
                                                          int nfrac, int L, unsigned long long *keys) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const size_t plane = (size_t)W * H;
    const size_t i = (size_t)y * W + x;
    const uint32_t db = __float_as_uint(__ldg(depth + i));
    const uint32_t ux = __float_as_uint(__ldg(mv + i)), uy = __float_as_uint(__ldg(mv + plane + i));
    if (!depth_ok(db) || !finite_bits(ux) || !finite_bits(uy)) return;
    const AxisDec dx = axis_dec(ux, L), dy = axis_dec(uy, L);
    if (!dx.land || !dy.land) return;
    const unsigned long long key = pack_key_global(db, (uint32_t)i);
    for (int kk = 0; kk < nfrac; ++kk) {
        const int k = k0 + kk;
        const int gx = x + axis_off(dx, k), gy = y + axis_off(dy, k);
        if (gx < 0 || gx >= W || gy < 0 || gy >= H) continue;
        atomicMin(keys + kk * plane + (size_t)gy * W + gx, key);
    }
}

template <typename CT, bool FUSED>
static cudaError_t launch_bwd_tiles(const BwdArgs &a, cudaStream_t s) {
    constexpr size_t kSmem = sizeof(BwdSmem<CT>);
    // set on every launch: the attribute belongs to the current device's context
    const cudaError_t e =
        cudaFuncSetAttribute(bwd_tile_kernel<CT, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    const dim3 g((unsigned)ceil_div(a.W, kFillTile), (unsigned)ceil_div(a.H, kFillTile), 1);
    bwd_tile_kernel<CT, FUSED><<<g, kBwdThreads, kSmem, s>>>(a);
    return cudaSuccess;
}

cudaError_t launch_backward(const float *grad_out, const void *color, exw_dtype cdt, const float *depth,
                            const float *mv, const uint64_t *keys, int W, int H, int k, int L, float *grad_color,
                            float *grad_mv, cudaStream_t s) {
    BwdArgs a{};
    a.color = color;
    a.depth = depth;
    a.mv = mv;
    a.keys = (const unsigned long long *)keys;
    a.grad_out = grad_out;
    a.W = W;
    a.H = H;
    a.nfrac = 1;
    a.k0 = k;
    a.L = L;
    a.grad_color = grad_color;
    a.grad_mv = grad_mv;
    timing_begin("exw_backward", s);
    const cudaError_t e = cdt == EXW_F32 ? launch_bwd_tiles<float, false>(a, s) : launch_bwd_tiles<__half, false>(a, s);
    count_launch();
    timing_end("exw_backward", s);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Workspace of exw_warp_l2_grad: the key planes of the fractions, the CTAs' loss partials and the arrival counter.
struct TrainLayout {
    size_t keys, partial, arrived, total;
};
static TrainLayout train_layout(int W, int H, int nfrac) {
    TrainLayout t{};
    size_t off = 0;
    t.keys = off;
    off += align_up((size_t)nfrac * W * H * 8);
    t.partial = off;
    off += align_up((size_t)ceil_div(W, kFillTile) * ceil_div(H, kFillTile) * 8);
    t.arrived = off;
    off += kAlign;
    t.total = off;
    return t;
}

size_t train_workspace_bytes(int W, int H, int nfrac) { return train_layout(W, H, nfrac).total; }

// One frame of exw_warp_l2_grad: keys of every fraction (one clear, one splat pass), then the fused pass.
cudaError_t launch_train_frame(const exw_train_frame &f, int nfrac, double *loss, void *ws, cudaStream_t s) {
    const int W = f.src.W, H = f.src.H;
    const TrainLayout t = train_layout(W, H, nfrac);
    char *b = (char *)ws;
    unsigned long long *keys = (unsigned long long *)(b + t.keys);
    cudaError_t e = launch_clear_keys((uint64_t *)keys, (size_t)nfrac * W * H, s);
    if (e == cudaSuccess) e = launch_zero(b + t.arrived, 4, s);
    if (e != cudaSuccess) return e;
    timing_begin("exw_splat_multi", s);
    splat_multi_kernel<<<dim3((unsigned)ceil_div(W, 256), (unsigned)H), 256, 0, s>>>(f.src.depth, f.src.mv, W, H, 1,
                                                                                    nfrac, 2, keys);
    count_launch();
    timing_end("exw_splat_multi", s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    BwdArgs a{};
    a.color = f.src.color;
    a.depth = f.src.depth;
    a.mv = f.src.mv;
    a.keys = keys;
    for (int j = 0; j < nfrac; ++j) a.target[j] = f.target[j];
    a.W = W;
    a.H = H;
    a.nfrac = nfrac;
    a.k0 = 1;
    a.L = 2;
    a.grad_color = f.grad_color;
    a.grad_mv = f.grad_mv;
    a.partial = (double *)(b + t.partial);
    a.arrived = (unsigned int *)(b + t.arrived);
    a.loss = loss;
    timing_begin("exw_train", s);
    e = f.src.cdt == EXW_F32 ? launch_bwd_tiles<float, true>(a, s) : launch_bwd_tiles<__half, true>(a, s);
    count_launch();
    timing_end("exw_train", s);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace exw
