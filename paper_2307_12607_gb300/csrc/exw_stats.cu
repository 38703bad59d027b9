// exw_stats.cu -- frame statistics of the decision stage: the motion-variance features Var_x(F_mv), Var_y(F_mv) of
// the environment vector (Sec. IV-C, Eq. 1) and the colour MSE behind the reward's PSNR (Sec. IV-C, Eq. 3).
//
// Both are FP64 reductions over a fixed grid (kStatBlocks x kStatThreads, independent of the GPU), so the order of
// every addition is fixed and the result is deterministic.  Each thread reads a grid-strided subsequence
// (coalesced) and keeps plain FP64 sums -- for the variance, of the count and of x - K, y - K and their squares,
// with one shift K for the whole frame (a value of the field, so the final subtraction loses little) -- which
// are added in trees across the warp, the block and, in the last block to finish, the blocks.
#include "exw_device.cuh"
#include "exw_internal.h"

namespace exw {
namespace {

constexpr int kStatBlocks = 256, kStatThreads = 256;

struct Moments {  // a block's partial: count, shifted sums of x and y, shifted sums of squares
    double n, mx, my, vx, vy;
};

// Workspace: the blocks' partial results, then the arrival counter of the last-block pattern.
struct StatWs {
    Moments part[kStatBlocks];
    unsigned int arrived;
};

// The last block to finish (by an atomic ticket after a fence) sees every partial.
__device__ __forceinline__ bool last_block(unsigned int *arrived) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(arrived, 1u) == gridDim.x - 1;
    __syncthreads();
    return last;
}

// Shift of the variance's sums: the first finite vector among the first kShiftScan pixels (0 when there is none);
// every block finds the same one.  Any value of the field keeps the shifted sums' cancellation small.
constexpr int kShiftScan = 1024;

__global__ void __launch_bounds__(kStatThreads) mv_variance_kernel(const float *__restrict__ mv, size_t n,
                                                                   StatWs *ws, double *out) {
    __shared__ double shift[2];
    __shared__ double red[5][kStatThreads / 32];
    if (threadIdx.x < 32) {
        int first = kShiftScan;
        for (int i0 = 0; i0 < kShiftScan && (size_t)i0 < n && first == kShiftScan; i0 += 32) {
            const int i = i0 + (int)threadIdx.x;
            const bool ok = (size_t)i < n && isfinite(__ldg(mv + i)) && isfinite(__ldg(mv + n + i));
            const unsigned int b = __ballot_sync(0xFFFFFFFFu, ok);
            if (b) first = i0 + __ffs(b) - 1;
        }
        if (threadIdx.x == 0) {
            shift[0] = first < kShiftScan ? (double)mv[first] : 0.0;
            shift[1] = first < kShiftScan ? (double)mv[n + first] : 0.0;
        }
    }
    __syncthreads();
    const double kx = shift[0], ky = shift[1];
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // count, sums of (x - kx), (y - ky) and of their squares
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = __ldg(mv + i), y = __ldg(mv + n + i);
        if (!isfinite(x) || !isfinite(y)) continue;
        const double dx = (double)x - kx, dy = (double)y - ky;
        v[0] += 1.0;
        v[1] += dx;
        v[2] += dy;
        v[3] = fma(dx, dx, v[3]);
        v[4] = fma(dy, dy, v[4]);
    }
    // plain sums from here on: warp tree, block, then the blocks in a tree in the last block
#pragma unroll
    for (int c = 0; c < 5; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xFFFFFFFFu, v[c], o);
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = v[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Moments &pb = ws->part[blockIdx.x];
        double t[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            t[c] = red[c][0];
            for (int w = 1; w < kStatThreads / 32; ++w) t[c] += red[c][w];
        }
        pb = Moments{t[0], t[1], t[2], t[3], t[4]};
    }
    if (!last_block(&ws->arrived)) return;
    // the partials of all blocks: thread j takes block j (kStatThreads == kStatBlocks), then a tree
    static_assert(kStatThreads == kStatBlocks, "one partial per thread");
    const Moments pj = ws->part[threadIdx.x];
    double u[5] = {pj.n, pj.mx, pj.my, pj.vx, pj.vy};
#pragma unroll
    for (int c = 0; c < 5; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u[c] += __shfl_xor_sync(0xFFFFFFFFu, u[c], o);
    }
    __syncthreads();  // red is reused
#pragma unroll
    for (int c = 0; c < 5; ++c)
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = u[c];
    __syncthreads();
    if (threadIdx.x != 0) return;
    double t[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        t[c] = red[c][0];
        for (int w = 1; w < kStatThreads / 32; ++w) t[c] += red[c][w];
    }
    const double cnt = t[0];
    out[0] = cnt;
    if (cnt == 0.0) {
        out[1] = out[2] = 0.0;
    } else {
        const double ax = t[1] / cnt, ay = t[2] / cnt;  // mean - shift
        out[1] = fmax(t[3] / cnt - ax * ax, 0.0);
        out[2] = fmax(t[4] / cnt - ay * ay, 0.0);
    }
    ws->arrived = 0u;
}

template <typename CT>
__global__ void __launch_bounds__(kStatThreads) color_mse_kernel(const CT *__restrict__ a, const CT *__restrict__ b,
                                                                 size_t n, StatWs *ws, double *out, bool psnr) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double d = (double)to_f<CT>(a[i]) - (double)to_f<CT>(b[i]);
        s = fma(d, d, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    __shared__ double warps[kStatThreads / 32];
    if ((threadIdx.x & 31) == 0) warps[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kStatThreads / 32; ++w) t += warps[w];
        ws->part[blockIdx.x].n = t;
    }
    if (!last_block(&ws->arrived) || threadIdx.x != 0) return;
    double t = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) t += ws->part[k].n;
    const double mse = t / (double)n;
    out[0] = mse;
    // PSNR of colours in [0, 1] scaled by 255: 10 log10(255^2 / MSE) = -10 log10(MSE); +inf for equal images
    if (psnr) out[1] = mse == 0.0 ? __longlong_as_double(0x7FF0000000000000ll) : -10.0 * log10(mse);
    ws->arrived = 0u;
}

// SSIM (Sec. IV-C, Eq. 3; the standard 11 x 11 Gaussian-window index, sigma 1.5, C1 = 1e-4, C2 = 9e-4 for
// colours in [0, 1]): each block takes 32 x 32 output positions at a time (a 42 x 42 input tile per channel in
// shared memory), filters the five maps a, b, a^2, b^2, ab horizontally into shared memory, then vertically per
// output, in FP32 on values shifted by -1/2 (variances and covariance are shift-invariant; the shift keeps the
// raw second moments small), and sums the per-position SSIM in FP64 in a fixed order.
constexpr int kSsimTile = 32, kSsimIn = kSsimTile + 10;

template <typename CT>
__global__ void __launch_bounds__(kStatThreads) ssim_kernel(const CT *__restrict__ a, const CT *__restrict__ b,
                                                            int W, int H, StatWs *ws, double *out) {
    __shared__ float ia[kSsimIn][kSsimIn + 1], ib[kSsimIn][kSsimIn + 1];
    __shared__ float hor[5][kSsimIn][kSsimTile];
    __shared__ float g[11];
    __shared__ double red[kStatThreads / 32];
    const int tid = threadIdx.x;
    if (tid < 11) {
        float e[11], sum = 0.0f;
        for (int i = 0; i < 11; ++i) {
            e[i] = expf(-(float)((i - 5) * (i - 5)) / 4.5f);
            sum += e[i];
        }
        g[tid] = e[tid] / sum;
    }
    const int OW = W - 10, OH = H - 10;
    const int ntx = (OW + kSsimTile - 1) / kSsimTile, nt = ntx * ((OH + kSsimTile - 1) / kSsimTile);
    const size_t plane = (size_t)W * H;
    const float C1 = 1e-4f, C2 = 9e-4f;
    double acc = 0.0;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int X0 = (t % ntx) * kSsimTile, Y0 = (t / ntx) * kSsimTile;
        for (int c = 0; c < 3; ++c) {
            __syncthreads();  // the previous channel's tiles are consumed
            for (int i = tid; i < kSsimIn * kSsimIn; i += kStatThreads) {
                const int r = i / kSsimIn, q = i - r * kSsimIn, x = X0 + q, y = Y0 + r;
                const bool in = x < W && y < H;
                const size_t o = c * plane + (size_t)y * W + x;
                ia[r][q] = in ? to_f<CT>(a[o]) - 0.5f : 0.0f;
                ib[r][q] = in ? to_f<CT>(b[o]) - 0.5f : 0.0f;
            }
            __syncthreads();
            for (int i = tid; i < kSsimIn * kSsimTile; i += kStatThreads) {
                const int r = i / kSsimTile, q = i - r * kSsimTile;
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
#pragma unroll
                for (int j = 0; j < 11; ++j) {
                    const float va = ia[r][q + j], vb = ib[r][q + j], w = g[j];
                    s0 = fmaf(w, va, s0);
                    s1 = fmaf(w, vb, s1);
                    s2 = fmaf(w, va * va, s2);
                    s3 = fmaf(w, vb * vb, s3);
                    s4 = fmaf(w, va * vb, s4);
                }
                hor[0][r][q] = s0;
                hor[1][r][q] = s1;
                hor[2][r][q] = s2;
                hor[3][r][q] = s3;
                hor[4][r][q] = s4;
            }
            __syncthreads();
            for (int i = tid; i < kSsimTile * kSsimTile; i += kStatThreads) {
                const int r = i / kSsimTile, q = i - r * kSsimTile;
                if (X0 + q >= OW || Y0 + r >= OH) continue;
                float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int k = 0; k < 11; ++k) {
                    const float w = g[k];
#pragma unroll
                    for (int v = 0; v < 5; ++v) m[v] = fmaf(w, hor[v][r + k][q], m[v]);
                }
                const float va2 = m[2] - m[0] * m[0], vb2 = m[3] - m[1] * m[1], cab = m[4] - m[0] * m[1];
                const float mua = m[0] + 0.5f, mub = m[1] + 0.5f;
                const float num = (2.0f * mua * mub + C1) * (2.0f * cab + C2);
                const float den = (mua * mua + mub * mub + C1) * (va2 + vb2 + C2);
                acc += (double)(num / den);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        double s = red[0];
        for (int w = 1; w < kStatThreads / 32; ++w) s += red[w];
        ws->part[blockIdx.x].n = s;
    }
    if (!last_block(&ws->arrived)) return;
    static_assert(kStatThreads == kStatBlocks, "one partial per thread");
    double u = tid < (int)gridDim.x ? ws->part[tid].n : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xFFFFFFFFu, u, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = u;
    __syncthreads();
    if (tid != 0) return;
    double s = red[0];
    for (int w = 1; w < kStatThreads / 32; ++w) s += red[w];
    out[0] = s / (3.0 * (double)OW * (double)OH);
    ws->arrived = 0u;
}

}  // namespace

size_t stats_workspace_bytes() { return (sizeof(StatWs) + 255) & ~(size_t)255; }

cudaError_t launch_mv_variance(const float *mv, int W, int H, double *out, void *ws, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&static_cast<StatWs *>(ws)->arrived, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    timing_begin("exw_mv_variance", s);
    mv_variance_kernel<<<kStatBlocks, kStatThreads, 0, s>>>(mv, (size_t)W * H, static_cast<StatWs *>(ws), out);
    count_launch();
    timing_end("exw_mv_variance", s);
    return cudaGetLastError();
}

cudaError_t launch_color_mse(const void *a, const void *b, exw_dtype cdt, int W, int H, double *out, void *ws,
                             cudaStream_t s, bool psnr) {
    cudaError_t e = cudaMemsetAsync(&static_cast<StatWs *>(ws)->arrived, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const size_t n = 3 * (size_t)W * H;
    timing_begin("exw_color_mse", s);
    if (cdt == EXW_F16)
        color_mse_kernel<__half><<<kStatBlocks, kStatThreads, 0, s>>>((const __half *)a, (const __half *)b, n,
                                                                       static_cast<StatWs *>(ws), out, psnr);
    else
        color_mse_kernel<float><<<kStatBlocks, kStatThreads, 0, s>>>((const float *)a, (const float *)b, n,
                                                                      static_cast<StatWs *>(ws), out, psnr);
    count_launch();
    timing_end("exw_color_mse", s);
    return cudaGetLastError();
}

}  // namespace exw

namespace exw {

cudaError_t launch_ssim(const void *a, const void *b, exw_dtype cdt, int W, int H, double *out, void *ws,
                        cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&static_cast<StatWs *>(ws)->arrived, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    timing_begin("exw_ssim", s);
    if (cdt == EXW_F16)
        ssim_kernel<__half><<<kStatBlocks, kStatThreads, 0, s>>>((const __half *)a, (const __half *)b, W, H,
                                                                  static_cast<StatWs *>(ws), out);
    else
        ssim_kernel<float><<<kStatBlocks, kStatThreads, 0, s>>>((const float *)a, (const float *)b, W, H,
                                                                 static_cast<StatWs *>(ws), out);
    count_launch();
    timing_end("exw_ssim", s);
    return cudaGetLastError();
}

}  // namespace exw
