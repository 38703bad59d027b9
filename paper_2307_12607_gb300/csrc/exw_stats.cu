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
                                                                 size_t n, StatWs *ws, double *out) {
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
    out[0] = t / (double)n;
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
                             cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&static_cast<StatWs *>(ws)->arrived, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const size_t n = 3 * (size_t)W * H;
    timing_begin("exw_color_mse", s);
    if (cdt == EXW_F16)
        color_mse_kernel<__half><<<kStatBlocks, kStatThreads, 0, s>>>((const __half *)a, (const __half *)b, n,
                                                                       static_cast<StatWs *>(ws), out);
    else
        color_mse_kernel<float><<<kStatBlocks, kStatThreads, 0, s>>>((const float *)a, (const float *)b, n,
                                                                      static_cast<StatWs *>(ws), out);
    count_launch();
    timing_end("exw_color_mse", s);
    return cudaGetLastError();
}

}  // namespace exw
