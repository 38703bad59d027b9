// exw_aux.cu -- global-memory splat, motion bounds, workspace clearing and the L2 loss.
#include "exw_items.cuh"

namespace exw {

__global__ void clear_keys_kernel(unsigned long long *keys, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        keys[i] = kKeyEmpty;
}

__global__ void zero_kernel(uint32_t *p, size_t nwords) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += (size_t)gridDim.x * blockDim.x)
        p[i] = 0u;
}

// Stage (a) into a global key buffer: one thread per source pixel, 64-bit atomicMin at the target.
__global__ void __launch_bounds__(256) splat_global_kernel(const float *__restrict__ depth,
                                                           const float *__restrict__ mv, int W, int H, int k, int L,
                                                           unsigned long long *keys) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const size_t plane = (size_t)W * H;
    const size_t i = (size_t)y * W + x;
    const uint32_t db = __float_as_uint(__ldg(depth + i));
    const uint32_t ux = __float_as_uint(__ldg(mv + i)), uy = __float_as_uint(__ldg(mv + plane + i));
    if (!depth_ok(db) || !finite_bits(ux) || !finite_bits(uy)) return;
    const AxisDec dx = axis_dec(ux, L), dy = axis_dec(uy, L);
    if (!dx.land || !dy.land) return;
    const int gx = x + axis_off(dx, k), gy = y + axis_off(dy, k);
    if (gx < 0 || gx >= W || gy < 0 || gy >= H) return;
    atomicMin(keys + (size_t)gy * W + gx, (unsigned long long)pack_key_global(db, (uint32_t)i));
}

// Stage (a0): one 32 x 32 source region per CTA of 4 warps (8 rows each, 24 loads in flight per thread), up to 12
// CTAs per SM.
__global__ void __launch_bounds__(128, 12) bounds_kernel(const float *__restrict__ depth, const float *__restrict__ mv,
                                                        int W, int H, float4 *tile_bounds, float2 *tile_depth,
                                                        float4 *region_bounds, FrameHeader *fh) {
    __shared__ float4 part[32];
    grid_dependency_wait();  // the frame header is zeroed by the kernel before
    grid_dependents_launch();
    bounds_region<4>(depth, mv, W, H, tile_bounds, tile_depth, region_bounds, fh, blockIdx.x, blockIdx.y, part, true,
                     (int)threadIdx.x, CtaBarrier{});
}

__global__ void bounds_finalize_kernel(const FrameHeader *fh, float *out) {
    if (threadIdx.x != 0) return;
    if (fh->acc[1] == 0u) {
        out[0] = __int_as_float(0x7F800000);
        out[1] = __int_as_float(0xFF800000);
        out[2] = __int_as_float(0x7F800000);
        out[3] = __int_as_float(0xFF800000);
        return;
    }
    out[0] = -float_unorder(fh->acc[0]);
    out[1] = float_unorder(fh->acc[1]);
    out[2] = -float_unorder(fh->acc[2]);
    out[3] = float_unorder(fh->acc[3]);
}

template <typename CT>
__global__ void __launch_bounds__(256) l2_loss_kernel(const CT *__restrict__ out, const CT *__restrict__ target,
                                                      const uint8_t *__restrict__ mask, size_t n, float *grad,
                                                      float *loss) {
    __shared__ float red[8];
    float acc = 0.0f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const bool valid = __ldg(mask + i) == 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float d = load_c<CT>(out + c * n + i) - load_c<CT>(target + c * n + i);
            grad[c * n + i] = valid ? 2.0f * d : 0.0f;
            if (valid) acc += d * d;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if (threadIdx.x == 0) atomicAdd(loss, v);
    }
}

static unsigned grid_for(size_t n, unsigned per_block) {
    size_t g = (n + per_block - 1) / per_block;
    if (g > 8192) g = 8192;
    return (unsigned)(g ? g : 1);
}

cudaError_t launch_clear_keys(uint64_t *keys, size_t n, cudaStream_t s) {
    timing_begin("exw_clear_keys", s);
    clear_keys_kernel<<<grid_for(n, 256 * 4), 256, 0, s>>>((unsigned long long *)keys, n);
    count_launch();
    timing_end("exw_clear_keys", s);
    return cudaGetLastError();
}

cudaError_t launch_zero(void *p, size_t bytes, cudaStream_t s) {
    const size_t words = bytes / 4;
    zero_kernel<<<grid_for(words, 256 * 4), 256, 0, s>>>((uint32_t *)p, words);
    count_launch();
    return cudaGetLastError();
}

// Depth and motion of a warped frame for warping it again (the recursive warps of decision paths S5/S6, Table V):
// a target that is not a hole takes its winner's depth and motion bits; a hole gets depth NaN (it never lands
// again) and motion 0.  One target per thread (coalesced reads of keys and mask, gathered reads of the winners).
__global__ void __launch_bounds__(256) carry_motion_kernel(const uint64_t *__restrict__ keys,
                                                           const uint8_t *__restrict__ mask,
                                                           const float *__restrict__ depth,
                                                           const float *__restrict__ mv, size_t n,
                                                           float *__restrict__ depth_out, float *__restrict__ mv_out) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint64_t k = keys[q];
    if (mask[q] == 0 && k != kKeyEmpty) {
        const size_t p = (size_t)(k & 0xFFFFFFFFull);
        depth_out[q] = __ldg(depth + p);
        mv_out[q] = __ldg(mv + p);
        mv_out[n + q] = __ldg(mv + n + p);
    } else {
        depth_out[q] = __int_as_float(0x7FC00000);
        mv_out[q] = 0.0f;
        mv_out[n + q] = 0.0f;
    }
}

cudaError_t launch_carry_motion(const uint64_t *keys, const uint8_t *mask, const float *depth, const float *mv,
                                int W, int H, float *depth_out, float *mv_out, cudaStream_t s) {
    const size_t n = (size_t)W * H;
    timing_begin("exw_carry_motion", s);
    carry_motion_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, mask, depth, mv, n, depth_out, mv_out);
    count_launch();
    timing_end("exw_carry_motion", s);
    return cudaGetLastError();
}

cudaError_t launch_splat_global(const float *depth, const float *mv, int W, int H, int k, int L, uint64_t *keys,
                                cudaStream_t s) {
    const dim3 g((unsigned)((W + 255) / 256), (unsigned)H, 1);
    timing_begin("exw_splat_global", s);
    splat_global_kernel<<<g, 256, 0, s>>>(depth, mv, W, H, k, L, (unsigned long long *)keys);
    count_launch();
    timing_end("exw_splat_global", s);
    return cudaGetLastError();
}

cudaError_t launch_bounds(const float *depth, const float *mv, int W, int H, float4 *tile_bounds, float2 *tile_depth,
                          float4 *region_bounds, FrameHeader *fh, cudaStream_t s) {
    const dim3 g((unsigned)ceil_div(W, 32), (unsigned)ceil_div(H, 32), 1);
    timing_begin("exw_bounds", s);
    const cudaError_t e = launch_dependent(bounds_kernel, g, dim3(128), 0, s, depth, mv, W, H, tile_bounds, tile_depth,
                                           region_bounds, fh);
    count_launch();
    timing_end("exw_bounds", s);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_bounds_finalize(const FrameHeader *fh, float *frame_bounds, cudaStream_t s) {
    bounds_finalize_kernel<<<1, 32, 0, s>>>(fh, frame_bounds);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_l2_loss(const void *out, const void *target, exw_dtype cdt, const uint8_t *mask, int W, int H,
                           float *grad_out, float *loss, cudaStream_t s) {
    const size_t n = (size_t)W * H;
    const unsigned g = grid_for(n, 256 * 4);
    timing_begin("exw_l2_loss", s);
    if (cdt == EXW_F32)
        l2_loss_kernel<float><<<g, 256, 0, s>>>((const float *)out, (const float *)target, mask, n, grad_out, loss);
    else
        l2_loss_kernel<__half><<<g, 256, 0, s>>>((const __half *)out, (const __half *)target, mask, n, grad_out,
                                                 loss);
    count_launch();
    timing_end("exw_l2_loss", s);
    return cudaGetLastError();
}

}  // namespace exw
