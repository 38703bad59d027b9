// exw_engine.cu -- the persistent engine kernel (exw_engine.cuh): one CTA of 800 threads per SM, 199.7 KB of shared
// memory, working through the item queue of up to 48 streams.
#include "exw_engine.cuh"

namespace exw {

template <bool FILL, int SHAPE>
__global__ void __launch_bounds__(kEngineThreads, 1) engine_kernel(const __grid_constant__ EngineParams ep) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    EngineSmem &s = *reinterpret_cast<EngineSmem *>(smem_raw);
    if (threadIdx.x == 0) {
        mbar_init(&s.full[0], 1);
        mbar_init(&s.full[1], 1);
        mbar_init(&s.empty[0], kConsumerWarps);
        mbar_init(&s.empty[1], kConsumerWarps);
        fence_mbar_init();
        s.abort = 0;
    }
    // both key sets start empty; a group empties its fraction's keys again after each gather from them
    for (int r = threadIdx.x; r < 2 * kMaxFrac * kRegionN; r += blockDim.x) (&s.key[0][0][0])[r] = kKeyEmpty;
    grid_dependency_wait();  // the bounds and plan kernels of the first stream, or the previous launch
    __syncthreads();
    if (threadIdx.x >= kConsumerThreads) engine_producer<SHAPE>(s, ep);
    else engine_consumer<FILL, SHAPE>(s, ep);
}

template <bool FILL, int SHAPE>
static cudaError_t launch_one(const EngineParams &ep, int grid, cudaStream_t s) {
    constexpr size_t kSmem = sizeof(EngineSmem);
    // set on every launch: the attribute belongs to the current device's context
    const cudaError_t e =
        cudaFuncSetAttribute(engine_kernel<FILL, SHAPE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    return launch_dependent(engine_kernel<FILL, SHAPE>, dim3(grid), dim3(kEngineThreads), kSmem, s, ep);
}

cudaError_t launch_engine(const EngineParams &ep, bool fill, int shape, int grid, cudaStream_t s) {
    timing_begin("exw_engine", s);
    cudaError_t e;
    if (shape == 0) e = fill ? launch_one<true, 0>(ep, grid, s) : launch_one<false, 0>(ep, grid, s);
    else e = fill ? launch_one<true, 1>(ep, grid, s) : launch_one<false, 1>(ep, grid, s);
    count_launch();
    timing_end("exw_engine", s);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace exw
