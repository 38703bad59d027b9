// exw_engine.cu -- the persistent engine kernel (exw_engine.cuh): one CTA of 800 threads per SM, about 165 KB of
// shared memory, working through the item queue of up to 48 streams.
#include "exw_engine.cuh"

namespace exw {

template <bool FILL>
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
    __syncthreads();
    if (threadIdx.x >= kConsumerThreads) engine_producer(s, ep);
    else engine_consumer<FILL>(s, ep.status);
}

cudaError_t launch_engine(const EngineParams &ep, bool fill, int grid, cudaStream_t s) {
    constexpr size_t kSmem = sizeof(EngineSmem);
    static bool configured = false;
    if (!configured) {
        cudaError_t e =
            cudaFuncSetAttribute(engine_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(engine_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    timing_begin("exw_engine", s);
    if (fill) engine_kernel<true><<<grid, kEngineThreads, kSmem, s>>>(ep);
    else engine_kernel<false><<<grid, kEngineThreads, kSmem, s>>>(ep);
    count_launch();
    timing_end("exw_engine", s);
    return cudaGetLastError();
}

}  // namespace exw
