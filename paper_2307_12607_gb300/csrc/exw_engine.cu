// exw_engine.cu -- the warp-specialised persistent kernel of the fused forward pass (exw_engine.cuh) and its
// launcher: one CTA of 800 threads per SM, about 166 KB of shared memory.
#include "exw_engine.cuh"

namespace exw {

template <typename CT, int WX, int WY, bool FILL>
__global__ void __launch_bounds__(kEngineThreads, 1)
    engine_kernel(TileParams p, const __grid_constant__ CUtensorMap tcol, const __grid_constant__ CUtensorMap tdep,
                  const __grid_constant__ CUtensorMap tmv, int vec) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    EngineSmem<CT, WX, WY> &s = *reinterpret_cast<EngineSmem<CT, WX, WY> *>(smem_raw);
    if (threadIdx.x == 0) {
        mbar_init(&s.full[0], 1);
        mbar_init(&s.full[1], 1);
        mbar_init(&s.empty[0], kConsumerWarps);
        mbar_init(&s.empty[1], kConsumerWarps);
        fence_mbar_init();
        s.abort = 0;
        for (int g = 0; g < kMaxFrac; ++g) s.last[g] = 0;
    }
    __syncthreads();
    if (threadIdx.x >= kConsumerThreads) engine_producer(s, p, &tcol, &tdep, &tmv);
    else engine_consumer<CT, WX, WY, FILL>(s, p, vec != 0);
}

template <typename CT, int WX, int WY, bool FILL>
static cudaError_t launch_engine_t(const TileParams &p, const TmaMaps &m, int grid, bool vec, cudaStream_t s) {
    constexpr size_t kSmem = sizeof(EngineSmem<CT, WX, WY>);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(engine_kernel<CT, WX, WY, FILL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    engine_kernel<CT, WX, WY, FILL><<<grid, kEngineThreads, kSmem, s>>>(p, m.col, m.depth, m.mv, vec ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_engine(const TileParams &p, const TmaMaps &m, exw_dtype cdt, bool fill, int grid, bool vec,
                          cudaStream_t s) {
    timing_begin("exw_engine", s);
    cudaError_t e;
    if (cdt == EXW_F32)
        e = fill ? launch_engine_t<float, kWinXF32, kWinYF32, true>(p, m, grid, vec, s)
                 : launch_engine_t<float, kWinXF32, kWinYF32, false>(p, m, grid, vec, s);
    else
        e = fill ? launch_engine_t<__half, kWinXF16, kWinYF16, true>(p, m, grid, vec, s)
                 : launch_engine_t<__half, kWinXF16, kWinYF16, false>(p, m, grid, vec, s);
    count_launch();
    timing_end("exw_engine", s);
    return e;
}

}  // namespace exw
