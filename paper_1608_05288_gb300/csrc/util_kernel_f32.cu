// Instantiation of the UTIL and VALUE kernels for fp32 -log p costs (Section 3).
#include "util_kernel.cuh"

namespace gpube {

cudaError_t launch_util_f32(const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(util_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    util_kernel<float><<<grid, threads, smem, s>>>(L);
    return cudaGetLastError();
}

int util_max_blocks_f32(int threads, int smem)
{
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(util_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<float>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_value_f32(const ValueDev &V, int smem, cudaStream_t s)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(value_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    value_kernel<float><<<1, 256, smem, s>>>(V);
    return cudaGetLastError();
}

}  // namespace gpube
