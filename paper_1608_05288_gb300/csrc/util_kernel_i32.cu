// Instantiation of the UTIL and VALUE kernels for integer WCSP costs saturating at the top cost (Section 2).
#include "util_kernel.cuh"

namespace gpube {

cudaError_t launch_util_i32(const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(util_kernel<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    util_kernel<int32_t><<<grid, threads, smem, s>>>(L);
    return cudaGetLastError();
}

int util_max_blocks_i32(int threads, int smem)
{
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(util_kernel<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<int32_t>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_value_i32(const ValueDev &V, int smem, cudaStream_t s)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(value_kernel<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    value_kernel<int32_t><<<1, 256, smem, s>>>(V);
    return cudaGetLastError();
}

}  // namespace gpube
