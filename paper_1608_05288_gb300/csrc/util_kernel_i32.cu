// Instantiation of the UTIL and VALUE kernels for integer WCSP costs saturating at the top cost (Section 2).
#include "util_kernel.cuh"
#include "value_kernel.cuh"

namespace gpube {

cudaError_t launch_util_i32(const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s, bool pdl)
{
    return launch_util_kernel(util_kernel<Cost<int32_t>>, L, grid, threads, smem, s, pdl);
}

cudaError_t launch_util_i32_rows4(const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s, bool pdl)
{
    return launch_util_kernel(util_kernel<Cost<int32_t>, 1>, L, grid, threads, smem, s, pdl);
}

int util_max_blocks_i32(int threads, int smem)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<Cost<int32_t>>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

int util_max_blocks_i32_rows4(int threads, int smem)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<Cost<int32_t>, 1>, threads, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_value_i32(const ValueDev &V, int smem, cudaStream_t s)
{
    value_kernel<int32_t><<<1, 256, smem, s>>>(V);
    return cudaGetLastError();
}

cudaError_t launch_value_batch_i32(const ValueBatch &B, int smem, cudaStream_t s)
{
    value_kernel_batch<int32_t><<<B.n, 256, smem, s>>>(B);
    return cudaGetLastError();
}

// Raise the dynamic shared-memory limit of this type's kernels to the
// device maximum, once per device, outside any stream capture.
cudaError_t kernel_attrs_i32(int max_smem)
{
    cudaError_t e = cudaFuncSetAttribute(util_kernel<Cost<int32_t>>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(util_kernel<Cost<int32_t>, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(value_kernel<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(value_kernel_batch<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    return e;
}

}  // namespace gpube
