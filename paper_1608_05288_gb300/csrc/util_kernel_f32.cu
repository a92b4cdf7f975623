// Instantiation of the UTIL and VALUE kernels for fp32 -log p costs (Section 3).
#include "util_kernel.cuh"
#include "value_kernel.cuh"

namespace gpube {

cudaError_t launch_util_f32(const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s, bool pdl)
{
    return launch_util_kernel(util_kernel<Cost<float>>, L, grid, threads, smem, s, pdl);
}

int util_max_blocks_f32(int threads, int smem)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<Cost<float>>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_value_f32(const ValueDev &V, int smem, cudaStream_t s)
{
    value_kernel<float><<<1, 256, smem, s>>>(V);
    return cudaGetLastError();
}

cudaError_t launch_value_batch_f32(const ValueBatch &B, int smem, cudaStream_t s)
{
    value_kernel_batch<float><<<B.n, 256, smem, s>>>(B);
    return cudaGetLastError();
}

// Raise the dynamic shared-memory limit of this type's kernels to the
// device maximum, once per device, outside any stream capture.
cudaError_t kernel_attrs_f32(int max_smem)
{
    cudaError_t e = cudaFuncSetAttribute(util_kernel<Cost<float>>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(value_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(value_kernel_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    return e;
}

}  // namespace gpube
