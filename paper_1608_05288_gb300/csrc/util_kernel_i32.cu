// Instantiation of the UTIL and VALUE kernels for integer WCSP costs saturating at the top cost (Section 2).
#include "util_kernel.cuh"
#include "value_kernel.cuh"

namespace gpube {

cudaError_t launch_util_i32(const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s, bool pdl)
{
    return launch_util_kernel(util_kernel<Cost<int32_t>>, L, grid, threads, smem, s, pdl);
}

// The single-body instantiations of the two-term rows of domain D (2..4).
cudaError_t launch_util_i32_rows(int D, const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s, bool pdl)
{
    switch (D) {
    case 2: return launch_util_kernel(util_kernel<Cost<int32_t>, 2>, L, grid, threads, smem, s, pdl);
    case 3: return launch_util_kernel(util_kernel<Cost<int32_t>, 3>, L, grid, threads, smem, s, pdl);
    default: return launch_util_kernel(util_kernel<Cost<int32_t>, 4>, L, grid, threads, smem, s, pdl);
    }
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

int util_max_blocks_i32_rows(int D, int threads, int smem)
{
    int nb = 0;
    cudaError_t e;
    switch (D) {
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<Cost<int32_t>, 2>, threads, smem); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<Cost<int32_t>, 3>, threads, smem); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<Cost<int32_t>, 4>, threads, smem); break;
    }
    if (e != cudaSuccess) {
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
        e = cudaFuncSetAttribute(util_kernel<Cost<int32_t>, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(util_kernel<Cost<int32_t>, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(util_kernel<Cost<int32_t>, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(value_kernel<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(value_kernel_batch<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    return e;
}

}  // namespace gpube
