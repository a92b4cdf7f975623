// Instantiation of the UTIL kernel for the sum-product problem: fp32 -log
// weights, each variable eliminated by -log sum exp(-.) (the weighted counting
// / partition function extension of the conclusions; solution counting,
// Section 2.1).  Its root reduction runs on the fp32 VALUE kernel.
#include "util_kernel.cuh"

namespace gpube {

cudaError_t launch_util_sum(const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s, bool pdl)
{
    return launch_util_kernel(util_kernel<SumProduct>, L, grid, threads, smem, s, pdl);
}

// The single-body instantiations of the factored two-term rows of domain D (2..4).
cudaError_t launch_util_sum_rows(int D, const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s, bool pdl)
{
    switch (D) {
    case 2: return launch_util_kernel(util_kernel<SumProduct, 2>, L, grid, threads, smem, s, pdl);
    case 3: return launch_util_kernel(util_kernel<SumProduct, 3>, L, grid, threads, smem, s, pdl);
    default: return launch_util_kernel(util_kernel<SumProduct, 4>, L, grid, threads, smem, s, pdl);
    }
}

int util_max_blocks_sum(int threads, int smem)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<SumProduct>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

int util_max_blocks_sum_rows(int D, int threads, int smem)
{
    int nb = 0;
    cudaError_t e;
    switch (D) {
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<SumProduct, 2>, threads, smem); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<SumProduct, 3>, threads, smem); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<SumProduct, 4>, threads, smem); break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t kernel_attrs_sum(int max_smem)
{
    cudaError_t e = cudaFuncSetAttribute(util_kernel<SumProduct>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(util_kernel<SumProduct, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(util_kernel<SumProduct, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(util_kernel<SumProduct, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    return e;
}

}  // namespace gpube
