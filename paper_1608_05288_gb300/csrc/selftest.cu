// util_selftest_wait: exercises the library's bounded device-side wait on a
// barrier that nothing completes, so that callers (and the tests) can see the
// failure path end in GPUBE_ETIMEDOUT with a usable context.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gpube_internal.h"

using namespace gpube;

namespace {
static __device__ int32_t g_selftest_status;
}

extern "C" int util_selftest_wait(uint64_t timeout_ns, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t *status = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&status), g_selftest_status);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = launch_selftest_wait(status, timeout_ns, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "util_selftest_wait");
    int32_t h = 0;
    e = cudaMemcpy(&h, status, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "util_selftest_wait status");
    if (h == kStatusTimeout) return set_error(GPUBE_ETIMEDOUT, "bounded wait gave up after %llu ns (expected)",
                                              static_cast<unsigned long long>(timeout_ns));
    return GPUBE_OK;
}
