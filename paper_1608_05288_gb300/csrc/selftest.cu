// Diagnostics of the library's bounded device-side waits: each runs one wait
// that nothing will ever satisfy, so that callers (and the tests) can see the
// failure path end in GPUBE_ETIMEDOUT with a usable context.
//   util_selftest_wait      the wait on a TMA mbarrier of the UTIL kernel;
//   util_selftest_dep_wait  the wait of a launch over several levels for the
//                           tasks that produce a task's inputs.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gpube_internal.h"
#include "util_kernel.cuh"

using namespace gpube;

namespace {
static __device__ int32_t g_selftest_status;

// A two-task launch in which task 1 reads task 0's output, with task 0's
// completion count held at zero: prefix [0, 1, 2], dep_off [0, 0, 1],
// deps [0], done [0, 0].
static __device__ int32_t g_dep_fake[16];

__global__ void selftest_dep_wait_kernel(int32_t *fake, int32_t *status, unsigned long long limit_ns)
{
    if (threadIdx.x != 0) return;
    LaunchDev L{};
    L.prefix = fake;
    L.dep_off = fake + 4;
    L.deps = fake + 8;
    L.done = fake + 12;
    L.status = status;
    L.n_tasks = 2;
    L.total_items = 2;
    if (!wait_producers(L, 1, limit_ns)) atomicExch(status, kStatusTimeout);
}

int finish(cudaError_t e, int32_t *status, cudaStream_t st, uint64_t timeout_ns, const char *what)
{
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, what);
    int32_t h = 0;
    e = cudaMemcpy(&h, status, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, what);
    if (h == kStatusTimeout) return set_error(GPUBE_ETIMEDOUT, "bounded wait gave up after %llu ns (expected)",
                                              static_cast<unsigned long long>(timeout_ns));
    return GPUBE_OK;
}
}  // namespace

extern "C" int util_selftest_wait(uint64_t timeout_ns, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t *status = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&status), g_selftest_status);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = launch_selftest_wait(status, timeout_ns, st);
    return finish(e, status, st, timeout_ns, "util_selftest_wait");
}

extern "C" int util_selftest_dep_wait(uint64_t timeout_ns, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t *status = nullptr, *fake = nullptr;
    const int32_t init[16] = {0, 1, 2, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&status), g_selftest_status);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void **>(&fake), g_dep_fake);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fake, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        selftest_dep_wait_kernel<<<1, 32, 0, st>>>(fake, status, timeout_ns);
        e = cudaGetLastError();
    }
    return finish(e, status, st, timeout_ns, "util_selftest_dep_wait");
}
