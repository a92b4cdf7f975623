// Plan expansion kernel and the cost-type dispatch of the launchers.
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

#include "gpube_dev.h"

namespace gpube {

// defined in util_kernel_i32.cu / util_kernel_f32.cu / util_kernel_sum.cu
cudaError_t launch_util_i32(const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s, bool pdl);
cudaError_t launch_util_f32(const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s, bool pdl);
cudaError_t launch_util_sum(const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s, bool pdl);
cudaError_t launch_util_i32_rows(int D, const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s, bool pdl);
cudaError_t launch_util_sum_rows(int D, const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s, bool pdl);
int util_max_blocks_i32(int threads, int smem);
int util_max_blocks_f32(int threads, int smem);
int util_max_blocks_sum(int threads, int smem);
int util_max_blocks_i32_rows(int D, int threads, int smem);
int util_max_blocks_sum_rows(int D, int threads, int smem);
cudaError_t launch_value_i32(const ValueDev &V, int smem, cudaStream_t s);
cudaError_t launch_value_f32(const ValueDev &V, int smem, cudaStream_t s);
cudaError_t launch_value_batch_i32(const ValueBatch &B, int smem, cudaStream_t s);
cudaError_t launch_value_batch_f32(const ValueBatch &B, int smem, cudaStream_t s);
cudaError_t kernel_attrs_i32(int max_smem);
cudaError_t kernel_attrs_f32(int max_smem);
cudaError_t kernel_attrs_sum(int max_smem);

// ------------------------------------------------------ plan expansion
// Fills every task's A and B offset tables from its compact plan: the row h
// of A decodes h in the task's hi iteration order; the row lo of B decodes
// the lowest separator digits.  Each entry is sum(digit * input stride).
__global__ void expand_kernel(const ExpandDev *tasks, const int64_t *prefix, int n_tasks, int64_t total,
                              const int32_t *pool)
{
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int a = 0, b = n_tasks;
        while (b - a > 1) {
            const int mid = (a + b) >> 1;
            if (prefix[mid] <= e) a = mid;
            else b = mid;
        }
        const ExpandDev x = tasks[a];
        const int32_t *rad = pool + x.rad_off;
        const int32_t *perm = pool + x.perm_off;
        const int32_t *st = pool + x.stride_off;
        int64_t r = e - prefix[a];
        if (r <= x.G) {
            // group rows: the hi digits other than the fastest one (perm[0]);
            // row G: the strides of perm[0] (zero when there is no hi digit)
            int32_t *row = x.A + r * x.sa;
            for (int f = 0; f < x.sa; ++f) row[f] = 0;
            if (r == x.G) {
                if (x.nh > 0) {
                    const int j = perm[0];
                    row[0] = st[x.F * x.m + j];
                    for (int f = 0; f < x.F; ++f) row[1 + f] = st[f * x.m + j];
                }
            } else {
                int64_t h = r;
                for (int i = 1; i < x.nh; ++i) {
                    const int j = perm[i];
                    const int dig = static_cast<int>(h % rad[j]);
                    h /= rad[j];
                    if (dig) {
                        row[0] += dig * st[x.F * x.m + j];
                        for (int f = 0; f < x.F; ++f) row[1 + f] += dig * st[f * x.m + j];
                    }
                }
            }
        } else {
            const int64_t lo = r - x.G - 1;
            int32_t *row = x.B + lo * x.sb;
            for (int f = 0; f < x.sb; ++f) row[f] = 0;
            int64_t q = lo;
            for (int j = x.m - 1; j >= x.m - x.L; --j) {
                const int dig = static_cast<int>(q % rad[j]);
                q /= rad[j];
                if (dig)
                    for (int f = 0; f < x.F; ++f) row[f] += dig * st[f * x.m + j];
            }
        }
    }
}

// ------------------------------------------------------ wait self-test
// One CTA waits on an mbarrier that nothing ever arrives at: the bounded wait
// must give up after limit_ns, record the timeout and return, leaving the
// context usable.
__device__ __forceinline__ uint32_t st_smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__global__ void selftest_wait_kernel(int32_t *status, unsigned long long limit_ns)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(st_smem_addr(&bar)), "r"(1) : "memory");
    __syncthreads();
    const unsigned long long t0 = [] {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        return t;
    }();
    bool ok = false;
    for (int i = 0; i < kMaxSpin && !ok; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(st_smem_addr(&bar)), "r"(0)
            : "memory");
        ok = done != 0;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) break;
    }
    if (__syncthreads_or(!ok) && threadIdx.x == 0) *status = kStatusTimeout;
}

cudaError_t launch_selftest_wait(int32_t *status, unsigned long long limit_ns, cudaStream_t s)
{
    selftest_wait_kernel<<<1, 64, 0, s>>>(status, limit_ns);
    return cudaGetLastError();
}

// -------------------------------------------------------- host launchers
// ktype: kKTypeInt (int32 min-sum), kKTypeFloat (fp32 min-sum), kKTypeSum
// (fp32 sum-product), kKTypeIntRows + D - 2 / kKTypeSumRows + D - 2 (the
// same, two-term rows of domain D = 2..4 only)
cudaError_t launch_util(const LaunchDev &L, int ktype, int grid, int threads, int smem, cudaStream_t s, bool pdl)
{
    if (ktype >= kKTypeIntRows && ktype < kKTypeIntRows + 3)
        return launch_util_i32_rows(ktype - kKTypeIntRows + 2, L, grid, threads, smem, s, pdl);
    if (ktype >= kKTypeSumRows && ktype < kKTypeSumRows + 3)
        return launch_util_sum_rows(ktype - kKTypeSumRows + 2, L, grid, threads, smem, s, pdl);
    switch (ktype) {
    case kKTypeFloat: return launch_util_f32(L, grid, threads, smem, s, pdl);
    case kKTypeSum: return launch_util_sum(L, grid, threads, smem, s, pdl);
    default: return launch_util_i32(L, grid, threads, smem, s, pdl);
    }
}

// Resident CTAs per SM for a launch shape, cached per (device, instantiation,
// CTA size, shared memory): every plan and every merged server launch asks.
int util_max_blocks_per_sm(int ktype, int threads, int smem)
{
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, ktype, threads, smem);
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int nb;
    if (ktype >= kKTypeIntRows && ktype < kKTypeIntRows + 3) {
        nb = util_max_blocks_i32_rows(ktype - kKTypeIntRows + 2, threads, smem);
    } else if (ktype >= kKTypeSumRows && ktype < kKTypeSumRows + 3) {
        nb = util_max_blocks_sum_rows(ktype - kKTypeSumRows + 2, threads, smem);
    } else {
        switch (ktype) {
        case kKTypeFloat: nb = util_max_blocks_f32(threads, smem); break;
        case kKTypeSum: nb = util_max_blocks_sum(threads, smem); break;
        default: nb = util_max_blocks_i32(threads, smem); break;
        }
    }
    std::lock_guard<std::mutex> g(mu);
    cache[key] = nb;
    return nb;
}

cudaError_t launch_expand(const ExpandDev *tasks, const int64_t *prefix, int n_tasks, int64_t total,
                          const int32_t *pool, int num_sms, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    int64_t want = (total + 255) / 256;
    int grid = static_cast<int>(want < 8LL * num_sms ? want : 8LL * num_sms);
    expand_kernel<<<grid, 256, 0, s>>>(tasks, prefix, n_tasks, total, pool);
    return cudaGetLastError();
}

cudaError_t launch_value(const ValueDev &V, int ktype, int smem, cudaStream_t s)
{
    return ktype == kKTypeInt ? launch_value_i32(V, smem, s) : launch_value_f32(V, smem, s);
}

cudaError_t launch_value_batch(const ValueBatch &B, int ktype, int smem, cudaStream_t s)
{
    if (B.n <= 0) return cudaSuccess;
    return ktype == kKTypeInt ? launch_value_batch_i32(B, smem, s) : launch_value_batch_f32(B, smem, s);
}

// Largest dynamic shared memory a UTIL launch may request on the current
// device (the attribute kernels_init_device sets).
int max_dynamic_smem()
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 48 * 1024;
    }
    return optin - 1024;
}

// Once per device (current device): allow every kernel the device's largest
// dynamic shared-memory size, so that no launch needs an attribute change
// (in particular none during a stream capture).
cudaError_t kernels_init_device()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(mu);
    if (done[dev]) return cudaSuccess;
    int max_smem = 0;
    e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = kernel_attrs_i32(max_smem - 1024);
    if (e == cudaSuccess) e = kernel_attrs_f32(max_smem - 1024);
    if (e == cudaSuccess) e = kernel_attrs_sum(max_smem - 1024);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

}  // namespace gpube
