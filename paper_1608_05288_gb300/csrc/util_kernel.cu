// UTIL-table kernels for sm_103a.
//
// One kernel computes every bucket function of Algorithms 1-2 (and DPOP's
// UTIL messages): for each separator row r and each value l of the
// eliminated variable x_i it gathers one entry of every input table, sums
// them (saturating at the top cost for integer WCSPs, Section 2; fp32 for
// -log p costs, Section 3), and keeps the minimum and first argmin over l.
// This fuses the paper's Gpu::Aggregate (Eq. 3 gather, Section 6.3) and
// Gpu::Eliminate (Section 6.4): no joint table is materialised, every input
// entry is read where it is needed, the output is written once.
//
// Index arithmetic.  Rows are split r = hi * P_lo + lo (lo = the lowest
// separator digits).  A thread keeps its lo fixed and walks a range of hi
// values; the per-input offsets of Eq. 3 are read from two small tables
// (A[hi][f] uniform across the CTA, B[lo][f] once per thread), so the hot
// loop has no division or modulo.  The order in which hi is walked is the
// planner's choice (digits absent from the largest input first), which makes
// consecutive steps of a thread reread the same input rows from L1 instead
// of DRAM.
//
// Small input tables are staged in shared memory by TMA bulk copies
// (cp.async.bulk, completion on an mbarrier); their x_i-runs are then read
// with vector loads.  Work items (one lo chunk of blockDim.x rows times a
// range of hi values) are taken from an atomic counter, so one launch can
// serve one bucket (the per-bucket form) or every bucket of an
// elimination-tree level (the batched form).
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "gpube_dev.h"

namespace gpube {

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on the staging barrier; false when the limit was reached.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (int i = 0; i < kMaxSpin; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ------------------------------------------------------------ cost ops
template <typename T> struct Cost;

// Integer WCSP costs in [0, k]: sums saturate at k (k means "not allowed").
// Both operands are <= k < 2^31, so their uint32 sum cannot wrap.
template <> struct Cost<int32_t> {
    using acc = uint32_t;
    static __device__ __forceinline__ acc from(int32_t v) { return static_cast<uint32_t>(v); }
    static __device__ __forceinline__ acc add(acc a, int32_t v, uint32_t k)
    {
        uint32_t s = a + static_cast<uint32_t>(v);
        return s < k ? s : k;
    }
    static __device__ __forceinline__ int32_t store(acc a) { return static_cast<int32_t>(a); }
};

// -log p costs in fp32; +inf (p = 0) propagates through the sum.
template <> struct Cost<float> {
    using acc = float;
    static __device__ __forceinline__ acc from(float v) { return v; }
    static __device__ __forceinline__ acc add(acc a, float v, uint32_t) { return a + v; }
    static __device__ __forceinline__ float store(acc a) { return a; }
};

template <typename T> using A_t = typename Cost<T>::acc;

// The d entries of one x_i-run, loaded with the widest aligned vector:
// offsets are multiples of d, so d % 4 == 0 runs are 16-byte aligned.
template <int D, typename T>
__device__ __forceinline__ void load_run(const T *p, T (&v)[D])
{
    if constexpr (D % 4 == 0) {
        using V4 = typename std::conditional<std::is_same<T, float>::value, float4, int4>::type;
#pragma unroll
        for (int i = 0; i < D / 4; ++i) {
            V4 x = reinterpret_cast<const V4 *>(p)[i];
            v[4 * i + 0] = x.x;
            v[4 * i + 1] = x.y;
            v[4 * i + 2] = x.z;
            v[4 * i + 3] = x.w;
        }
    } else if constexpr (D % 2 == 0) {
        using V2 = typename std::conditional<std::is_same<T, float>::value, float2, int2>::type;
#pragma unroll
        for (int i = 0; i < D / 2; ++i) {
            V2 x = reinterpret_cast<const V2 *>(p)[i];
            v[2 * i + 0] = x.x;
            v[2 * i + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i) v[i] = p[i];
    }
}

// Base pointer of input f: its shared-memory copy when staged.
template <typename T>
__device__ __forceinline__ const T *input_base(const InDev &in, const unsigned char *stage)
{
    return in.stage_off >= 0 ? reinterpret_cast<const T *>(stage + in.stage_off)
                             : reinterpret_cast<const T *>(in.ptr);
}

// --------------------------------------------------------- item bodies
template <int N>
__device__ __forceinline__ void load_ints(const int32_t *p, int32_t (&a)[N])
{
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
        const int4 x = reinterpret_cast<const int4 *>(p)[i];
        a[4 * i + 0] = x.x;
        a[4 * i + 1] = x.y;
        a[4 * i + 2] = x.z;
        a[4 * i + 3] = x.w;
    }
}

// Fixed domain D, any number of inputs (offsets reread per input).
template <typename T, int D>
__device__ __forceinline__ void item_fixed_anyF(const TaskDev &tk, const unsigned char *stage, int lo,
                                                int g0, int g1, uint32_t k)
{
    using C = Cost<T>;
    using A = typename C::acc;
    const int F = tk.F;
    const int32_t *Brow = tk.B + static_cast<int64_t>(lo) * tk.sb;
    const int32_t *du = tk.A + static_cast<int64_t>(tk.G) * tk.sa;
    T *out = static_cast<T *>(tk.out);
    for (int g = g0; g < g1; ++g) {
        const int32_t *Ar = tk.A + static_cast<int64_t>(g) * tk.sa;
        for (int u = 0; u < tk.R0; ++u) {
            A acc[D];
#pragma unroll
            for (int l = 0; l < D; ++l) acc[l] = A(0);
            for (int f = 0; f < F; ++f) {
                T v[D];
                load_run<D>(input_base<T>(tk.in[f], stage) + (Ar[1 + f] + u * du[1 + f] + Brow[f]), v);
#pragma unroll
                for (int l = 0; l < D; ++l) acc[l] = C::add(acc[l], v[l], k);
            }
            A best = acc[0];
            int bi = 0;
#pragma unroll
            for (int l = 1; l < D; ++l)
                if (acc[l] < best) {
                    best = acc[l];
                    bi = l;
                }
            const int o = Ar[0] + u * du[0] + lo;
            out[o] = C::store(best);
            tk.arg[o] = static_cast<uint8_t>(bi);
        }
    }
}

// One item for a fixed domain D, at most FC inputs (FC = 3 or 7: A rows of
// FC + 1 ints, one or two 16-byte loads) of which NR are per-row inputs
// (they mention the fastest hi digit u).  Lo-only inputs are summed once per
// item, group inputs once per group (NG groups at a time, so that NG
// independent loads of the large input are in flight per thread), and each
// row adds its NR runs, takes the min and first argmin over x_i and writes
// both.  Row offsets advance by the stride of u: a row costs NR vector
// loads, the adds, the argmin and two stores.
template <typename T, int D, int FC, int NR>
__device__ __forceinline__ void item_fixed_nr(const TaskDev &tk, const unsigned char *stage, int lo, int g0,
                                              int g1, uint32_t k)
{
    using C = Cost<T>;
    using A = typename C::acc;
    constexpr int SA = FC + 1;
    constexpr int SB = (FC + 3) / 4 * 4;
    constexpr int NG = (FC <= 3 && D <= 4) ? 2 : 1;
    constexpr int R = NR > 0 ? NR : 1;
    const int F = tk.F, nlo = tk.n_lo, ngi = tk.n_gi, R0 = tk.R0;
    const int32_t *Brow = tk.B + static_cast<int64_t>(lo) * SB;
    // lo-only inputs: summed once
    A base[D];
#pragma unroll
    for (int l = 0; l < D; ++l) base[l] = A(0);
    for (int f = 0; f < nlo; ++f) {
        T v[D];
        load_run<D>(input_base<T>(tk.in[f], stage) + Brow[f], v);
#pragma unroll
        for (int l = 0; l < D; ++l) base[l] = C::add(base[l], v[l], k);
    }
    // group inputs [nlo, ngi) and per-row inputs [ngi, F)
    const T *gp[FC];
#pragma unroll
    for (int f = 0; f < FC; ++f)
        gp[f] = (f >= nlo && f < ngi) ? input_base<T>(tk.in[f], stage) + Brow[f] : nullptr;
    const T *rp[R];
    int32_t dr[R];
    const int32_t *du = tk.A + static_cast<int64_t>(tk.G) * SA;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        rp[r] = input_base<T>(tk.in[ngi + r], stage) + Brow[ngi + r];
        dr[r] = du[1 + ngi + r];
    }
    const int32_t d0 = du[0];
    T *out = static_cast<T *>(tk.out);
    uint8_t *arg = tk.arg;
    for (int g = g0; g < g1; g += NG) {
        A pre[NG][D];
        int32_t ro[NG][R], oo[NG];
        {
            int32_t a[NG][SA];
#pragma unroll
            for (int j = 0; j < NG; ++j) {
                load_ints<SA>(tk.A + static_cast<int64_t>(g + j < g1 ? g + j : g) * SA, a[j]);
#pragma unroll
                for (int l = 0; l < D; ++l) pre[j][l] = base[l];
            }
            // all group-input loads of the NG groups first, then the sums
#pragma unroll
            for (int f = 0; f < FC; ++f)
                if (f >= nlo && f < ngi) {
                    T x[NG][D];
#pragma unroll
                    for (int j = 0; j < NG; ++j) load_run<D>(gp[f] + a[j][1 + f], x[j]);
#pragma unroll
                    for (int j = 0; j < NG; ++j)
#pragma unroll
                        for (int l = 0; l < D; ++l) pre[j][l] = C::add(pre[j][l], x[j][l], k);
                }
#pragma unroll
            for (int j = 0; j < NG; ++j) {
                oo[j] = a[j][0] + lo;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    ro[j][r] = 0;
#pragma unroll
                    for (int f = 0; f < FC; ++f)
                        if (f == ngi + r) ro[j][r] = a[j][1 + f];
                }
            }
        }
        const int nj = (g + 1 < g1) ? NG : 1;
        for (int u = 0; u < R0; ++u) {
#pragma unroll
            for (int j = 0; j < NG; ++j) {
                if (j < nj) {
                    A acc[D];
#pragma unroll
                    for (int l = 0; l < D; ++l) acc[l] = pre[j][l];
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        T v[D];
                        load_run<D>(rp[r] + ro[j][r], v);
                        ro[j][r] += dr[r];
#pragma unroll
                        for (int l = 0; l < D; ++l) acc[l] = C::add(acc[l], v[l], k);
                    }
                    A best = acc[0];
                    int bi = 0;
#pragma unroll
                    for (int l = 1; l < D; ++l)
                        if (acc[l] < best) {
                            best = acc[l];
                            bi = l;
                        }
                    out[oo[j]] = C::store(best);
                    arg[oo[j]] = static_cast<uint8_t>(bi);
                    oo[j] += d0;
                }
            }
        }
    }
}

template <typename T, int D, int FC>
__device__ __forceinline__ void item_fixed(const TaskDev &tk, const unsigned char *stage, int lo,
                                           int g0, int g1, uint32_t k)
{
    switch (tk.F - tk.n_gi) {
    case 0: item_fixed_nr<T, D, FC, 0>(tk, stage, lo, g0, g1, k); break;
    case 1: item_fixed_nr<T, D, FC, 1>(tk, stage, lo, g0, g1, k); break;
    case 2: item_fixed_nr<T, D, FC, 2>(tk, stage, lo, g0, g1, k); break;
    default:
        if constexpr (FC <= 3) item_fixed_nr<T, D, FC, 3>(tk, stage, lo, g0, g1, k);
        else item_fixed_anyF<T, D>(tk, stage, lo, g0, g1, k);
        break;
    }
}

// Any domain size (runtime loop over x_i's values), at most FC inputs.
template <typename T, int FC>
__device__ __forceinline__ void item_anyD(const TaskDev &tk, const unsigned char *stage, int lo, int g0,
                                          int g1, uint32_t k)
{
    using C = Cost<T>;
    using A = typename C::acc;
    constexpr int SA = FC + 1;
    constexpr int SB = (FC + 3) / 4 * 4;
    const int F = tk.F, d = tk.d;
    int32_t b[SB];
    load_ints<SB>(tk.B + static_cast<int64_t>(lo) * SB, b);
    int32_t du[SA];
    load_ints<SA>(tk.A + static_cast<int64_t>(tk.G) * SA, du);
    const T *p[FC];
#pragma unroll
    for (int f = 0; f < FC; ++f) p[f] = (f < F) ? input_base<T>(tk.in[f], stage) + b[f] : nullptr;
    T *out = static_cast<T *>(tk.out);
    for (int g = g0; g < g1; ++g) {
        int32_t a[SA];
        load_ints<SA>(tk.A + static_cast<int64_t>(g) * SA, a);
        for (int u = 0; u < tk.R0; ++u) {
            const T *q[FC];
#pragma unroll
            for (int f = 0; f < FC; ++f) q[f] = (f < F) ? p[f] + (a[1 + f] + u * du[1 + f]) : nullptr;
            A best = A(0);
            int bi = 0;
            for (int l = 0; l < d; ++l) {
                A s = C::from(q[0][l]);
#pragma unroll
                for (int f = 1; f < FC; ++f)
                    if (f < F) s = C::add(s, q[f][l], k);
                if (l == 0 || s < best) {
                    best = s;
                    bi = l;
                }
            }
            const int o = a[0] + u * du[0] + lo;
            out[o] = C::store(best);
            tk.arg[o] = static_cast<uint8_t>(bi);
        }
    }
}

// Any domain size, any number of inputs.
template <typename T>
__device__ __forceinline__ void item_anyD_anyF(const TaskDev &tk, const unsigned char *stage, int lo,
                                               int g0, int g1, uint32_t k)
{
    using C = Cost<T>;
    using A = typename C::acc;
    const int F = tk.F, d = tk.d;
    const int32_t *Brow = tk.B + static_cast<int64_t>(lo) * tk.sb;
    const int32_t *du = tk.A + static_cast<int64_t>(tk.G) * tk.sa;
    T *out = static_cast<T *>(tk.out);
    for (int g = g0; g < g1; ++g) {
        const int32_t *Ar = tk.A + static_cast<int64_t>(g) * tk.sa;
        for (int u = 0; u < tk.R0; ++u) {
            A best = A(0);
            int bi = 0;
            for (int l = 0; l < d; ++l) {
                A s = A(0);
                for (int f = 0; f < F; ++f)
                    s = C::add(s, input_base<T>(tk.in[f], stage)[Ar[1 + f] + u * du[1 + f] + Brow[f] + l], k);
                if (l == 0 || s < best) {
                    best = s;
                    bi = l;
                }
            }
            const int o = Ar[0] + u * du[0] + lo;
            out[o] = C::store(best);
            tk.arg[o] = static_cast<uint8_t>(bi);
        }
    }
}

template <typename T, int D>
__device__ __forceinline__ void dispatch_f(const TaskDev &tk, int fc, const unsigned char *stage, int lo,
                                           int h0, int h1, uint32_t k)
{
    if constexpr (D == 0) {
        switch (fc) {
        case 0: item_anyD<T, 3>(tk, stage, lo, h0, h1, k); break;
        case 1: item_anyD<T, 7>(tk, stage, lo, h0, h1, k); break;
        default: item_anyD_anyF<T>(tk, stage, lo, h0, h1, k); break;
        }
    } else {
        switch (fc) {
        case 0: item_fixed<T, D, 3>(tk, stage, lo, h0, h1, k); break;
        case 1: item_fixed<T, D, 7>(tk, stage, lo, h0, h1, k); break;
        default: item_fixed_anyF<T, D>(tk, stage, lo, h0, h1, k); break;
        }
    }
}

template <typename T>
__device__ __forceinline__ void dispatch(const TaskDev &tk, const unsigned char *stage, int lo, int h0,
                                         int h1, uint32_t k)
{
    const int dc = tk.variant / kNumFClass, fc = tk.variant % kNumFClass;
    switch (dc) {
    case 1: dispatch_f<T, 2>(tk, fc, stage, lo, h0, h1, k); break;
    case 2: dispatch_f<T, 3>(tk, fc, stage, lo, h0, h1, k); break;
    case 3: dispatch_f<T, 4>(tk, fc, stage, lo, h0, h1, k); break;
    case 4: dispatch_f<T, 5>(tk, fc, stage, lo, h0, h1, k); break;
    case 5: dispatch_f<T, 6>(tk, fc, stage, lo, h0, h1, k); break;
    case 6: dispatch_f<T, 7>(tk, fc, stage, lo, h0, h1, k); break;
    case 7: dispatch_f<T, 8>(tk, fc, stage, lo, h0, h1, k); break;
    default: dispatch_f<T, 0>(tk, fc, stage, lo, h0, h1, k); break;
    }
}

// ------------------------------------------------------------- kernel
template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 2) util_kernel(const LaunchDev L)
{
    extern __shared__ __align__(128) unsigned char stage[];
    __shared__ uint64_t bar;
    __shared__ int s_item[2];
    __shared__ int s_staged;  // task whose tables are in shared memory, -1 = none

    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar, 1);
        s_staged = -1;
        s_item[0] = atomicAdd(L.counter, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    int it = 0;
    int item = s_item[0];
    while (item < L.total_items) {
        const int nb = (it + 1) & 1;
        if (tid == 0) s_item[nb] = atomicAdd(L.counter, 1);  // prefetch the next item

        // task of this item: last t with prefix[t] <= item
        int a = 0, b = L.n_tasks;
        while (b - a > 1) {
            const int mid = (a + b) >> 1;
            if (L.prefix[mid] <= item) a = mid;
            else b = mid;
        }
        const TaskDev tk = L.tasks[a];

        if (tk.stage_bytes > 0 && s_staged != a) {
            __syncthreads();  // every thread is done with the previous copies
            if (tid == 0) {
                fence_proxy_async();
                mbar_arrive_expect_tx(&bar, static_cast<uint32_t>(tk.stage_bytes));
                for (int f = 0; f < tk.F; ++f) {
                    const InDev in = tk.in[f];
                    if (in.stage_off >= 0)
                        tma_bulk_g2s(stage + in.stage_off, in.ptr, static_cast<uint32_t>(in.bytes16),
                                     &bar);
                }
                s_staged = a;
            }
            bool ok = mbar_wait_bounded(&bar, phase);
            if (__syncthreads_or(!ok)) {
                // give up on this launch: flag it, let the copies land (bounded), leave
                if (tid == 0) atomicExch(L.status, kStatusTimeout);
                mbar_wait_bounded(&bar, phase);
                return;
            }
            phase ^= 1u;
        }

        const int local = item - L.prefix[a];
        const int hr = local / tk.nlc;
        const int lc = local - hr * tk.nlc;
        const int h0 = hr * tk.hc;
        const int h1 = min(h0 + tk.hc, tk.G);
        const int lo = lc * blockDim.x + tid;
        if (lo < tk.P_lo) dispatch<T>(tk, stage, lo, h0, h1, L.top_k);

        __syncthreads();
        item = s_item[nb];
        ++it;
    }
}

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

// ------------------------------------------------------------- VALUE
__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Index of a term's table entry under the current assignment (warp-wide).
__device__ __forceinline__ long long term_index(const ValueDev &V, const ValueTerm &t,
                                                const unsigned char *sig, int lane)
{
    long long idx = 0;
    for (int j = lane; j < t.nv; j += 32)
        idx += static_cast<long long>(sig[V.vvars[t.var_off + j]]) * V.vstrides[t.var_off + j];
    return warp_sum_ll(idx);
}

// VALUE phase in one CTA: variables grouped by dependency level (a variable
// depends on the other variables of its bucket, all eliminated later), one
// warp per variable.  BE / DPOP read the stored argmin of the bucket
// function at the separator's assignment; MBE takes the first argmin of the
// sum of every function of the bucket.  Then the root constants are summed
// (the optimum or lower bound) and the Eq. 1 cost of the assignment is
// evaluated over the original functions.
template <typename T>
__global__ void __launch_bounds__(256) value_kernel(const ValueDev V)
{
    using C = Cost<T>;
    using A = typename C::acc;
    extern __shared__ unsigned char sig[];
    __shared__ double red[2][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int v = threadIdx.x; v < V.n; v += blockDim.x) sig[v] = 0;
    __syncthreads();
    for (int lev = 0; lev < V.n_levels; ++lev) {
        const int b = V.lev_off[lev], e = V.lev_off[lev + 1];
        for (int i = b + warp; i < e; i += nw) {
            const int v = V.vorder[i];
            const ValueVar vi = V.vinfo[v];
            int val = 0;
            if (vi.mode == 1) {
                const ValueTerm t = V.terms[vi.term_off];
                const long long idx = term_index(V, t, sig, lane);
                val = static_cast<const uint8_t *>(t.tab)[idx];
            } else if (vi.mode == 2) {
                constexpr int kMaxRuns = 8;  // domains up to 256 values
                A acc[kMaxRuns];
                for (int term = 0; term < vi.n_terms; ++term) {
                    const ValueTerm t = V.terms[vi.term_off + term];
                    const long long base = term_index(V, t, sig, lane);
                    const T *tab = static_cast<const T *>(t.tab) + base;
#pragma unroll
                    for (int r = 0; r < kMaxRuns; ++r) {
                        const int l = lane + 32 * r;
                        if (l < vi.d) acc[r] = term == 0 ? C::from(tab[l]) : C::add(acc[r], tab[l], V.top_k);
                    }
                }
                // first argmin over l: per lane, then across the warp
                A best = A(0);
                int bl = -1;
#pragma unroll
                for (int r = 0; r < kMaxRuns; ++r) {
                    const int l = lane + 32 * r;
                    if (l < vi.d && (bl < 0 || acc[r] < best)) {
                        best = acc[r];
                        bl = l;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const A ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
                    if (ol >= 0 && (bl < 0 || ob < best || (!(best < ob) && ol < bl))) {
                        best = ob;
                        bl = ol;
                    }
                }
                val = bl < 0 ? 0 : bl;
            }
            if (lane == 0) sig[v] = static_cast<unsigned char>(val);
        }
        __syncthreads();
    }
    // Eq. 1 cost of the assignment and the sum of the root constants
    double c = 0.0, rb = 0.0;
    for (int i = threadIdx.x; i < V.n_evals; i += blockDim.x) {
        const ValueTerm t = V.evals[i];
        long long idx = 0;
        for (int j = 0; j < t.nv; ++j)
            idx += static_cast<long long>(sig[V.vvars[t.var_off + j]]) * V.vstrides[t.var_off + j];
        c += static_cast<double>(static_cast<const T *>(t.tab)[idx]);
    }
    for (int i = threadIdx.x; i < V.n_roots; i += blockDim.x)
        rb += static_cast<double>(static_cast<const T *>(V.roots[i])[0]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        rb += __shfl_xor_sync(0xffffffffu, rb, o);
    }
    if (lane == 0) {
        red[0][warp] = c;
        red[1][warp] = rb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tc = V.const_sum, tb = V.const_sum;
        for (int w = 0; w < nw; ++w) {
            tc += red[0][w];
            tb += red[1][w];
        }
        if (!V.is_float) {
            const double k = static_cast<double>(V.top_k);
            tc = tc > k ? k : tc;
            tb = tb > k ? k : tb;
        }
        V.result[0] = tb;
        V.result[1] = tc;
    }
    for (int v = threadIdx.x; v < V.n; v += blockDim.x) V.sigma[v] = sig[v];
}

// -------------------------------------------------------- host launchers
cudaError_t launch_util(const LaunchDev &L, int cost_type, int grid, int threads, int smem,
                        cudaStream_t s)
{
    if (cost_type == 1)
        util_kernel<float><<<grid, threads, smem, s>>>(L);
    else
        util_kernel<int32_t><<<grid, threads, smem, s>>>(L);
    return cudaGetLastError();
}

int util_max_blocks_per_sm(int cost_type, int threads, int smem)
{
    int nb = 0;
    cudaError_t e = cost_type == 1
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<float>, threads, smem)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, util_kernel<int32_t>, threads, smem);
    if (e != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
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

cudaError_t launch_value(const ValueDev &V, int cost_type, int smem, cudaStream_t s)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cost_type == 1
            ? cudaFuncSetAttribute(value_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
            : cudaFuncSetAttribute(value_kernel<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    if (cost_type == 1)
        value_kernel<float><<<1, 256, smem, s>>>(V);
    else
        value_kernel<int32_t><<<1, 256, smem, s>>>(V);
    return cudaGetLastError();
}

}  // namespace gpube
