// UTIL kernel templates for sm_103a; instantiated per cost type and
// elimination operator in util_kernel_i32.cu, util_kernel_f32.cu and
// util_kernel_sum.cu (the VALUE kernels are in value_kernel.cuh).
#pragma once
// UTIL-table kernels for sm_103a.
//
// One kernel computes every bucket function of Algorithms 1-2 (and DPOP's
// UTIL messages): for each separator row r and each value l of the
// eliminated variable x_i it gathers one entry of every input table, sums
// them (saturating at the top cost for integer WCSPs, Section 2; fp32 for
// -log p costs, Section 3), and keeps the minimum and first argmin over l
// (or, for the sum-product problem, -log of the sum over l of exp(-sum)).
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

// Raise an mbarrier phase's expected transaction bytes without arriving.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
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

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: false once limit_ns has passed (or the
// iteration backstop is reached) without the phase completing.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitNs)
{
    const unsigned long long t0 = global_ns();
    for (int i = 0; i < kMaxSpin; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// Per-thread asynchronous global -> shared copies (completion tracked per
// thread by commit / wait groups).
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src)
{
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES)
                     : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ------------------------------------------------------------ cost ops
template <typename T> struct Cost;

// Integer WCSP costs in [0, k]: sums saturate at k (k means "not allowed").
// Both operands are <= k < 2^31, so their uint32 sum cannot wrap.
template <> struct Cost<int32_t> {
    using val = int32_t;
    using acc = uint32_t;
    static constexpr bool kSum = false;
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
    using val = float;
    using acc = float;
    static constexpr bool kSum = false;
    static __device__ __forceinline__ acc from(float v) { return v; }
    static __device__ __forceinline__ acc add(acc a, float v, uint32_t) { return a + v; }
    static __device__ __forceinline__ float store(acc a) { return a; }
};

// Sum-product in the -log domain (weighted counting, partition function):
// the terms add as fp32 -log weights, and x_i is eliminated by
// -log sum_l exp(-s_l) instead of min_l s_l.  No argmin is written.
struct SumProduct : Cost<float> {
    static constexpr bool kSum = true;
};

constexpr float kInfF = __builtin_huge_valf();

__device__ __forceinline__ float min_of(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ uint32_t min_of(uint32_t a, uint32_t b) { return min(a, b); }
// Factored sum-product rows below this sum of products are recomputed from
// their raw terms (fp32 keeps full relative precision well above it).
constexpr float kSfTiny = 1e-20f;

// Elimination of one row's D sums: the first minimum and its index; for the
// sum-product, -log sum exp(-acc[l]) taken relative to that minimum (every
// exponent <= 0, one term is 1), +inf when every term is +inf.  Where no
// argmin is wanted (ARG = false, or the sum-product) the minimum is taken by
// min instructions alone (the sums hold no NaN: costs are >= 0 or +inf).
template <typename C, int D, bool ARG = true>
__device__ __forceinline__ typename C::acc reduce_run(const typename C::acc (&acc)[D], int &bi)
{
    using A = typename C::acc;
    A best = acc[0];
    bi = 0;
    if constexpr (ARG && !C::kSum) {
#pragma unroll
        for (int l = 1; l < D; ++l)
            if (acc[l] < best) {
                best = acc[l];
                bi = l;
            }
    } else {
#pragma unroll
        for (int l = 1; l < D; ++l) best = min_of(best, acc[l]);
    }
    if constexpr (C::kSum) {
        if (best < kInfF) {
            float t = 0.f;
#pragma unroll
            for (int l = 0; l < D; ++l) t += __expf(best - acc[l]);
            best -= __logf(t);
        }
    }
    return best;
}

// The same elimination for values that arrive one at a time (runtime domain
// size) keeps a running minimum best and, for the sum-product, the running
// sum t of exp(best - s_l), rescaled whenever the minimum drops; lse_value
// turns the pair into -log sum exp(-s_l).
__device__ __forceinline__ float lse_value(float best, float t)
{
    return best < kInfF ? best - __logf(t) : best;
}

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

// A thread's run of D values stored in shared memory as D*4/CH chunks of CH
// bytes laid out [chunk][thread] (chunk c of thread t at base + (c*NT + t)*CH,
// base a 32-bit shared-window address): one vector access per chunk keeps a
// warp's accesses conflict-free.
template <int D, int CH, typename V>
__device__ __forceinline__ void slot_load(uint32_t base, int NT, int tid, V (&v)[D])
{
    static_assert(sizeof(V) == 4, "4-byte values");
#pragma unroll
    for (int c = 0; c < D * 4 / CH; ++c) {
        const uint32_t q = base + static_cast<uint32_t>((c * NT + tid) * CH);
        if constexpr (CH == 16) {
            uint32_t x0, x1, x2, x3;
            asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(x0), "=r"(x1), "=r"(x2), "=r"(x3)
                         : "r"(q)
                         : "memory");
            v[4 * c + 0] = __builtin_bit_cast(V, x0);
            v[4 * c + 1] = __builtin_bit_cast(V, x1);
            v[4 * c + 2] = __builtin_bit_cast(V, x2);
            v[4 * c + 3] = __builtin_bit_cast(V, x3);
        } else if constexpr (CH == 8) {
            uint32_t x0, x1;
            asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(x0), "=r"(x1) : "r"(q) : "memory");
            v[2 * c + 0] = __builtin_bit_cast(V, x0);
            v[2 * c + 1] = __builtin_bit_cast(V, x1);
        } else {
            uint32_t x0;
            asm volatile("ld.shared.b32 %0, [%1];" : "=r"(x0) : "r"(q) : "memory");
            v[c] = __builtin_bit_cast(V, x0);
        }
    }
}

template <int D, int CH, typename V>
__device__ __forceinline__ void slot_store(uint32_t base, int NT, int tid, const V (&v)[D])
{
#pragma unroll
    for (int c = 0; c < D * 4 / CH; ++c) {
        const uint32_t q = base + static_cast<uint32_t>((c * NT + tid) * CH);
        if constexpr (CH == 16) {
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(q), "r"(__builtin_bit_cast(uint32_t, v[4 * c])),
                         "r"(__builtin_bit_cast(uint32_t, v[4 * c + 1])), "r"(__builtin_bit_cast(uint32_t, v[4 * c + 2])),
                         "r"(__builtin_bit_cast(uint32_t, v[4 * c + 3]))
                         : "memory");
        } else if constexpr (CH == 8) {
            asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(q), "r"(__builtin_bit_cast(uint32_t, v[2 * c])),
                         "r"(__builtin_bit_cast(uint32_t, v[2 * c + 1]))
                         : "memory");
        } else {
            asm volatile("st.shared.b32 [%0], %1;" ::"r"(q), "r"(__builtin_bit_cast(uint32_t, v[c])) : "memory");
        }
    }
}

// Four ints from a 32-bit shared-window address (a uniform A row).
__device__ __forceinline__ void lds_int4(uint32_t q, int32_t (&a)[4])
{
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(q)
                 : "memory");
}

__device__ __forceinline__ int32_t lds_int(uint32_t q)
{
    int32_t x;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(x) : "r"(q) : "memory");
    return x;
}

// Asynchronous copy into a 32-bit shared-window address.
template <int BYTES>
__device__ __forceinline__ void cp_async_s(uint32_t dst, const void *src)
{
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(BYTES) : "memory");
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

// Fixed domain D, any number of inputs (offsets read from the tables per
// input): the lo-only inputs are summed once per item, the group inputs once
// per group, and each row adds only the inputs that mention the fastest hi
// digit u.
template <typename C, int D, bool WA = true>
__device__ __noinline__ void item_fixed_anyF(const TaskDev *__restrict__ tkp, const unsigned char *stage, int lo,
                                                int g0, int g1, uint32_t k)
{
    const TaskDev tk = *tkp;
    using T = typename C::val;
    using A = typename C::acc;
    const int F = tk.F, nlo = tk.n_lo, ngi = tk.n_gi;
    const int32_t *Brow = tk.B + static_cast<int64_t>(lo) * tk.sb;
    const int32_t *du = tk.A + static_cast<int64_t>(tk.G) * tk.sa;
    T *out = static_cast<T *>(tk.out);
    A base[D];
#pragma unroll
    for (int l = 0; l < D; ++l) base[l] = A(0);
    for (int f = 0; f < nlo; ++f) {
        T v[D];
        load_run<D>(input_base<T>(tk.in[f], stage) + Brow[f], v);
#pragma unroll
        for (int l = 0; l < D; ++l) base[l] = C::add(base[l], v[l], k);
    }
    for (int g = g0; g < g1; ++g) {
        const int32_t *Ar = tk.A + static_cast<int64_t>(g) * tk.sa;
        A pre[D];
#pragma unroll
        for (int l = 0; l < D; ++l) pre[l] = base[l];
        for (int f = nlo; f < ngi; ++f) {
            T v[D];
            load_run<D>(input_base<T>(tk.in[f], stage) + (Ar[1 + f] + Brow[f]), v);
#pragma unroll
            for (int l = 0; l < D; ++l) pre[l] = C::add(pre[l], v[l], k);
        }
        for (int u = 0; u < tk.R0; ++u) {
            A acc[D];
#pragma unroll
            for (int l = 0; l < D; ++l) acc[l] = pre[l];
            for (int f = ngi; f < F; ++f) {
                T v[D];
                load_run<D>(input_base<T>(tk.in[f], stage) + (Ar[1 + f] + u * du[1 + f] + Brow[f]), v);
#pragma unroll
                for (int l = 0; l < D; ++l) acc[l] = C::add(acc[l], v[l], k);
            }
            int bi;
            const A best = reduce_run<C, D, WA>(acc, bi);
            const int o = Ar[0] + u * du[0] + lo;
            out[o] = C::store(best);
            if constexpr (!C::kSum && WA) tk.arg[o] = static_cast<uint8_t>(bi);
        }
    }
}

// Fixed domain D, more than 7 inputs, at most 8 of them group inputs and at
// most 2 per-row inputs (the shape of the hub buckets of scale-free graphs:
// many small tables on the hub and the separator): the base pointers of the
// group and per-row inputs, their row lo included, stay in registers for the
// whole item, so a group costs one A-row entry and one run per group input and
// a row one run per per-row input, with no descriptor loads.
template <typename C, int D>
__device__ __noinline__ void item_fixed_manyF(const TaskDev *__restrict__ tkp, const unsigned char *stage, int lo,
                                              int g0, int g1, uint32_t k)
{
    const TaskDev tk = *tkp;
    using T = typename C::val;
    using A = typename C::acc;
    constexpr int GMAX = 8, RMAX = 2;
    const int F = tk.F, nlo = tk.n_lo, ngi = tk.n_gi, ng = ngi - nlo, nr = F - ngi;
    const int32_t *Brow = tk.B + static_cast<int64_t>(lo) * tk.sb;
    const int32_t *du = tk.A + static_cast<int64_t>(tk.G) * tk.sa;
    T *out = static_cast<T *>(tk.out);
    A base[D];
#pragma unroll
    for (int l = 0; l < D; ++l) base[l] = A(0);
    for (int f = 0; f < nlo; ++f) {
        T v[D];
        load_run<D>(input_base<T>(tk.in[f], stage) + Brow[f], v);
#pragma unroll
        for (int l = 0; l < D; ++l) base[l] = C::add(base[l], v[l], k);
    }
    const T *gp[GMAX];
#pragma unroll
    for (int i = 0; i < GMAX; ++i) gp[i] = i < ng ? input_base<T>(tk.in[nlo + i], stage) + Brow[nlo + i] : nullptr;
    const T *rp[RMAX];
    int32_t dr[RMAX];
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
        rp[r] = r < nr ? input_base<T>(tk.in[ngi + r], stage) + Brow[ngi + r] : nullptr;
        dr[r] = r < nr ? du[1 + ngi + r] : 0;
    }
    for (int g = g0; g < g1; ++g) {
        const int32_t *Ar = tk.A + static_cast<int64_t>(g) * tk.sa;
        A pre[D];
#pragma unroll
        for (int l = 0; l < D; ++l) pre[l] = base[l];
#pragma unroll
        for (int i = 0; i < GMAX; ++i) {
            if (i >= ng) break;
            T v[D];
            load_run<D>(gp[i] + Ar[1 + nlo + i], v);
#pragma unroll
            for (int l = 0; l < D; ++l) pre[l] = C::add(pre[l], v[l], k);
        }
        int32_t o = Ar[0] + lo;
        int32_t ro[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; ++r) ro[r] = r < nr ? Ar[1 + ngi + r] : 0;
        for (int u = 0; u < tk.R0; ++u) {
            A acc[D];
#pragma unroll
            for (int l = 0; l < D; ++l) acc[l] = pre[l];
#pragma unroll
            for (int r = 0; r < RMAX; ++r) {
                if (r >= nr) break;
                T v[D];
                load_run<D>(rp[r] + ro[r], v);
                ro[r] += dr[r];
#pragma unroll
                for (int l = 0; l < D; ++l) acc[l] = C::add(acc[l], v[l], k);
            }
            int bi;
            const A best = reduce_run<C, D>(acc, bi);
            out[o] = C::store(best);
            if constexpr (!C::kSum) tk.arg[o] = static_cast<uint8_t>(bi);
            o += du[0];
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
// loads, the adds, the argmin and two stores.  U > 0: the radix R0 of u is
// U, and the per-row runs of all U rows of the NG groups are loaded before
// any of them is summed (U x NG x NR loads in flight per thread).  WA =
// false: a variant that writes no argmin table (for tasks whose arg is null).
template <typename C, int D, int FC, int NR, int U = 0, bool WA = true>
__device__ __noinline__ void item_fixed_nr(const TaskDev *__restrict__ tkp, const unsigned char *stage, int lo, int g0,
                                              int g1, uint32_t k)
{
    const TaskDev tk = *tkp;
    using T = typename C::val;
    using A = typename C::acc;
    constexpr int SA = FC + 1;
    constexpr int SB = (FC + 3) / 4 * 4;
    constexpr int NG = (FC <= 3 && D <= 4) ? 2 : 1;
    constexpr int R = NR > 0 ? NR : 1;
    const int nlo = tk.n_lo, ngi = tk.n_gi, R0 = tk.R0;
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
            // (inputs [nlo, ngi); the unrolled loop branches past the rest)
#pragma unroll
            for (int f = 0; f < FC; ++f) {
                if (f >= ngi) break;
                if (f >= nlo) {
                    T x[NG][D];
#pragma unroll
                    for (int j = 0; j < NG; ++j) load_run<D>(gp[f] + a[j][1 + f], x[j]);
#pragma unroll
                    for (int j = 0; j < NG; ++j)
#pragma unroll
                        for (int l = 0; l < D; ++l) pre[j][l] = C::add(pre[j][l], x[j][l], k);
                }
            }
#pragma unroll
            for (int j = 0; j < NG; ++j) {
                oo[j] = a[j][0] + lo;
                // the per-row inputs' offsets of the group, read at their column
                // of the A row (already in L1) rather than selected out of the
                // registers by the runtime input index
                const int32_t *ar = tk.A + static_cast<int64_t>(g + j < g1 ? g + j : g) * SA + 1 + ngi;
#pragma unroll
                for (int r = 0; r < NR; ++r) ro[j][r] = ar[r];
            }
        }
        const int nj = (g + 1 < g1) ? NG : 1;
        if constexpr (U > 0 && NR > 0) {
            T v[U][NG][NR][D];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int j = 0; j < NG; ++j)
#pragma unroll
                    for (int r = 0; r < NR; ++r)
                        if (j < nj) load_run<D>(rp[r] + (ro[j][r] + u * dr[r]), v[u][j][r]);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int j = 0; j < NG; ++j)
                    if (j < nj) {
                        A acc[D];
#pragma unroll
                        for (int l = 0; l < D; ++l) acc[l] = pre[j][l];
#pragma unroll
                        for (int r = 0; r < NR; ++r)
#pragma unroll
                            for (int l = 0; l < D; ++l) acc[l] = C::add(acc[l], v[u][j][r][l], k);
                        int bi;
                        const A best = reduce_run<C, D, WA>(acc, bi);
                        const int32_t o = oo[j] + u * d0;
                        out[o] = C::store(best);
                        if constexpr (!C::kSum && WA) arg[o] = static_cast<uint8_t>(bi);
                    }
        } else {
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
                        int bi;
                        const A best = reduce_run<C, D, WA>(acc, bi);
                        out[oo[j]] = C::store(best);
                        if constexpr (!C::kSum && WA) arg[oo[j]] = static_cast<uint8_t>(bi);
                        oo[j] += d0;
                    }
                }
            }
        }
    }
}

// Same item, when exactly one input is a group input and lives in global
// memory (the usual large child bucket function): its run for group g + KP
// is copied to this thread's shared-memory slot by cp.async while group g is
// processed, so KP loads per thread are in flight without holding
// registers.  Slot layout [slot][chunk][thread] keeps the reads conflict-free.
//
// FOLD (R0 <= 4): the inputs whose only hi digit is u are added, once per
// item, into one partial sum per value of u, so such rows need no load.
// NRG counts the remaining per-row inputs.  With no per-row input a row sums
// two terms (partial sum + group run, each <= k, no uint32 wrap), so the
// saturation is applied once, after the min: if the minimum reaches k every
// clamped entry equals k and the first argmin is 0.
// U > 0: the radix R0 of u is U (rows unrolled, the per-u partial sums held
// in registers); U = 0: any R0 <= 4 (partial sums read from shared memory).
// PK (integer costs whose sums stay below the top cost and 2^30, D <= 4): the
// partial sums are kept as keys (s << 2 | l) and the group run as (x << 2),
// so a row's sums are D adds of keys, its minimum and first argmin one
// unsigned min over them (equal sums: the lower l has the lower key), and no
// saturation is needed.  WA = false: no argmin table is written.
template <typename C, int D, int NRG, bool FOLD, int U = 0, bool PK = false, bool WA = true>
__device__ __noinline__ void item_pipe(const TaskDev *__restrict__ tkp, const unsigned char *stage, unsigned char *pipe,
                                          const int32_t *arows, int lo, int g0, int g1, uint32_t k)
{
    const TaskDev tk = *tkp;
    using T = typename C::val;
    using A = typename C::acc;
    constexpr bool kInt = std::is_same<T, int32_t>::value;
    static_assert(!PK || (kInt && FOLD && NRG == 0 && U > 0 && D <= 4), "packed keys: integer rows of two terms");
    constexpr int SA = 4, SB = 4, UMAX = 4;  // at most 3 inputs: A and B rows of 4 ints
    constexpr int R = NRG > 0 ? NRG : 1;
    constexpr int CH = (D % 4 == 0) ? 16 : (D % 2 == 0) ? 8 : 4;  // bytes per copy
    constexpr int NCH = D * 4 / CH;                                  // copies per run
    // groups in flight (pipe_depth(D)); packed-key rows hold the per-u
    // partial sums in registers once the prologue has read them back, and
    // their four shared-memory slots become four more pipeline slots
    constexpr int KP = (D <= 4 ? kPipeSmall : kPipe) + (PK ? 4 : 0);
    const int NT = blockDim.x, tid = threadIdx.x;
    const int nlo = tk.n_lo, ngi = tk.n_gi, R0 = tk.R0;
    const int rg0 = FOLD ? tk.n_uo : ngi;  // first general per-row input
    const int32_t *Brow = tk.B + static_cast<int64_t>(lo) * SB;
    const int32_t *du = tk.A + static_cast<int64_t>(tk.G) * SA;
    A base[D];
#pragma unroll
    for (int l = 0; l < D; ++l) base[l] = A(0);
    for (int f = 0; f < nlo; ++f) {
        T v[D];
        load_run<D>(input_base<T>(tk.in[f], stage) + Brow[f], v);
#pragma unroll
        for (int l = 0; l < D; ++l) base[l] = C::add(base[l], v[l], k);
    }
    // shared-memory areas of this thread: the pipeline slots (group runs),
    // the slots' A rows, and the per-u partial sums, each laid out
    // [index][chunk][thread] so that the 16-byte reads are conflict-free
    const uint32_t pipe_s = smem_addr(pipe);
    // (PK: the partial sums occupy the last four pipeline slots until they
    // are read back into registers)
    const uint32_t bus_s = pipe_s + static_cast<uint32_t>((PK ? KP - 4 : KP) * NCH * NT * CH);
    const uint32_t arows_s = smem_addr(arows);
    A bur[U ? U : 1][D];
    // SF: sum-product rows of two terms with the radix of u fixed.  Because
    // exp(-(b_l + x_l)) = exp(-b_l) exp(-x_l), each partial sum b (once per
    // item) and each group run x (once per group, shared by its U rows) is
    // turned into its minimum and the exp of its offsets from it; a row is
    // then D multiply-adds and one log: -log sum = mb + mx - log sum_l
    // eb_l ex_l.  When that sum is tiny (the two minima at different l, far
    // apart; or +inf terms) the row is recomputed from the raw terms.
    constexpr bool SF = C::kSum && FOLD && NRG == 0 && U > 0;
    float mbu[SF ? U : 1];
    int32_t zdep = 0;
    if constexpr (FOLD) {
        for (int u = 0; u < R0; ++u) {
            A bu[D];
#pragma unroll
            for (int l = 0; l < D; ++l) bu[l] = base[l];
            for (int f = ngi; f < tk.n_uo; ++f) {
                T v[D];
                load_run<D>(input_base<T>(tk.in[f], stage) + (Brow[f] + u * du[1 + f]), v);
#pragma unroll
                for (int l = 0; l < D; ++l) bu[l] = C::add(bu[l], v[l], k);
            }
            slot_store<D, CH>(bus_s + static_cast<uint32_t>(u * NCH * NT * CH), NT, tid, bu);
        }
        if constexpr (U > 0) {
#pragma unroll
            for (int u = 0; u < U; ++u) slot_load<D, CH>(bus_s + static_cast<uint32_t>(u * NCH * NT * CH), NT, tid, bur[u]);
        }
        if constexpr (PK) {
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int l = 0; l < D; ++l) bur[u][l] = (bur[u][l] << 2) | static_cast<uint32_t>(l);
            // a zero that depends on every value read back: the copies into
            // the slots that held the partial sums take it in their address,
            // so they are issued only after those shared loads returned
            uint32_t all = 0;
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int l = 0; l < D; ++l) all |= bur[u][l];
            asm volatile("and.b32 %0, %1, 0;" : "=r"(zdep) : "r"(all));
        }
        if constexpr (SF) {
            // partial sums as (minimum, exp(minimum - b_l)); the raw values stay
            // in the shared-memory slots for the rows that need them
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float m = bur[u][0];
#pragma unroll
                for (int l = 1; l < D; ++l) m = fminf(m, bur[u][l]);
                mbu[u] = m;
#pragma unroll
                for (int l = 0; l < D; ++l) bur[u][l] = m < kInfF ? __expf(m - bur[u][l]) : 0.f;
            }
        }
    }
    const int gf = nlo;  // the group input
    const T *gp = reinterpret_cast<const T *>(tk.in[gf].ptr) + Brow[gf];
    const T *rp[R];
    int32_t dr[R];
#pragma unroll
    for (int r = 0; r < NRG; ++r) {
        rp[r] = input_base<T>(tk.in[rg0 + r], stage) + Brow[rg0 + r];
        dr[r] = du[1 + rg0 + r];
    }
    const int32_t d0 = du[0];
    T *out = static_cast<T *>(tk.out);
    uint8_t *arg = tk.arg;
    // the item's A rows are in shared memory (arows[(g - g0) * SA + slot]);
    // each pipeline slot holds, per thread, one group run
    auto issue = [&](int g, int slot, int32_t zoff = 0) {
        if (g < g1) {
            const T *src = gp + (lds_int(arows_s + static_cast<uint32_t>(((g - g0) * SA + 1 + gf) * 4)) + zoff);
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                cp_async_s<CH>(pipe_s + static_cast<uint32_t>(((slot * NCH + c) * NT + tid) * CH),
                               reinterpret_cast<const unsigned char *>(src) + c * CH);
        }
        cp_async_commit();
    };
    // minimum (or -log sum exp) and first argmin of one row's sums, written
    auto reduce_store = [&](A (&acc)[D], int32_t o) {
        A best = acc[0];
        int bi = 0;
        if constexpr (WA && !C::kSum) {
#pragma unroll
            for (int l = 1; l < D; ++l)
                if (acc[l] < best) {
                    best = acc[l];
                    bi = l;
                }
        } else {
#pragma unroll
            for (int l = 1; l < D; ++l) best = min_of(best, acc[l]);
        }
        if constexpr (C::kSum) {
            if (best < kInfF) {
                float t = 0.f;
#pragma unroll
                for (int l = 0; l < D; ++l) t += __expf(best - acc[l]);
                best -= __logf(t);
            }
        }
        if constexpr (NRG == 0 && kInt) {
            if (best >= k) {
                best = k;
                bi = 0;
            }
        }
        out[o] = C::store(best);
        if constexpr (!C::kSum && WA) arg[o] = static_cast<uint8_t>(bi);
    };
    // one output row: b (partial sum) + x (group run) + the NRG per-row runs
    auto row = [&](const A (&b)[D], const T (&x)[D], int32_t (&ro)[R], int32_t o) {
        A acc[D];
        if constexpr (NRG == 0 && kInt) {
#pragma unroll
            for (int l = 0; l < D; ++l) acc[l] = b[l] + static_cast<A>(x[l]);  // <= 2k, no wrap
        } else {
#pragma unroll
            for (int l = 0; l < D; ++l) acc[l] = C::add(b[l], x[l], k);
#pragma unroll
            for (int r = 0; r < NRG; ++r) {
                T v[D];
                load_run<D>(rp[r] + ro[r], v);
                ro[r] += dr[r];
#pragma unroll
                for (int l = 0; l < D; ++l) acc[l] = C::add(acc[l], v[l], k);
            }
        }
        reduce_store(acc, o);
    };
#pragma unroll
    for (int s = 0; s < KP; ++s) issue(g0 + s, s, (PK && s >= KP - 4) ? zdep : 0);
    int slot = 0;
    for (int g = g0; g < g1; ++g) {
        cp_async_wait<KP - 1>();
        int32_t a[SA];
        lds_int4(arows_s + static_cast<uint32_t>((g - g0) * SA * 4), a);
        T x[D];
        slot_load<D, CH>(pipe_s + static_cast<uint32_t>(slot * NCH * NT * CH), NT, tid, x);
        int32_t ro[R];
#pragma unroll
        for (int r = 0; r < NRG; ++r)  // the per-row inputs' offsets, at their column of the A row
            ro[r] = lds_int(arows_s + static_cast<uint32_t>(((g - g0) * SA + 1 + rg0 + r) * 4));
        int32_t o = a[0] + lo;
        if constexpr (SF) {
            float mx = x[0];
#pragma unroll
            for (int l = 1; l < D; ++l) mx = fminf(mx, x[l]);
            float ex[D];
#pragma unroll
            for (int l = 0; l < D; ++l) ex[l] = mx < kInfF ? __expf(mx - x[l]) : 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float t = bur[u][0] * ex[0];
#pragma unroll
                for (int l = 1; l < D; ++l) t = fmaf(bur[u][l], ex[l], t);
                float h;
                if (t >= kSfTiny) {
                    h = (mbu[u] + mx) - __logf(t);
                } else {
                    A bu[D], acc[D];
                    slot_load<D, CH>(bus_s + static_cast<uint32_t>(u * NCH * NT * CH), NT, tid, bu);
#pragma unroll
                    for (int l = 0; l < D; ++l) acc[l] = bu[l] + x[l];
                    int bi;
                    h = reduce_run<C, D>(acc, bi);
                }
                out[o] = h;
                o += d0;
            }
            issue(g + KP, slot);  // the slot's data has been consumed
        } else if constexpr (PK) {
            uint32_t xs[D];
#pragma unroll
            for (int l = 0; l < D; ++l) xs[l] = static_cast<uint32_t>(x[l]) << 2;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t m = bur[u][0] + xs[0];
#pragma unroll
                for (int l = 1; l < D; ++l) m = min(m, bur[u][l] + xs[l]);
                out[o] = static_cast<T>(m >> 2);
                if constexpr (WA) arg[o] = static_cast<uint8_t>(m & 3u);
                o += d0;
            }
            issue(g + KP, slot);  // the slot's data has been consumed
        } else if constexpr (FOLD && U > 0 && NRG > 0) {
            // the per-row runs of all U rows are loaded before any row is
            // summed (stores to the output would otherwise keep later loads
            // behind them)
            T rv[U][R][D];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int r = 0; r < NRG; ++r) load_run<D>(rp[r] + (ro[r] + u * dr[r]), rv[u][r]);
            issue(g + KP, slot);  // x is in registers
#pragma unroll
            for (int u = 0; u < U; ++u) {
                A acc[D];
#pragma unroll
                for (int l = 0; l < D; ++l) acc[l] = C::add(bur[u][l], x[l], k);
#pragma unroll
                for (int r = 0; r < NRG; ++r)
#pragma unroll
                    for (int l = 0; l < D; ++l) acc[l] = C::add(acc[l], rv[u][r][l], k);
                reduce_store(acc, o);
                o += d0;
            }
        } else if constexpr (FOLD) {
#pragma unroll
            for (int u = 0; u < (U ? U : UMAX); ++u)
                if (U || u < R0) {
                    A bu[D];
                    if constexpr (U > 0) {
#pragma unroll
                        for (int l = 0; l < D; ++l) bu[l] = bur[U > 0 ? u : 0][l];
                    } else {
                        slot_load<D, CH>(bus_s + static_cast<uint32_t>(u * NCH * NT * CH), NT, tid, bu);
                    }
                    row(bu, x, ro, o);
                    o += d0;
                }
            issue(g + KP, slot);  // the slot's data has been consumed
        } else {
            A pre[D];
#pragma unroll
            for (int l = 0; l < D; ++l) pre[l] = C::add(base[l], x[l], k);
            issue(g + KP, slot);
            T zero[D];
#pragma unroll
            for (int l = 0; l < D; ++l) zero[l] = T(0);
            for (int u = 0; u < R0; ++u) {
                row(pre, zero, ro, o);
                o += d0;
            }
        }
        slot = (slot + 1 == KP) ? 0 : slot + 1;
    }
    cp_async_wait<0>();
}

// Four consecutive output rows per thread: rows lo4 .. lo4 + 3 of each hi
// value (P_lo % 4 == 0, so the four share their hi digits), fixed domain
// D of 2 or 3, at most 3 inputs.  The four costs go out as one 16-byte store and
// the four argmins as one 4-byte store.  How an input is read depends on how
// its offsets vary over the four rows (host-side classes):
//   bit f of tk.lin: its layout ends with the separator's lo digits and x_i,
//     so the four rows' runs are one contiguous, 16-byte aligned block of 4D
//     entries, read with vector loads;
//   bit f of tk.uni: it mentions none of the digits that vary within an
//     aligned block of four rows, so one run serves the four rows;
//   otherwise each row's run is read at its own offset from the B table
//     (L1-resident), so that no per-row offsets are held in registers.
// Inputs [0, n_gi) mention no u and are summed once per group, the others
// once per row.
template <typename C, int D, bool WA = true>
__device__ __noinline__ void item_v4(const TaskDev *__restrict__ tkp, const unsigned char *stage, int lo4, int g0,
                                     int g1, uint32_t k)
{
    const TaskDev tk = *tkp;
    using T = typename C::val;
    using A = typename C::acc;
    constexpr int FC = 3, SA = 4, SB = 4;
    const int F = tk.F, ngi = tk.n_gi, R0 = tk.R0, lin = tk.lin, uni = tk.uni;
    const int32_t *Brow = tk.B + static_cast<int64_t>(lo4) * SB;
    int32_t b0[SB];
    load_ints<SB>(Brow, b0);
    const T *ip[FC];
#pragma unroll
    for (int f = 0; f < FC; ++f) ip[f] = f < F ? input_base<T>(tk.in[f], stage) + b0[f] : nullptr;
    int32_t du[SA];
    load_ints<SA>(tk.A + static_cast<int64_t>(tk.G) * SA, du);
    T *out = static_cast<T *>(tk.out);
    uint8_t *arg = tk.arg;
    // the four rows' runs of input f at hi offset h
    auto runs = [&](int f, int32_t h, T (&v)[4][D]) {
        if ((lin >> f) & 1) {
            T w[4 * D];
            load_run<4 * D>(ip[f] + h, w);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int l = 0; l < D; ++l) v[i][l] = w[i * D + l];
        } else if ((uni >> f) & 1) {
            load_run<D>(ip[f] + h, v[0]);
#pragma unroll
            for (int i = 1; i < 4; ++i)
#pragma unroll
                for (int l = 0; l < D; ++l) v[i][l] = v[0][l];
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) load_run<D>(ip[f] + (h + (Brow[i * SB + f] - b0[f])), v[i]);
        }
    };
    for (int g = g0; g < g1; ++g) {
        int32_t a[SA];
        load_ints<SA>(tk.A + static_cast<int64_t>(g) * SA, a);
        A pre[4][D];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int l = 0; l < D; ++l) pre[i][l] = A(0);
#pragma unroll
        for (int f = 0; f < FC; ++f) {  // lo-only and group inputs (the unrolled loop branches past the rest)
            if (f >= ngi) break;
            T v[4][D];
            runs(f, a[1 + f], v);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int l = 0; l < D; ++l) pre[i][l] = C::add(pre[i][l], v[i][l], k);
        }
        int32_t o = a[0] + lo4;
        int32_t h[FC];
#pragma unroll
        for (int f = 0; f < FC; ++f) h[f] = a[1 + f];
        for (int u = 0; u < R0; ++u) {
            A acc[4][D];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int l = 0; l < D; ++l) acc[i][l] = pre[i][l];
#pragma unroll
            for (int f = 0; f < FC; ++f) {  // per-row inputs
                if (f >= F) break;
                if (f < ngi) continue;
                T v[4][D];
                runs(f, h[f], v);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int l = 0; l < D; ++l) acc[i][l] = C::add(acc[i][l], v[i][l], k);
            }
            T best[4];
            uint32_t bi = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int bb;
                best[i] = C::store(reduce_run<C, D, WA>(acc[i], bb));
                bi |= static_cast<uint32_t>(bb) << (8 * i);
            }
            using V4 = typename std::conditional<std::is_same<T, float>::value, float4, int4>::type;
            *reinterpret_cast<V4 *>(out + o) = V4{best[0], best[1], best[2], best[3]};
            if constexpr (!C::kSum && WA) *reinterpret_cast<uint32_t *>(arg + o) = bi;
            o += du[0];
#pragma unroll
            for (int f = 0; f < FC; ++f) h[f] += du[1 + f];
        }
    }
}

template <typename C, int D, int FC, bool WA = true>
__device__ __forceinline__ void item_fixed(const TaskDev *__restrict__ tkp, const TaskDev &tk,
                                           const unsigned char *stage, unsigned char *pipe, const int32_t *arows,
                                           int lo, int g0, int g1, uint32_t k)
{
    if constexpr (FC <= 3 && D <= 3) {
        if (tk.v4) {
            item_v4<C, D, WA>(tkp, stage, lo, g0, g1, k);
            return;
        }
    }
    if constexpr (FC <= 3 && D <= 8) {  // the host pipelines domains up to 8
        if (tk.pipe) {
            if (tk.R0 <= 4) {
                switch (tk.F - tk.n_uo) {
                case 0:  // the radix of u as a template constant: unrolled rows, partial sums in registers
                    if constexpr (std::is_same<C, Cost<int32_t>>::value && D <= 4) {
                        if (tk.nosat && tk.R0 >= 2) {  // sums below the top cost: packed keys
                            if (tk.R0 == 4) item_pipe<C, D, 0, true, 4, true, WA>(tkp, stage, pipe, arows, lo, g0, g1, k);
                            else if (tk.R0 == 3) item_pipe<C, D, 0, true, 3, true, WA>(tkp, stage, pipe, arows, lo, g0, g1, k);
                            else item_pipe<C, D, 0, true, 2, true, WA>(tkp, stage, pipe, arows, lo, g0, g1, k);
                            break;
                        }
                    }
                    if (tk.R0 == 4) item_pipe<C, D, 0, true, 4, false, WA>(tkp, stage, pipe, arows, lo, g0, g1, k);
                    else if (tk.R0 == 3) item_pipe<C, D, 0, true, 3, false, WA>(tkp, stage, pipe, arows, lo, g0, g1, k);
                    else if (tk.R0 == 2) item_pipe<C, D, 0, true, 2, false, WA>(tkp, stage, pipe, arows, lo, g0, g1, k);
                    else item_pipe<C, D, 0, true, 0, false, WA>(tkp, stage, pipe, arows, lo, g0, g1, k);
                    break;
                case 1:  // one per-row input: its runs for the U rows loaded together
                         // (domains up to 4; larger ones would spill them)
                    if constexpr (D <= 4) {
                        if (tk.R0 == 2) {
                            item_pipe<C, D, 1, true, 2, false, WA>(tkp, stage, pipe, arows, lo, g0, g1, k);
                            break;
                        }
                        if (tk.R0 == 3) {
                            item_pipe<C, D, 1, true, 3, false, WA>(tkp, stage, pipe, arows, lo, g0, g1, k);
                            break;
                        }
                        if (tk.R0 == 4) {
                            item_pipe<C, D, 1, true, 4, false, WA>(tkp, stage, pipe, arows, lo, g0, g1, k);
                            break;
                        }
                    }
                    item_pipe<C, D, 1, true, 0, false, WA>(tkp, stage, pipe, arows, lo, g0, g1, k);
                    break;
                default: item_pipe<C, D, 2, true, 0, false, WA>(tkp, stage, pipe, arows, lo, g0, g1, k); break;
                }
            } else {
                switch (tk.F - tk.n_gi) {
                case 0: item_pipe<C, D, 0, false, 0, false, WA>(tkp, stage, pipe, arows, lo, g0, g1, k); break;
                case 1: item_pipe<C, D, 1, false, 0, false, WA>(tkp, stage, pipe, arows, lo, g0, g1, k); break;
                default: item_pipe<C, D, 2, false, 0, false, WA>(tkp, stage, pipe, arows, lo, g0, g1, k); break;
                }
            }
            return;
        }
    }
    switch (tk.F - tk.n_gi) {
    case 0: item_fixed_nr<C, D, FC, 0, 0, WA>(tkp, stage, lo, g0, g1, k); break;
    case 1:  // one per-row input: the rows of u unrolled for small radices and
             // domains (larger ones would spill the loaded runs)
        if constexpr (D <= 3) {
            if (tk.R0 == 2) {
                item_fixed_nr<C, D, FC, 1, 2, WA>(tkp, stage, lo, g0, g1, k);
                break;
            }
            if (tk.R0 == 3) {
                item_fixed_nr<C, D, FC, 1, 3, WA>(tkp, stage, lo, g0, g1, k);
                break;
            }
        }
        item_fixed_nr<C, D, FC, 1, 0, WA>(tkp, stage, lo, g0, g1, k);
        break;
    case 2: item_fixed_nr<C, D, FC, 2, 0, WA>(tkp, stage, lo, g0, g1, k); break;
    default:
        if constexpr (FC <= 3) item_fixed_nr<C, D, FC, 3, 0, WA>(tkp, stage, lo, g0, g1, k);
        else item_fixed_anyF<C, D, WA>(tkp, stage, lo, g0, g1, k);
        break;
    }
}

// Any domain size (runtime loop over x_i's values), at most FC inputs.
template <typename C, int FC>
__device__ __noinline__ void item_anyD(const TaskDev *__restrict__ tkp, const unsigned char *stage, int lo, int g0,
                                          int g1, uint32_t k)
{
    const TaskDev tk = *tkp;
    using T = typename C::val;
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
            float t = 1.f;  // sum-product only
            auto push = [&](A s, int l) {
                if (l == 0 || s < best) {
                    if constexpr (C::kSum) t = l == 0 ? 1.f : t * __expf(s - best) + 1.f;
                    best = s;
                    bi = l;
                } else if constexpr (C::kSum) {
                    if (s < kInfF) t += __expf(best - s);
                }
            };
            if (d % 4 == 0) {  // runs of a multiple of 4 entries are 16-byte aligned: vector loads
                for (int l0 = 0; l0 < d; l0 += 4) {
                    A s4[4];
                    T v[4];
                    load_run<4>(q[0] + l0, v);
#pragma unroll
                    for (int i = 0; i < 4; ++i) s4[i] = C::from(v[i]);
#pragma unroll
                    for (int f = 1; f < FC; ++f)
                        if (f < F) {
                            load_run<4>(q[f] + l0, v);
#pragma unroll
                            for (int i = 0; i < 4; ++i) s4[i] = C::add(s4[i], v[i], k);
                        }
#pragma unroll
                    for (int i = 0; i < 4; ++i) push(s4[i], l0 + i);
                }
            } else {
                for (int l = 0; l < d; ++l) {
                    A s = C::from(q[0][l]);
#pragma unroll
                    for (int f = 1; f < FC; ++f)
                        if (f < F) s = C::add(s, q[f][l], k);
                    push(s, l);
                }
            }
            if constexpr (C::kSum) best = lse_value(best, t);
            const int o = a[0] + u * du[0] + lo;
            out[o] = C::store(best);
            if constexpr (!C::kSum) tk.arg[o] = static_cast<uint8_t>(bi);
        }
    }
}

// Any domain size, any number of inputs.
template <typename C>
__device__ __noinline__ void item_anyD_anyF(const TaskDev *__restrict__ tkp, const unsigned char *stage, int lo,
                                               int g0, int g1, uint32_t k)
{
    const TaskDev tk = *tkp;
    using T = typename C::val;
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
            float t = 1.f;  // sum-product only
            for (int l = 0; l < d; ++l) {
                A s = A(0);
                for (int f = 0; f < F; ++f)
                    s = C::add(s, input_base<T>(tk.in[f], stage)[Ar[1 + f] + u * du[1 + f] + Brow[f] + l], k);
                if (l == 0 || s < best) {
                    if constexpr (C::kSum) t = l == 0 ? 1.f : t * __expf(s - best) + 1.f;
                    best = s;
                    bi = l;
                } else if constexpr (C::kSum) {
                    if (s < kInfF) t += __expf(best - s);
                }
            }
            if constexpr (C::kSum) best = lse_value(best, t);
            const int o = Ar[0] + u * du[0] + lo;
            out[o] = C::store(best);
            if constexpr (!C::kSum) tk.arg[o] = static_cast<uint8_t>(bi);
        }
    }
}

// Order-preserving map of a non-NaN float to uint32 (unsigned order of the
// keys = numeric order of the floats), and its inverse.
__device__ __forceinline__ uint32_t float_key(float x)
{
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_float(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Wide domains (d >= 32): a warp computes one output row at a time, lane j
// holding x_i's values j, j + 32, ...; every input's run is read by one
// coalesced warp access per 32 values.  The row minimum is one warp min
// (redux) over each lane's minimum (floats as order-preserving keys), its
// first argmin a second warp min over the lowest value index that holds it.
// The warp's row is lo (a lo chunk of a wide task has one row per warp); the
// rows of two consecutive values of u are loaded before either is reduced,
// so that two rows' loads are in flight.  RUNS = 32-value runs per lane
// (4: d <= 128, 8: d <= 255).
template <typename C, int FC, int RUNS>
__device__ __noinline__ void item_wide(const TaskDev *__restrict__ tkp, const unsigned char *stage, int lo,
                                       int g0, int g1, uint32_t k)
{
    const TaskDev tk = *tkp;
    using T = typename C::val;
    using A = typename C::acc;
    const int lane = threadIdx.x & 31;
    const int F = tk.F, d = tk.d, R0 = tk.R0;
    const int32_t *du = tk.A + static_cast<int64_t>(tk.G) * tk.sa;
    T *out = static_cast<T *>(tk.out);
    const int32_t *Brow = tk.B + static_cast<int64_t>(lo) * tk.sb;
    // with the input count a template bound, each input's base (its row lo
    // included) and u stride stay in registers for the whole item
    const T *p[FC > 0 ? FC : 1];
    int32_t pu[FC > 0 ? FC : 1];
#pragma unroll
    for (int f = 0; f < FC; ++f) {
        p[f] = (f < F) ? input_base<T>(tk.in[f], stage) + Brow[f] : nullptr;
        pu[f] = (f < F) ? du[1 + f] : 0;
    }
    // minimum and first argmin of one row's sums (sum-product: -log sum exp),
    // written by lane 0; every lane holds at least one value (d >= 32)
    auto finish = [&](const A (&acc)[RUNS], int o) {
        uint32_t m = 0xffffffffu;
#pragma unroll
        for (int j = 0; j < RUNS; ++j) {
            if (lane + 32 * j < d) {
                uint32_t key;
                if constexpr (std::is_same<A, uint32_t>::value) key = acc[j];
                else key = float_key(acc[j]);
                m = key < m ? key : m;
            }
        }
        m = __reduce_min_sync(0xffffffffu, m);
        A best;
        if constexpr (std::is_same<A, uint32_t>::value) best = m;
        else best = key_float(m);
        uint32_t bi = 0;
        if constexpr (!C::kSum) {
            uint32_t li = 0xffffffffu;
#pragma unroll
            for (int j = RUNS - 1; j >= 0; --j)
                if (lane + 32 * j < d && acc[j] == best) li = lane + 32 * j;
            bi = __reduce_min_sync(0xffffffffu, li);
        } else {
            // sum exp(min - s_l) over the lane's values, then over the warp
            if (best < kInfF) {
                float t = 0.f;
#pragma unroll
                for (int j = 0; j < RUNS; ++j)
                    if (lane + 32 * j < d) t += __expf(best - acc[j]);
#pragma unroll
                for (int s = 16; s > 0; s >>= 1) t += __shfl_xor_sync(0xffffffffu, t, s);
                best -= __logf(t);
            }
        }
        if (lane == 0) {
            out[o] = C::store(best);
            if constexpr (!C::kSum) tk.arg[o] = static_cast<uint8_t>(bi);
        }
    };
    for (int g = g0; g < g1; ++g) {
        const int32_t *Ar = tk.A + static_cast<int64_t>(g) * tk.sa;
        for (int u = 0; u < R0; u += 2) {
            const bool two = u + 1 < R0;  // uniform across the warp
            A a0[RUNS], a1[RUNS];
#pragma unroll
            for (int j = 0; j < RUNS; ++j) a0[j] = a1[j] = A(0);
            for (int f = 0; f < F; ++f) {
                const T *q0;
                int32_t step;
                if (FC > 0 && f < FC) {
                    step = pu[f];
                    q0 = p[f] + (Ar[1 + f] + u * step);
                } else {
                    step = du[1 + f];
                    q0 = input_base<T>(tk.in[f], stage) + (Ar[1 + f] + u * step + Brow[f]);
                }
                const T *q1 = q0 + step;
#pragma unroll
                for (int j = 0; j < RUNS; ++j) {
                    const int l = lane + 32 * j;
                    if (l < d) {
                        a0[j] = C::add(a0[j], q0[l], k);
                        if (two) a1[j] = C::add(a1[j], q1[l], k);
                    }
                }
            }
            finish(a0, Ar[0] + u * du[0] + lo);
            if (two) finish(a1, Ar[0] + (u + 1) * du[0] + lo);
        }
    }
}

template <typename C, int D>
__device__ __forceinline__ void dispatch_f(const TaskDev *__restrict__ tkp, const TaskDev &tk, int fc,
                                           const unsigned char *stage, unsigned char *pipe, const int32_t *arows,
                                           int lo, int h0, int h1, uint32_t k)
{
    if constexpr (D == 0) {
        switch (fc) {
        case 0: item_anyD<C, 3>(tkp, stage, lo, h0, h1, k); break;
        case 1: item_anyD<C, 7>(tkp, stage, lo, h0, h1, k); break;
        default: item_anyD_anyF<C>(tkp, stage, lo, h0, h1, k); break;
        }
    } else {
        // fp32 min-sum with domains up to 4 (the -log p mini-bucket bounds,
        // whose plans keep no argmin tables) has variants that leave the
        // argmin out altogether
        constexpr bool kNoArg = std::is_same<C, Cost<float>>::value && D <= 4;
        switch (fc) {
        case 0:
            if constexpr (kNoArg) {
                if (!tk.arg) {
                    item_fixed<C, D, 3, false>(tkp, tk, stage, pipe, arows, lo, h0, h1, k);
                    break;
                }
            }
            item_fixed<C, D, 3>(tkp, tk, stage, pipe, arows, lo, h0, h1, k);
            break;
        case 1:
            if constexpr (kNoArg) {
                if (!tk.arg) {
                    item_fixed<C, D, 7, false>(tkp, tk, stage, pipe, arows, lo, h0, h1, k);
                    break;
                }
            }
            item_fixed<C, D, 7>(tkp, tk, stage, pipe, arows, lo, h0, h1, k);
            break;
        default:
            if constexpr (D <= 10) {
                if (tk.n_gi - tk.n_lo <= 8 && tk.F - tk.n_gi <= 2) {
                    item_fixed_manyF<C, D>(tkp, stage, lo, h0, h1, k);
                    break;
                }
            }
            item_fixed_anyF<C, D>(tkp, stage, lo, h0, h1, k);
            break;
        }
    }
}

template <typename C>
__device__ __forceinline__ void dispatch(const TaskDev *__restrict__ tkp, const TaskDev &tk,
                                         const unsigned char *stage, unsigned char *pipe, const int32_t *arows,
                                         int lo, int h0, int h1, uint32_t k)
{
    const int dc = tk.variant / kNumFClass, fc = tk.variant % kNumFClass;
    switch (dc) {
    case 1: dispatch_f<C, 2>(tkp, tk, fc, stage, pipe, arows, lo, h0, h1, k); break;
    case 2: dispatch_f<C, 3>(tkp, tk, fc, stage, pipe, arows, lo, h0, h1, k); break;
    case 3: dispatch_f<C, 4>(tkp, tk, fc, stage, pipe, arows, lo, h0, h1, k); break;
    case 4: dispatch_f<C, 5>(tkp, tk, fc, stage, pipe, arows, lo, h0, h1, k); break;
    case 5: dispatch_f<C, 6>(tkp, tk, fc, stage, pipe, arows, lo, h0, h1, k); break;
    case 6: dispatch_f<C, 7>(tkp, tk, fc, stage, pipe, arows, lo, h0, h1, k); break;
    case 7: dispatch_f<C, 8>(tkp, tk, fc, stage, pipe, arows, lo, h0, h1, k); break;
    case 8: dispatch_f<C, 9>(tkp, tk, fc, stage, pipe, arows, lo, h0, h1, k); break;
    case 9: dispatch_f<C, 10>(tkp, tk, fc, stage, pipe, arows, lo, h0, h1, k); break;
    case kDClass16: dispatch_f<C, 16>(tkp, tk, fc, stage, pipe, arows, lo, h0, h1, k); break;
    case kDClassWide:
        if (tk.d <= 128) {
            if (fc == 0) item_wide<C, 3, 4>(tkp, stage, lo, h0, h1, k);
            else if (fc == 1) item_wide<C, 7, 4>(tkp, stage, lo, h0, h1, k);
            else item_wide<C, 0, 4>(tkp, stage, lo, h0, h1, k);
        } else {
            if (fc == 0) item_wide<C, 3, 8>(tkp, stage, lo, h0, h1, k);
            else if (fc == 1) item_wide<C, 7, 8>(tkp, stage, lo, h0, h1, k);
            else item_wide<C, 0, 8>(tkp, stage, lo, h0, h1, k);
        }
        break;
    default: dispatch_f<C, 0>(tkp, tk, fc, stage, pipe, arows, lo, h0, h1, k); break;
    }
}

// Programmatic dependent launch (consecutive levels of one run): a launch may
// start while the previous one drains; griddep_wait blocks until the previous
// launch has completed and its writes are visible, griddep_launch_dependents
// lets the next launch be scheduled (its CTAs still wait before reading).
// Both are no-ops for a launch without a programmatic predecessor / successor.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Dependencies of a launch over several levels: an acquire load of a
// completion counter, and the wait for every producer task of task a to
// complete all of its items.  Bounded in time (kWaitNs from the first poll)
// and in polls; gives up at once when another CTA has set the status word.
__device__ __forceinline__ int ld_acquire(const int32_t *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool wait_producers(const LaunchDev &L, int a, unsigned long long limit_ns = kWaitNs)
{
    const int j0 = L.dep_off[a], j1 = L.dep_off[a + 1];
    unsigned long long t0 = 0;
    int polls = 0;
    for (int j = j0; j < j1; ++j) {
        const int p = L.deps[j];
        const int need = L.prefix[p + 1] - L.prefix[p];
        while (ld_acquire(L.done + p) < need) {
            if (polls == 0) t0 = global_ns();
            if (*reinterpret_cast<volatile int32_t *>(L.status) != kStatusOk) return false;
            if (++polls > kMaxSpin || global_ns() - t0 > limit_ns) return false;
            __nanosleep(64);
        }
    }
    // the producers' tables may next be read by bulk copies (async proxy)
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return true;
}

// ------------------------------------------------------------- kernel
// SPEC = 0: every variant (dispatch by the task's descriptor); SPEC = D
// (2..4; int32 and the sum-product): the two-term rows of domain D with u of
// radix D alone, for launches whose tasks all take them (a task that does
// not fit sets kStatusBadSpec).
template <typename C, int SPEC = 0>
__global__ void __launch_bounds__(kMaxThreads, 2) util_kernel(const LaunchDev L)
{
    extern __shared__ __align__(128) unsigned char stage[];
    __shared__ uint64_t bar;
    __shared__ int s_item[2];
    __shared__ int s_staged;  // task whose tables are in shared memory, -1 = none
    __shared__ int s_ready;   // task whose producers are known to be complete, -1 = none
    __shared__ int s_ok;

    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar, 1);
        s_staged = -1;
        s_ready = -1;
        s_item[0] = atomicAdd(L.counter, 1);  // this launch's own counter, cleared before the run
        fence_mbar_init();
    }
    // the work-item prefixes (written before the launch, like every
    // descriptor) in shared memory when they fit
    const int32_t *prefix = L.prefix;
    if (L.prefix_smem >= 0) {
        int32_t *sp = reinterpret_cast<int32_t *>(stage + L.prefix_smem);
        for (int i = tid; i <= L.n_tasks; i += blockDim.x) sp[i] = L.prefix[i];
        prefix = sp;
    }
    __syncthreads();
    // the next level may be scheduled now: its CTAs become resident only as
    // this launch's CTAs exit (every CTA of this launch is resident already)
    griddep_launch_dependents();
    // the first item's offset rows (cp.async path) are descriptors written
    // before the launch, and its staged tables may all be originals, which
    // the run does not write: thread 0 starts those copies while the previous
    // level completes (the bytes are expected on the barrier without an
    // arrival; the item's own arrival below completes the phase)
    bool early = false;
    if (s_item[0] < L.total_items) {
        const int item0 = s_item[0];
        int a = 0, b = L.n_tasks;
        while (b - a > 1) {
            const int mid = (a + b) >> 1;
            if (prefix[mid] <= item0) a = mid;
            else b = mid;
        }
        const TaskDev *t0 = L.tasks + a;
        const bool rows = t0->pipe != 0;
        const bool stg = t0->stage_bytes > 0 && t0->cin;
        if (rows || stg) {
            if (tid == 0) {
                const int nlc = t0->nlc, hc = t0->hc, G = t0->G;
                const int h0 = ((item0 - prefix[a]) / nlc) * hc;
                const uint32_t rows_bytes = rows ? static_cast<uint32_t>(min(h0 + hc, G) - h0) * 16u : 0u;
                fence_proxy_async();
                mbar_expect_tx(&bar, rows_bytes + (stg ? static_cast<uint32_t>(t0->stage_bytes) : 0u));
                if (stg) {
                    for (int f = 0; f < t0->F; ++f) {
                        const InDev in = t0->in[f];
                        if (in.stage_off >= 0)
                            tma_bulk_g2s(stage + in.stage_off, in.ptr, static_cast<uint32_t>(in.bytes16), &bar);
                    }
                    s_staged = a;
                }
                if (rows) tma_bulk_g2s(stage + L.arows_off, t0->A + static_cast<int64_t>(h0) * 4, rows_bytes, &bar);
            }
            early = true;
        }
    }
    __syncthreads();  // s_staged
    // tables written by the previous level are read only after this point.
    // (The next item is claimed after it too: a CTA that claimed two items
    // while waiting would take work from the CTAs that start later.)
    griddep_wait();
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
            if (prefix[mid] <= item) a = mid;
            else b = mid;
        }
        const TaskDev tk = L.tasks[a];

        if (L.done != nullptr && s_ready != a) {
            // a launch over several levels: wait for the tasks this one reads.
            // Every thread has read s_ready once all are at this barrier;
            // only then may thread 0 change it (a thread that read it after
            // the change would skip the barriers below)
            __syncthreads();
            if (tid == 0) {
                s_ok = wait_producers(L, a) ? 1 : 0;
                if (!s_ok) atomicExch(L.status, kStatusTimeout);
                s_ready = a;
            }
            __syncthreads();
            if (!s_ok) {
                if (early) {  // let the first item's early copies land (bounded) before leaving
                    if (tid == 0) mbar_arrive_expect_tx(&bar, 0u);
                    mbar_wait_bounded(&bar, phase);
                }
                return;
            }
        }

        const int local = item - prefix[a];
        const int hr = local / tk.nlc;
        const int lc = local - hr * tk.nlc;
        const int h0 = hr * tk.hc;
        const int h1 = min(h0 + tk.hc, tk.G);
        // one TMA transaction per item: the task's small tables (when this CTA
        // has not staged them yet) and, for the cp.async path, the item's
        // contiguous A rows
        const bool restage = tk.stage_bytes > 0 && s_staged != a;
        const uint32_t rows_bytes = (tk.pipe && !early) ? static_cast<uint32_t>(h1 - h0) * 16u : 0u;
        if (restage || rows_bytes || early) {
            __syncthreads();  // every thread is done with the previous copies
            if (tid == 0) {
                fence_proxy_async();
                mbar_arrive_expect_tx(&bar, (restage ? static_cast<uint32_t>(tk.stage_bytes) : 0u) + rows_bytes);
                if (restage) {
                    for (int f = 0; f < tk.F; ++f) {
                        const InDev in = tk.in[f];
                        if (in.stage_off >= 0)
                            tma_bulk_g2s(stage + in.stage_off, in.ptr, static_cast<uint32_t>(in.bytes16), &bar);
                    }
                    s_staged = a;
                }
                if (rows_bytes) tma_bulk_g2s(stage + L.arows_off, tk.A + static_cast<int64_t>(h0) * 4, rows_bytes, &bar);
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

        // one thread per row, except the wide variant (one warp per row) and
        // the four-row variant (four consecutive rows per thread)
        const bool wide = tk.variant / kNumFClass == kDClassWide;
        const int lo = wide ? lc * static_cast<int>(blockDim.x >> 5) + (tid >> 5)
                            : (lc * static_cast<int>(blockDim.x) + tid) * (tk.v4 ? 4 : 1);
        if (lo < tk.P_lo) {
            if constexpr (SPEC > 0) {
                constexpr bool kPk = std::is_same<C, Cost<int32_t>>::value;
                if (rows_spec_of(tk, kPk) == SPEC)
                    item_pipe<C, SPEC, 0, true, SPEC, kPk>(L.tasks + a, stage, stage + L.pipe_off,
                                                           reinterpret_cast<const int32_t *>(stage + L.arows_off), lo,
                                                           h0, h1, L.top_k);
                else
                    atomicExch(L.status, kStatusBadSpec);
            } else {
                dispatch<C>(L.tasks + a, tk, stage, stage + L.pipe_off,
                            reinterpret_cast<const int32_t *>(stage + L.arows_off), lo, h0, h1, L.top_k);
            }
        }

        __syncthreads();
        if (L.done != nullptr && tid == 0) {
            // every thread's stores of this item precede the barrier above; the
            // release makes them visible to a CTA whose acquire load sees the count
            asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(L.done + a) : "memory");
        }
        item = s_item[nb];
        early = false;
        ++it;
    }
}

// Host: launch one UTIL kernel instantiation; with pdl the launch carries the
// programmatic stream serialization attribute (it may be scheduled while its
// predecessor on the stream drains, see griddep_wait).
template <typename K>
inline cudaError_t launch_util_kernel(K kernel, const LaunchDev &L, int grid, int threads, int smem, cudaStream_t s,
                                      bool pdl)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = static_cast<size_t>(smem);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, L);
}

}  // namespace gpube
