// VALUE-phase kernels (the value assignment of Algorithms 1-2 and DPOP's
// VALUE propagation, the root reduction and the Eq. 1 cost of the result);
// instantiated per cost type in util_kernel_i32.cu and util_kernel_f32.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "util_kernel.cuh"

namespace gpube {

// ------------------------------------------------------------- VALUE
__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Index of a term's table entry under the current assignment (warp-wide).
__device__ __forceinline__ long long term_index(const int32_t *vvars, const int32_t *vstrides, const ValueTerm &t,
                                                const unsigned char *sig, int lane)
{
    long long idx = 0;
    for (int j = lane; j < t.nv; j += 32)
        idx += static_cast<long long>(sig[vvars[t.var_off + j]]) * vstrides[t.var_off + j];
    return warp_sum_ll(idx);
}

// VALUE phase of a chain (every dependency level holds one variable, each
// read from an argmin table), run by one warp.  The variable of step j is
// read at an index that depends on the values assigned before it; the load
// is issued kChainAhead steps early, when the values of steps j-2 and j-1
// are not known yet: one candidate per combination of those two values
// (lane c holds digit c % D0 of step j-2 and c / D0 of step j-1), and step j
// picks its candidate by a shuffle.  The dependent load latency is thus
// spread over three steps.  The order of the steps is copied to shared memory.
constexpr int kChainAhead = 3;

__device__ __forceinline__ int warp_sum_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void value_chain(const ValueDev &V, const ValueVar *vinfo, const ValueTerm *terms,
                                            const int32_t *vvars, const int32_t *vstrides, unsigned char *sig,
                                            int32_t *order)
{
    const int lane = threadIdx.x & 31;
    const int n = V.n;
    for (int j = lane; j < n; j += 32) order[j] = V.vorder[j];
    __syncwarp();
    // issue the candidate load of step j (every step < j - 2 is assigned)
    // into the slot register c; table indices fit in int32 (tables hold
    // fewer than 2^31 entries).  Every lane loads (lanes past the candidates
    // reload candidate 0) and nothing reads c until its step: the load stays
    // in flight.
    auto prefetch = [&](int j, int &c) {
        if (j >= n) return;
        const int v = order[j];
        const ValueVar vi = vinfo[v];
        if (vi.mode != 1) return;
        const ValueTerm t = terms[vi.term_off];
        const int pa = j >= 2 ? order[j - 2] : -1, pb = j >= 1 ? order[j - 1] : -1;
        int base = 0, sa = 0, sb = 0;
        for (int q = lane; q < t.nv; q += 32) {
            const int x = vvars[t.var_off + q];
            const int st = vstrides[t.var_off + q];
            if (x == pa) sa = st;
            else if (x == pb) sb = st;
            else base += static_cast<int>(sig[x]) * st;  // assigned at a step <= j - 3
        }
        base = warp_sum_i(base);
        sa = warp_sum_i(sa);
        sb = warp_sum_i(sb);
        const int D0 = pa >= 0 ? vinfo[pa].d : 1, D1 = pb >= 0 ? vinfo[pb].d : 1;
        const int cand = lane < D0 * D1 ? lane : 0;
        const int hi = (cand * ((256 + D0 - 1) / D0)) >> 8;  // cand / D0 for cand < 32, D0 <= 5
        c = static_cast<const uint8_t *>(t.tab)[base + (cand - hi * D0) * sa + hi * sb];
    };
    // one register per slot, the loop unrolled by the slot count, so that a
    // step reads only its own slot (the other two loads stay in flight)
    // every lane writes each assigned value itself (the same value to the same
    // address), so each lane reads back its own writes: no warp barrier that
    // would wait for the loads in flight.  The last two values stay in
    // registers for the pick.
    int va = 0, vb = 0;  // values of steps j - 2 and j - 1
    auto step = [&](int j, int &c) {
        if (j >= n) return;
        const int v = order[j];
        const int pa = j >= 2 ? order[j - 2] : -1;
        const int D0 = pa >= 0 ? vinfo[pa].d : 1;
        const int pick = va + D0 * vb;
        const int val = vinfo[v].mode == 1 ? __shfl_sync(0xffffffffu, c, pick) : 0;
        sig[v] = static_cast<unsigned char>(val);
        va = vb;
        vb = val;
        prefetch(j + kChainAhead, c);  // the slot is free: load the candidates of step j + 3
    };
    int c0 = 0, c1 = 0, c2 = 0;
    prefetch(0, c0);
    prefetch(1, c1);
    prefetch(2, c2);
    for (int j = 0; j < n; j += kChainAhead) {
        step(j, c0);
        step(j + 1, c1);
        step(j + 2, c2);
    }
}

// VALUE phase in one CTA: variables grouped by dependency level (a variable
// depends on the other variables of its bucket, all eliminated later), one
// warp per variable.  BE / DPOP read the stored argmin of the bucket
// function at the separator's assignment; MBE takes the first argmin of the
// sum of every function of the bucket.  Then the root constants are summed
// (the optimum or lower bound) and the Eq. 1 cost of the assignment is
// evaluated over the original functions.
template <typename T>
__device__ __forceinline__ void value_body(const ValueDev &V)
{
    using C = Cost<T>;
    using A = typename C::acc;
    extern __shared__ __align__(16) unsigned char vsm[];
    __shared__ double red[2][32];
    unsigned char *sig = vsm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int v = threadIdx.x; v < V.n; v += blockDim.x) sig[v] = 0;
    // the per-variable plan, copied once to shared memory when it fits, so a
    // dependency level waits on one global load (the table entry) only
    const ValueVar *vinfo = V.vinfo;
    const ValueTerm *terms = V.terms;
    const int32_t *vvars = V.vvars, *vstrides = V.vstrides;
    if (V.plan_in_smem) {
        ValueVar *s_vinfo = reinterpret_cast<ValueVar *>(vsm + V.smem_sig);
        ValueTerm *s_terms = reinterpret_cast<ValueTerm *>(s_vinfo + ((V.n + 1) & ~1));
        int32_t *s_vvars = reinterpret_cast<int32_t *>(s_terms + V.n_terms);
        int32_t *s_vstrides = s_vvars + V.n_vv;
        for (int i = threadIdx.x; i < V.n; i += blockDim.x) s_vinfo[i] = V.vinfo[i];
        for (int i = threadIdx.x; i < V.n_terms; i += blockDim.x) s_terms[i] = V.terms[i];
        for (int i = threadIdx.x; i < V.n_vv; i += blockDim.x) {
            s_vvars[i] = V.vvars[i];
            s_vstrides[i] = V.vstrides[i];
        }
        vinfo = s_vinfo;
        terms = s_terms;
        vvars = s_vvars;
        vstrides = s_vstrides;
    }
    __syncthreads();
    if (V.chain) {
        if (warp == 0)
            value_chain(V, vinfo, terms, vvars, vstrides, sig, reinterpret_cast<int32_t *>(vsm + V.smem_step));
        __syncthreads();
    }
    for (int lev = 0; lev < (V.chain ? 0 : V.n_levels); ++lev) {
        const int b = V.lev_off[lev], e = V.lev_off[lev + 1];
        for (int i = b + warp; i < e; i += nw) {
            const int v = V.vorder[i];
            const ValueVar vi = vinfo[v];
            int val = 0;
            if (vi.mode == 1) {
                const ValueTerm t = terms[vi.term_off];
                const long long idx = term_index(vvars, vstrides, t, sig, lane);
                val = static_cast<const uint8_t *>(t.tab)[idx];
            } else if (vi.mode == 2) {
                constexpr int kMaxRuns = 8;  // domains up to 256 values
                A acc[kMaxRuns];
                for (int term = 0; term < vi.n_terms; ++term) {
                    const ValueTerm t = terms[vi.term_off + term];
                    const long long base = term_index(vvars, vstrides, t, sig, lane);
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

template <typename T>
__global__ void __launch_bounds__(256) value_kernel(const ValueDev V)
{
    value_body<T>(V);
}

// The VALUE phases of several finished problems in one launch (one CTA each).
template <typename T>
__global__ void __launch_bounds__(256) value_kernel_batch(const __grid_constant__ ValueBatch B)
{
    value_body<T>(B.v[blockIdx.x]);
}

}  // namespace gpube
