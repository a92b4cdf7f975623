// Device-side descriptors shared by the host planner (C++) and the kernels
// (CUDA).  Plain structs of pointers and sizes; the planner fills them and
// copies them to the arena once per bind.
#pragma once
#include <stdint.h>

namespace gpube {

// Launch-shape limits of the UTIL kernel.
constexpr int kMaxThreads = 512;      // CTA size upper bound (launch bounds)
constexpr int kStageAlign = 16;       // bytes: TMA bulk-copy granularity
constexpr int kMaxSpin = 1 << 20;     // iteration limit of every device-side wait

// Device status codes written to the status word.
constexpr int kStatusOk = 0;
constexpr int kStatusTimeout = 1;

// Kernel variants: the eliminated domain class times the input-count class.
// D class 0 = any domain size (runtime loop); 1..7 = domain 2..8.
// F class 0..2 = at most 4 or 8 inputs held in registers; 2 = any count.
constexpr int kNumFClass = 3;
inline int dclass_of(int d) { return (d >= 2 && d <= 8) ? d - 1 : 0; }
inline int fclass_of(int F) { return F <= 4 ? 0 : F <= 8 ? 1 : 2; }

// One input of a (mini-)bucket.
struct alignas(16) InDev {
    const void *ptr;     // device table, row-major over the input's scope
    int32_t stage_off;   // byte offset of its copy in shared memory, -1 = read from global
    int32_t bytes16;     // table bytes rounded up to 16 (copy size when staged)
};

// One (mini-)bucket = one task of the UTIL kernel.
//
// Its output rows r (the separator assignments, row-major) are split as
// r = hi * P_lo + lo: lo enumerates the lowest separator digits, hi the
// others.  For input f the row offset of x_i's d contiguous entries is
// A[h][f] + B[lo][f], where h is hi's index in the task's chosen iteration
// order and A[h][F] is the output offset of (hi, lo = 0).
struct alignas(16) TaskDev {
    const int32_t *A;    // [H][sa]
    const int32_t *B;    // [P_lo][sb]
    const InDev *in;     // [F]
    void *out;           // [rows] int32 or float
    uint8_t *arg;        // [rows]
    int32_t F, d, sa, sb;
    int32_t P_lo, H, hc, nlc;  // nlc = lo chunks of blockDim.x rows
    int32_t variant;           // dclass * kNumFClass + fclass
    int32_t stage_bytes;       // sum of staged bytes (multiple of 16)
    int32_t n_items;           // nlc * ceil(H / hc)
    int32_t pad;
};

// One kernel launch: a list of tasks whose work items are handed out by an
// atomic counter (a device-side work queue).
struct LaunchDev {
    const TaskDev *tasks;
    const int32_t *prefix;  // [n_tasks + 1] first work item of each task
    int32_t n_tasks;
    int32_t total_items;
    int32_t *counter;       // queue head, zeroed before the launch
    int32_t *status;        // error word (kStatus*)
    uint32_t top_k;         // WCSP saturation value
    int32_t pad;
};

// Compact plan of one task, expanded into its A and B tables on the device.
struct alignas(16) ExpandDev {
    int32_t *A;
    int32_t *B;
    int32_t m, L, nh, F;    // separator digits, lo digits, hi digits, inputs
    int32_t sa, sb;
    int32_t H, P_lo;
    int32_t rad_off;        // pool offset of rad[m] (natural digit order, slowest first)
    int32_t perm_off;       // pool offset of hperm[nh] (hi digits, fastest first)
    int32_t stride_off;     // pool offset of stride[(F + 1) * m] (slot F = output)
    int32_t pad;
};

// VALUE phase.
struct alignas(16) ValueTerm {
    const void *tab;        // cost table (sum terms) or argmin table (lookup)
    int32_t nv;             // scope variables other than the assigned one
    int32_t var_off;        // offset into vvars / vstrides
};

struct alignas(8) ValueVar {
    int32_t mode;           // 0: no bucket (value 0); 1: argmin lookup; 2: bucket sum
    int32_t d;
    int32_t term_off;
    int32_t n_terms;
};

struct ValueDev {
    const int32_t *lev_off;     // [n_levels + 1]
    const int32_t *vorder;      // [n]
    const ValueVar *vinfo;      // [n]
    const ValueTerm *terms;
    const int32_t *vvars;
    const int32_t *vstrides;
    const ValueTerm *evals;     // original functions, for the Eq. 1 cost
    const void *const *roots;   // root tables (one entry each)
    int32_t n, n_levels, n_evals, n_roots;
    double const_sum;           // constant functions
    uint32_t top_k;
    int32_t is_float;
    double *result;             // [2]: bound, cost
    int32_t *sigma;             // [n]
};

}  // namespace gpube
