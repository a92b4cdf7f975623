// Device-side descriptors shared by the host planner (C++) and the kernels
// (CUDA).  Plain structs of pointers and sizes; the planner fills them and
// copies them to the arena once per bind.
#pragma once
#include <stdint.h>

namespace gpube {

// Launch-shape limits of the UTIL kernel.
constexpr int kMaxThreads = 512;      // CTA size upper bound (launch bounds)
constexpr int kStageAlign = 16;       // bytes: TMA bulk-copy granularity
constexpr int kMaxSpin = 1 << 24;     // iteration limit of every device-side wait (backstop)
constexpr unsigned long long kWaitNs = 1000000000ull;  // time limit of every device-side wait: 1 s

// Device status codes written to the status word.
constexpr int kStatusOk = 0;
constexpr int kStatusTimeout = 1;
constexpr int kStatusBadSpec = 2;  // a task reached a specialised kernel it does not fit (host error)

// UTIL kernel instantiations: int32 min-sum (WCSP_INT32_SAT), fp32 min-sum
// (WCSP_FP32_LOG), fp32 sum-product
constexpr int kKTypeInt = 0;
constexpr int kKTypeFloat = 1;
constexpr int kKTypeSum = 2;
// The same instantiations compiled with one item body only, the two-term
// rows of domain D with u of radix D, D = 2, 3, 4 (the full-size buckets of
// grid-like problems; packed keys for int32, factored rows for the
// sum-product): a launch whose tasks all take that body runs it, with its
// few hundred instructions instead of the whole dispatch in the instruction
// caches.  Kernel types kKTypeIntRows + D - 2 and kKTypeSumRows + D - 2.
constexpr int kKTypeIntRows = 3;
constexpr int kKTypeSumRows = 6;

// Kernel variants: the eliminated domain class times the input-count class.
// D class 0 = any domain size (runtime loop, one thread per row); 1..9 =
// domain 2..10; 10 = domain 16; 11 = wide domains (>= 32 values: a warp per
// row, lanes over the values, warp-shuffle min / argmin).
// F class 0..2 = at most 3 or 7 inputs held in registers (A rows of 4 or 8
// ints, B rows of 4 or 8 ints); 2 = any count.
constexpr int kNumFClass = 3;
constexpr int kWideD = 32;
constexpr int kDClass16 = 10;
constexpr int kDClassWide = 11;
inline int dclass_of(int d)
{
    return (d >= 2 && d <= 10) ? d - 1 : d == 16 ? kDClass16 : d >= kWideD ? kDClassWide : 0;
}
inline int fclass_of(int F) { return F <= 3 ? 0 : F <= 7 ? 1 : 2; }
// Row widths of the A (output + inputs) and B (inputs) offset tables.
inline int arow_of(int F) { return F <= 3 ? 4 : F <= 7 ? 8 : (F + 1 + 3) / 4 * 4; }
inline int brow_of(int F) { return F <= 3 ? 4 : F <= 7 ? 8 : (F + 3) / 4 * 4; }

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
// others.  The hi values are walked in a planner-chosen digit order whose
// fastest digit u (radix R0) is one the largest input does not mention; the
// other hi digits form the group index g.  For input f the row offset of
// x_i's d contiguous entries is A[g][1 + f] + u * A[G][1 + f] + B[lo][f]
// (row G of A holds the per-slot stride of u), and the output row is
// A[g][0] + u * A[G][0] + lo.  Inputs are ordered: n_lo that mention no hi
// digit (summed once per item), then up to n_gi that do not mention u
// (read once per group), then the rest (read per row).
struct alignas(16) TaskDev {
    const int32_t *A;    // [G + 1][sa]
    const int32_t *B;    // [P_lo][sb]
    const InDev *in;     // [F]
    void *out;           // [rows] int32 or float
    uint8_t *arg;        // [rows] argmins; null when none is kept (fp32 min-sum, d 2-4, F <= 7 only)
    int32_t F, d, sa, sb;
    int32_t P_lo, G, hc, nlc;  // hc = groups per item; nlc = lo chunks (blockDim.x rows, or blockDim.x / 32 for wide domains)
    int32_t variant;           // dclass * kNumFClass + fclass
    int32_t stage_bytes;       // sum of staged bytes (multiple of 16)
    int32_t n_items;           // nlc * ceil(G / hc)
    int32_t n_lo;              // inputs [0, n_lo) depend on lo only
    int32_t n_gi;              // inputs [n_lo, n_gi) do not depend on u
    int32_t R0;                // radix of u (1 when there is no hi digit)
    int32_t pipe;              // 1: the one group input is prefetched by cp.async
    int32_t n_uo;              // inputs [n_gi, n_uo) mention no hi digit but u
    int32_t nosat;             // integer costs whose row sums stay below the top cost and 2^30
                               // (from upper bounds of the inputs): no saturation, and
                               // (sum << 2 | l) fits in 32 bits
    int32_t v4;                // 1: a thread computes four consecutive rows (P_lo % 4 == 0,
                               // d 2..4, at most 3 inputs); its lo chunk is 4 x blockDim.x rows
    int32_t lin;               // bit f: input f's layout ends with the lo digits and x_i, so
                               // B[lo][f] = d * lo (four consecutive rows read one block)
    int32_t uni;               // bit f: input f has one offset over each aligned block of four
                               // lo rows (it mentions no digit that varies within one)
    int32_t cin;               // 1: every staged input is a table the run does not write (an
                               // original), so it may be copied before the previous launch ends
    int32_t pad3;
};

static_assert(sizeof(TaskDev) == 128, "a task descriptor is one 128-byte line");

#if defined(__CUDACC__)
#define GPUBE_HD __host__ __device__
#else
#define GPUBE_HD
#endif

// The domain D of the single-body instantiation that a task fits, or 0: the
// tasks that item_fixed<C, D, 3> sends to item_pipe<C, D, 0, true, D,
// packed> (domain class 1..3 = domain 2..4, at most 3 inputs, the group
// input pipelined, u of radix D, no other per-row input; packed: int32 sums
// below the top cost, as packed keys).
GPUBE_HD inline int rows_spec_of(const TaskDev &t, bool packed)
{
    const int D = t.variant / kNumFClass + 1;
    if (t.variant % kNumFClass != 0 || D < 2 || D > 4) return 0;
    if (t.v4 || !t.pipe || t.R0 != D || t.F != t.n_uo || (packed && !t.nosat)) return 0;
    return D;
}

// Depth of the per-thread cp.async pipeline of group inputs (groups ahead),
// and the most groups one item of that path spans (its A rows are copied to
// shared memory, 16 bytes each).
constexpr int kPipe = 4;
constexpr int kPipeSmall = 8;  // the depth for runs of at most 16 bytes (d <= 4)
constexpr int kMaxPipeRows = 256;
// Pipeline depth and shared-memory bytes per thread of the cp.async path for
// domain d: the slots plus four per-u partial sums, 4d bytes each (the
// packed-key rows read their partial sums back into registers and then use
// those four as pipeline slots too).
constexpr int pipe_depth(int d) { return d <= 4 ? kPipeSmall : kPipe; }
constexpr int pipe_bytes_per_thread(int d) { return (pipe_depth(d) + 4) * 4 * d; }

// One kernel launch: a list of tasks whose work items are handed out by an
// atomic counter (a device-side work queue).
//
// A launch over every level of a run (done != nullptr) lists its tasks in
// level order; a CTA that takes an item of task t first waits until every
// task t depends on (its inputs' producers, deps[dep_off[t] .. dep_off[t+1]),
// all earlier in the list) has completed all of its items, counted in
// done[].  Items are taken in increasing order by CTAs that are running, and
// a task depends only on earlier tasks, so the item with the lowest index not
// yet completed never waits: the launch always progresses.  Each wait is
// bounded; on expiry the CTA sets the status word and leaves, and the others
// see the status and leave too.
struct LaunchDev {
    const TaskDev *tasks;
    const int32_t *prefix;  // [n_tasks + 1] first work item of each task
    int32_t n_tasks;
    int32_t total_items;
    int32_t *counter;       // queue head, zeroed before the launch
    int32_t *status;        // error word (kStatus*)
    uint32_t top_k;         // WCSP saturation value
    int32_t pipe_off;       // byte offset of the cp.async pipeline area in shared memory
    int32_t arows_off;      // byte offset of the item's A rows (cp.async path) in shared memory
    int32_t prefix_smem;    // byte offset of a shared-memory copy of prefix, -1 = none (read it
                            // from global memory)
    int32_t *done;          // [n_tasks] completed items per task, zeroed before the launch; nullptr:
                            // a launch whose tasks depend on no task of the same launch
    const int32_t *dep_off; // [n_tasks + 1]
    const int32_t *deps;    // producer tasks (indices into tasks), each below the consumer's index
};

// A launch's prefix array is copied to shared memory (after the launch's
// other shared-memory areas, which end at byte smem) when it is at most this
// large: the task of each work item is then found by a binary search in
// shared memory instead of a chain of dependent global loads.  Returns the
// launch's shared-memory size.
constexpr int kPrefixSmemMax = 16384;
inline int place_prefix_smem(LaunchDev &L, int smem)
{
    const int bytes = (L.n_tasks + 1) * 4;
    if (bytes > kPrefixSmemMax) {
        L.prefix_smem = -1;
        return smem;
    }
    L.prefix_smem = (smem + 15) / 16 * 16;
    return L.prefix_smem + bytes;
}

// Launch modes of a run (solve_opts.batched).
constexpr int kLaunchPerTask = 0;   // one launch per (mini-)bucket
constexpr int kLaunchPerLevel = 1;  // one launch per elimination-tree level
constexpr int kLaunchFused = 2;     // one launch for every level, dependencies waited for on the device

// Compact plan of one task, expanded into its A and B tables on the device.
struct alignas(16) ExpandDev {
    int32_t *A;
    int32_t *B;
    int32_t m, L, nh, F;    // separator digits, lo digits, hi digits, inputs
    int32_t sa, sb;
    int32_t G, P_lo;        // groups (hi values / R0), lo extent
    int32_t rad_off;        // pool offset of rad[m] (natural digit order, slowest first)
    int32_t perm_off;       // pool offset of hperm[nh] (hi digits, fastest first)
    int32_t stride_off;     // pool offset of stride[(F + 1) * m] (row F = output)
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
    int32_t n_terms, n_vv;      // entries of terms and of vvars / vstrides
    int32_t plan_in_smem;       // 1: vinfo, terms, vvars, vstrides are copied to shared memory
    int32_t smem_sig;           // bytes reserved for the assignment in shared memory (16-aligned)
    int32_t chain;              // 1: one variable per level, argmin lookups, domains <= 5 (one warp)
    int32_t smem_step;          // chain: byte offset of the copy of vorder in shared memory
};

// Several VALUE phases in one launch (kernel parameter, one CTA each).
constexpr int kMaxValueBatch = 64;
struct ValueBatch {
    int32_t n, pad;
    ValueDev v[kMaxValueBatch];
};

}  // namespace gpube
