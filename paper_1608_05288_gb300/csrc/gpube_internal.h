// Host-side structures of the library: the loaded problem, the elimination
// plan and the device state.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <memory>
#include <string>
#include <vector>

#include "../../include/gpube.h"
#include "gpube_dev.h"

struct wcsp {
    int32_t n = 0;
    std::vector<int32_t> dom;
    int32_t nf = 0;
    std::vector<std::vector<int32_t>> scope;   // as given
    std::vector<std::vector<int32_t>> itab;    // WCSP_INT32_SAT, clamped to top_k
    std::vector<std::vector<float>> ftab;      // WCSP_FP32_LOG
    int32_t cost_type = WCSP_INT32_SAT;
    uint32_t top_k = 1u << 30;
    std::vector<std::vector<int32_t>> adj;     // primal graph, sorted neighbour lists
    // holders: the caller (from wcsp_load until wcsp_free) and each server
    // request that still needs the problem; the last one deletes it
    std::atomic<int> refs{1};
    wcsp() = default;
    wcsp(const wcsp &o)
        : n(o.n), dom(o.dom), nf(o.nf), scope(o.scope), itab(o.itab), ftab(o.ftab), cost_type(o.cost_type),
          top_k(o.top_k), adj(o.adj)
    {
    }
    wcsp &operator=(const wcsp &) = delete;
};

inline void wcsp_ref(wcsp *w) { w->refs.fetch_add(1, std::memory_order_relaxed); }
inline void wcsp_unref(wcsp *w)
{
    if (w && w->refs.fetch_sub(1, std::memory_order_acq_rel) == 1) delete w;
}

namespace gpube {

int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);

// A cost function during planning: an original constraint or a bucket
// function.  Its canonical scope lists variables by descending elimination
// position, so its bucket variable is last and has stride 1.
struct Func {
    std::vector<int32_t> scope;
    int64_t size = 1;
    int32_t task = -1;        // producing task, -1 for an original
    size_t off = 0;           // arena byte offset of its cost table
    const void *ext = nullptr;  // device table outside the arena (single-bucket calls)
};

// VALUE plan with arena offsets (pointers are patched in at bind time).
struct ValueTermH {
    size_t tab_off;
    int32_t nv, var_off;
};

struct ValuePlanH {
    std::vector<int32_t> lev_off, vorder;
    std::vector<ValueVar> vinfo;
    std::vector<ValueTermH> terms, evals;
    std::vector<int32_t> vvars, vstrides;
    std::vector<size_t> roots;
    int32_t n_levels = 0;
};

struct Task {
    int32_t var = -1, level = 0, d = 1;
    std::vector<int32_t> sep;      // descending elimination position
    std::vector<int32_t> inputs;   // function ids, kernel input order
    int64_t rows = 1;              // separator rows (output entries)
    size_t out_off = 0, arg_off = 0;
    // work decomposition (see TaskDev)
    int32_t L = 0;                 // lo digits (the lowest separator digits)
    int64_t P_lo = 1, H = 1;       // lo extent, hi extent
    int64_t G = 1;                 // groups = H / R0
    int32_t R0 = 1;                // radix of the fastest hi digit
    int32_t n_gi = 0;              // inputs [n_lo, n_gi) do not mention the fastest hi digit
    int32_t n_uo = 0;              // inputs [n_gi, n_uo) mention no other hi digit
    int32_t sa = 4, sb = 4;
    int32_t n_lo = 0;              // leading inputs that depend on lo digits only
    std::vector<int32_t> hperm;    // hi digit indices, fastest first
    size_t A_off = 0, B_off = 0;
    void *ext_out = nullptr;       // caller's output tables (single-bucket calls)
    uint8_t *ext_arg = nullptr;
    std::vector<int32_t> stage_off;  // per input: shared-memory byte offset or -1
    int32_t stage_bytes = 0;
    bool keep_arg = true;            // its argmin table is written
};

// Mini-bucket partition (Algorithm 2) / sum-product elimination, by kind.
inline bool kind_mbe(int kind) { return kind == GPUBE_KIND_MBE || kind == GPUBE_KIND_SUM_MBE; }
inline bool kind_sum(int kind) { return kind == GPUBE_KIND_SUM || kind == GPUBE_KIND_SUM_MBE; }

struct Plan {
    int32_t kind = GPUBE_KIND_BE;
    int32_t i_bound = 0, ibound_mode = GPUBE_IB_SEP_VARS;
    std::vector<int32_t> order, pos;
    std::vector<Func> funcs;       // originals 0..nf-1, then task outputs nf+t
    std::vector<Task> tasks;
    int32_t n_levels = 0;
    std::vector<int32_t> level_order;  // task ids sorted by (level, id)
    std::vector<int32_t> level_off;    // [n_levels + 1] into level_order
    int32_t width = 0, max_inputs = 0;
    double const_sum = 0.0;
    int64_t util_entries = 0, out_entries = 0, in_entries = 0;
    int32_t lo_target = 2048;
    int32_t stage_max_entries = 4096;
    int32_t stage_max_bytes = 32768;
    bool allow_pipe = true;   // group runs prefetched by the per-thread cp.async pipeline (KP groups in
                              // flight) where a task allows it; false: register variants (1-2 groups)
    bool allow_v4 = false;    // four consecutive rows per thread where a task allows it
    bool keep_arg = true;     // argmin tables asked for: the VALUE phase of BE and DPOP reads
                              // them (mini-bucket plans re-minimise over the bucket's
                              // functions instead) or solve_opts.argmin_tables
    size_t peak_live_bytes = 0;
    ValuePlanH value;
};

// Whether a task writes its argmin table: never for the sum-product, always
// when the plan asks for them, and otherwise unless the kernel has variants
// that leave the argmin out for the task's shape (fp32 min-sum, domains 2-4,
// at most 7 inputs); other shapes write theirs, unread.
inline bool task_keeps_arg(int cost_type, const Plan &P, const Task &T)
{
    if (kind_sum(P.kind)) return false;
    if (P.keep_arg) return true;
    return !(cost_type == WCSP_FP32_LOG && T.d >= 2 && T.d <= 4 && T.inputs.size() <= 7);
}

// Algorithmic bytes of a plan: every input entry read once (4 bytes), every
// output entry written once (4 bytes) with its argmin where the task keeps
// its argmin table (1 byte).
inline int64_t alg_bytes_of(const Plan &P)
{
    int64_t arg_bytes = 0;
    for (const Task &T : P.tasks)
        if (T.keep_arg) arg_bytes += T.rows;
    return 4 * P.in_entries + 4 * P.out_entries + arg_bytes;
}

// Launch parameters of one run.
struct LaunchCfg {
    int32_t threads = 256;
    int32_t rows_per_item = 128;
};

// planner (plan.cpp)
const char *last_error();
// Greedy min-fill order and its width; an empty order once the width would
// exceed give_up_above.
std::vector<int32_t> order_minfill(const wcsp &w, int32_t *width, int32_t give_up_above = INT32_MAX);
int32_t induced_width(const wcsp &w, const std::vector<int32_t> &order);
std::vector<int32_t> dfs_pseudotree(const wcsp &w);
int pseudotree_order(const wcsp &w, const int32_t *parent, std::vector<int32_t> &order);
int build_plan(const wcsp &w, int kind, int i_bound, const int32_t *parent, const solve_opts &o, Plan &P);
void task_strides(const wcsp &w, const Plan &P, const Task &T, std::vector<int32_t> &st);
void shape_tasks(const wcsp &w, Plan &P);

// kernels (util_kernel.cu)
// ktype: kKTypeInt / kKTypeFloat / kKTypeSum (gpube_dev.h); pdl: programmatic
// dependent launch after the previous UTIL launch on the stream
cudaError_t launch_util(const LaunchDev &L, int ktype, int grid, int threads, int smem, cudaStream_t s,
                        bool pdl = false);
int util_max_blocks_per_sm(int ktype, int threads, int smem);
cudaError_t launch_expand(const ExpandDev *tasks, const int64_t *prefix, int n_tasks, int64_t total,
                          const int32_t *pool, int num_sms, cudaStream_t s);
cudaError_t launch_value(const ValueDev &V, int ktype, int smem, cudaStream_t s);
cudaError_t launch_value_batch(const ValueBatch &B, int ktype, int smem, cudaStream_t s);
cudaError_t kernels_init_device();
int max_dynamic_smem();
cudaError_t launch_selftest_wait(int32_t *status, unsigned long long limit_ns, cudaStream_t s);

}  // namespace gpube

struct util_state;
// api.cpp helpers used by the server
namespace gpube {
double now_ms();
}

// Byte offsets of the descriptor and value regions of a state's arena.
struct DescLayout {
    size_t taskdev = 0, indev = 0, prefix = 0, expand = 0, exp_prefix = 0, pool = 0, dep_off = 0, deps = 0;
    size_t lev_off = 0, vorder = 0, vinfo = 0, terms = 0, vvars = 0, vstrides = 0, evals = 0, roots = 0;
    size_t n_in = 0, n_prefix = 0, n_pool = 0;
};

struct util_state {
    const wcsp *w = nullptr;
    std::unique_ptr<wcsp> own_w;  // the problem as planned, when it differs from the caller's: the
                                  // counting weights of a WCSP (sum-product kinds) and/or the
                                  // evidence functions appended (w points here then)
    int ktype = 0;                // UTIL kernel instantiation (kKType*)
    std::vector<int32_t> ev_vars; // variables util_condition may clamp
    std::vector<int32_t> ev_val;  // their current value, -1 = free
    int32_t ev_fid0 = 0;          // function id of ev_vars[0]'s unary (the others follow)
    gpube::Plan plan;
    gpube::LaunchCfg cfg;
    solve_opts opts{};
    int launch_mode = 1;          // kLaunchPerTask / kLaunchPerLevel / kLaunchFused
    bool use_graph = true;
    int32_t n_zero = 1;           // work-area ints cleared before each run (queue heads, completion counts)
    double plan_ms = 0.0;
    // layout (byte offsets from the arena base)
    size_t upload_bytes = 0;     // originals, packed first
    size_t desc_off = 0, desc_bytes = 0;   // descriptor region (rebuilt per launch config)
    size_t value_off = 0, value_bytes = 0; // value plan region
    size_t work_off = 0;         // counters + status + result
    size_t arena_bytes = 0;
    size_t arena_cap = 0;         // bytes of the bound arena (a re-shaped plan must fit in it)
    bool tables_stale = false;    // re-shaped since the offset tables were last expanded
    // device binding
    int device = 0;
    unsigned char *base = nullptr;
    bool owns_arena = false;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool bound = false, ran = false, value_ran = false;
    bool sync_on_free = true;  // false when an owner (the server) knows the work is done
    int num_sms = 0;
    // launches of one run
    std::vector<gpube::LaunchDev> launches;
    std::vector<int32_t> launch_grid, launch_smem, launch_ktype;
    // value plan pointers
    gpube::ValueDev vdev{};
    int32_t value_smem = 0;
    size_t counters_off = 0, status_off = 0, result_off = 0, sigma_off = 0;
    std::vector<unsigned char> host_blob;  // staging for uploads
    std::vector<unsigned char> orig_blob;  // original tables in device layout, when packed before binding
    DescLayout dl;
};

// api.cpp: arena layout of a planned state, its device descriptors (into
// host_blob), and the UTIL launches of one run on a stream.
void gpube_layout(util_state *s);
void gpube_prepack(util_state *s);
int gpube_build_descriptors(util_state *s);
int gpube_enqueue_util(util_state *s, cudaStream_t st);
