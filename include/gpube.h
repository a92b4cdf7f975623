/*
 * gpube.h - C ABI of the GB300 UTIL-table library.
 *
 * The library computes the bucket functions (UTIL tables) of Bucket
 * Elimination (BE, Algorithm 1), Mini-Bucket Elimination (MBE, Algorithm 2)
 * and the UTIL phase of DPOP (Section 4.1) on one NVIDIA GB300 GPU, and the
 * value-assignment (VALUE) phase that follows them, for problems stated as in
 * Sections 2-4 of arXiv 1608.05288:
 *
 *   WCSP <X, D, C>          (Section 2): integer costs in [0, top_k]; top_k
 *                           stands for "infinity" (not allowed) and sums
 *                           saturate at it;
 *   Bayesian network / MPE  (Section 3): costs -log p in fp32, p = 0 -> +inf;
 *                           max-product becomes min-sum;
 *   DCOP <X, D, C, A, alpha> (Section 4): one variable per agent; the UTIL
 *                           messages are BE's bucket functions along the
 *                           post-order of a DFS pseudo-tree.
 *
 * Conventions shared by every call
 *   - Variables are 0..n_vars-1.  An elimination order lists variables in the
 *     order they are eliminated (order[0] first).
 *   - A cost table is row-major over its scope as listed: the first scope
 *     variable varies slowest (the lexicographic rows of the bucket-table,
 *     Section 6.1).
 *   - A bucket function's scope is its separator sorted by descending
 *     elimination position; its eliminated variable, when present in a table,
 *     is last (Section 6.2).
 *   - Ties in min / argmin go to the lowest domain value.
 *   - Return codes: 0 on success, or a negative GPUBE_E* status; no call
 *     aborts the process.  wcsp_last_error() describes the last failure of
 *     the calling thread.
 *   - Device memory: either the caller passes an arena (a device pointer and
 *     its size, e.g. from torch) or, when the arena is NULL, the library
 *     allocates one itself with cudaMalloc and frees it with the state.
 *   - Streams: every GPU call runs on the caller's cudaStream_t (passed as
 *     void*; NULL = the legacy default stream).
 */
#ifndef GPUBE_H
#define GPUBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define GPUBE_OK 0
#define GPUBE_EINVAL (-22)     /* malformed problem or argument              */
#define GPUBE_ENOMEM (-12)     /* arena or budget too small / host OOM       */
#define GPUBE_ETIMEDOUT (-110) /* a bounded device-side wait gave up         */
#define GPUBE_ECUDA (-1000)    /* a CUDA runtime call failed                 */
#define GPUBE_ENODEV (-19)     /* no usable CUDA device                      */
#define GPUBE_EAGAIN (-11)     /* serving: request not admitted yet / busy   */

/* ------------------------------------------------------------ enumerations */
enum wcsp_cost_type {
    WCSP_INT32_SAT = 0, /* int32 costs in [0, top_k], saturating sum (Section 2) */
    WCSP_FP32_LOG = 1   /* fp32 -log p costs, +inf allowed (Section 3)           */
};

enum gpube_order_kind {
    GPUBE_ORDER_MINFILL = 0,    /* greedy min-fill; ties: fewest neighbours, lowest id   */
    GPUBE_ORDER_BEST = 1,       /* min-fill or the natural order 0..n-1, whichever has the
                                   smaller induced width (ties keep min-fill)            */
    GPUBE_ORDER_GIVEN = 2,      /* solve_opts.order                                       */
    GPUBE_ORDER_NATURAL = 3,    /* 0, 1, ..., n-1                                         */
    GPUBE_ORDER_PSEUDOTREE = 4  /* post-order of solve_opts.parent, or of the library's DFS
                                   pseudo-tree when parent is NULL (Section 6.2)          */
};

enum gpube_ibound_mode {
    GPUBE_IB_SEP_VARS = 0,    /* |scope(mini-bucket) \ {x_i}| <= i_bound                 */
    GPUBE_IB_JOINT_VARS = 1,  /* |scope(mini-bucket)| <= i_bound (the bound of Algorithm 2) */
    GPUBE_IB_LOG2_ENTRIES = 2 /* product of the mini-bucket's domains <= 2^i_bound        */
};

enum gpube_kind {
    GPUBE_KIND_BE = 0,     /* Algorithm 1: min over the eliminated variable        */
    GPUBE_KIND_MBE = 1,    /* Algorithm 2: mini-buckets under i_bound              */
    GPUBE_KIND_DPOP = 2,   /* BE along the post-order of a pseudo-tree (Sec. 4.1)  */
    GPUBE_KIND_SUM = 3,    /* sum-product: BE's buckets, each variable eliminated
                              by -log sum_l exp(-s_l) (see logz_solve)             */
    GPUBE_KIND_SUM_MBE = 4 /* sum-product over Algorithm 2's mini-buckets          */
};

/* ------------------------------------------------------------------ structs */

/* A problem (Sections 2-4).  All arrays are host memory owned by the caller;
 * wcsp_load copies them.  Function j has scope scope[scope_off[j] ..
 * scope_off[j+1]) (distinct variables; an empty scope is a constant) and
 * table costs[tab_off[j] .. tab_off[j+1]), whose length must be the product
 * of the scope's domain sizes.  costs points to int32 (WCSP_INT32_SAT:
 * values in [0, top_k]; larger values are read as top_k, negative values are
 * EINVAL) or to float (WCSP_FP32_LOG: values >= 0 or +inf). */
typedef struct wcsp_desc {
    int32_t n_vars;
    const int32_t *dom;       /* [n_vars], each 1..255                    */
    int32_t n_funcs;
    const int32_t *scope_off; /* [n_funcs + 1]                            */
    const int32_t *scope;     /* [scope_off[n_funcs]]                     */
    const int64_t *tab_off;   /* [n_funcs + 1], in entries                */
    const void *costs;        /* int32_t* or float*                       */
    int32_t cost_type;        /* enum wcsp_cost_type                      */
    int32_t top_k;            /* WCSP top cost k, 1..2^31-1 (int type)    */
} wcsp_desc;

/* Options of a solve.  Initialise with solve_opts_init(). */
typedef struct solve_opts {
    int32_t order_kind;        /* enum gpube_order_kind                                  */
    const int32_t *order;      /* [n] host, for GPUBE_ORDER_GIVEN                        */
    const int32_t *parent;     /* [n] host pseudo-tree (-1 = root) for ORDER_PSEUDOTREE  */
    int32_t ibound_mode;       /* enum gpube_ibound_mode (MBE)                           */
    int32_t batched;           /* 1: one persistent launch per elimination-tree level;
                                  0: one launch per (mini-)bucket;
                                  2: one persistent launch over every level, whose CTAs
                                     wait on the device (bounded, GPUBE_ETIMEDOUT) for the
                                     buckets that produce a bucket's inputs              */
    int32_t use_graph;         /* 1: capture the launch sequence once in a CUDA graph    */
    int32_t block_threads;     /* UTIL kernel CTA size (64..1024, multiple of 32); 0 = auto */
    int32_t rows_per_item;     /* separator rows of one work item per thread; 0 = auto  */
    int32_t lo_target;         /* minimum extent of a work item's inner row block; 0 = auto */
    int32_t stage_max_entries; /* tables up to this many entries are staged in shared
                                  memory; 0 = auto, -1 = never stage                    */
    void *arena;               /* device memory for all tables, or NULL                 */
    size_t arena_bytes;
    void *stream;              /* cudaStream_t, NULL = legacy default stream            */
    const char *autotune_cache;/* file for tuned launch parameters, or NULL             */
    int32_t device;            /* CUDA device ordinal                                    */
    const int32_t *evidence_vars; /* [n_evidence_vars] host: variables that util_condition
                                  may clamp on this plan (distinct), or NULL             */
    int32_t n_evidence_vars;
    int32_t pipeline;          /* 0: group inputs prefetched by the cp.async pipeline where a
                                  task allows it; -1: register variants only              */
    int32_t vector_rows;       /* 1: a thread computes four consecutive output rows where a
                                  task allows it (domains 2-3, at most 3 inputs, lo extent
                                  a multiple of 4): 16-byte cost stores, 4-byte argmin
                                  stores, block loads of inputs laid out like the output;
                                  0: one row per thread (default)                          */
    int32_t argmin_tables;     /* 0: argmin tables are written where the VALUE phase reads
                                  them: BE and DPOP (Algorithm 1, Section 4.1).  The value
                                  step of Algorithm 2 re-minimises over the functions of
                                  each bucket and reads none, so a mini-bucket plan leaves
                                  them out where the kernel has variants without them
                                  (fp32 costs, domains 2-4, at most 7 inputs) and writes
                                  the others unread.  The sum-product writes none.
                                  1: every min-sum task writes its table (to inspect with
                                  util_fetch_table)                                     */
} solve_opts;

/* Result of a solve.  assignment, when non-NULL, is caller-owned host memory
 * of n_vars int32 and receives the VALUE-phase assignment.  For WCSP_INT32_SAT
 * the costs are integers held exactly in double; top_k means infeasible. */
typedef struct solve_result {
    double bound;           /* sum of the root constants: the optimum (BE, DPOP) or a
                               lower bound (MBE, Section 2.2)                       */
    double cost;            /* Eq. 1 cost of the returned assignment (an upper bound
                               for MBE)                                             */
    int32_t *assignment;    /* in: caller buffer or NULL                            */
    int32_t induced_width;  /* largest separator of the run                         */
    int32_t n_tasks;        /* (mini-)buckets computed                              */
    int32_t n_levels;       /* elimination-tree levels                              */
    int32_t n_launches;     /* UTIL kernel launches of one run                      */
    int64_t util_entries;   /* sum over tasks of separator rows x |D_x| (joint rows) */
    int64_t alg_bytes;      /* 4 x input entries + 4 x output entries, over tasks,
                               + 1 x output entries of the tasks that write an
                               argmin table (see solve_opts.argmin_tables)          */
    double plan_ms;         /* host planning time                                   */
    double util_ms;         /* device time of the UTIL phase (CUDA events)          */
    double value_ms;        /* device time of the VALUE phase                       */
} solve_result;

/* Planning summary, available right after util_plan (no GPU needed). */
typedef struct gpube_plan_info {
    int32_t n_vars, n_tasks, n_levels, induced_width;
    int64_t util_entries, out_entries, in_entries, alg_bytes;
    size_t arena_bytes;       /* device memory one state needs                  */
    size_t peak_live_bytes;   /* its part that is live at the same time         */
    int32_t max_sep;          /* largest separator                              */
    int32_t max_inputs;       /* most functions in one (mini-)bucket            */
    int32_t n_argmin_tables;  /* (mini-)buckets that write an argmin table      */
} gpube_plan_info;

/* One planned (mini-)bucket, for inspection and tests (no GPU needed).
 * sep and inputs are caller buffers of at least n_vars and
 * (max_inputs of gpube_plan_info) entries.  Input ids: original functions
 * are 0..n_funcs-1; the output of task t has id n_funcs + t. */
typedef struct gpube_task_info {
    int32_t var, level, n_sep, n_inputs;
    int64_t rows;           /* separator rows = entries of the output table */
    int32_t *sep;           /* out: separator, descending elimination position */
    int32_t *inputs;        /* out: input ids, in kernel input order */
    /* out: work decomposition (rows = groups x r0 x lo_extent); inputs
     * [0, n_lo) depend on the lowest separator digits only, [n_lo, n_group)
     * are read once per group, [n_group, n_uonly) depend on the fastest hi
     * digit only, the rest are read per row; argmin = 1 when the task
     * writes its argmin table */
    int64_t lo_extent, groups;
    int32_t r0, n_lo, n_group, n_uonly, staged_bytes, argmin;
} gpube_task_info;

typedef struct wcsp wcsp;             /* opaque, library-owned problem         */
typedef struct util_state util_state; /* opaque, library-owned plan + tables    */

/* ----------------------------------------------------------- problem calls */

/* Copy and validate a problem (Sections 2-4).  EINVAL on a malformed
 * description (bad domain, repeated scope variable, wrong table length,
 * negative cost, ...).  The caller keeps ownership of d's arrays. */
int wcsp_load(const wcsp_desc *d, wcsp **out);
/* Release the caller's hold on a problem (a server request still using it
 * keeps it alive until it no longer needs it).  States made from w
 * (util_plan and the solvers) must be freed first. */
void wcsp_free(wcsp *w);
const char *wcsp_last_error(void);
void solve_opts_init(solve_opts *o);

/* ------------------------------------------------------ one-call solvers */

/* Bucket Elimination (Algorithm 1): UTIL phase on the GPU along the order of
 * opts, root reduction, VALUE phase (argmin lookups), result to the host. */
int be_solve(wcsp *w, const solve_opts *opts, solve_result *res);

/* Mini-Bucket Elimination (Algorithm 2) with bound i_bound read in
 * opts->ibound_mode.  res->bound is the lower bound; the assignment picks,
 * per variable, the first argmin of the sum of all functions of its bucket. */
int mbe_solve(wcsp *w, int32_t i_bound, const solve_opts *opts, solve_result *res);

/* Sum-product (the weighted-counting / partition-function / probability-of-
 * evidence problem that the paper's conclusions name as the extension of
 * this work; solution counting, Section 2.1).  The buckets are BE's
 * (i_bound <= 0) or Algorithm 2's mini-buckets (i_bound > 0, read in
 * opts->ibound_mode); each variable is eliminated by -log sum_l exp(-s_l)
 * in fp32 instead of min.  res->bound receives -log Z, where
 *   WCSP_FP32_LOG:  Z = sum over all assignments of exp(-Eq. 1 cost), so for
 *                   a Bayesian network with evidence clamped by 0 / +inf unary
 *                   tables, Z is the probability of the evidence;
 *   WCSP_INT32_SAT: Z = the number of assignments in which no function is at
 *                   the top cost (each entry < top_k counts as weight 1, the
 *                   others as weight 0), so exp(-bound) counts solutions.
 * A variable in no function contributes a factor |D| to Z.  With mini-buckets
 * the bound is a lower bound on -log Z (each mini-bucket summed on its own
 * can only enlarge Z).  There is no value phase: res->cost is NaN and
 * res->assignment is not written, and no argmin tables are written.  +inf
 * means Z = 0. */
int logz_solve(wcsp *w, int32_t i_bound, const solve_opts *opts, solve_result *res);

/* DPOP UTIL phase (Section 4.1) along the pseudo-tree parent[] (host, n
 * entries, -1 = root; NULL = the library's DFS pseudo-tree).  Every
 * constraint must join an ancestor and a descendant of parent[] (EINVAL
 * otherwise).  On success *out holds the UTIL messages on the device; call
 * value_propagate for the VALUE phase and util_state_free afterwards. */
int dpop_util(wcsp *w, const int32_t *parent, const solve_opts *opts, util_state **out);

/* VALUE phase (Algorithm 1/2 value assignment, DPOP VALUE propagation) over a
 * state whose UTIL phase has run.  assignment (host, n) may be NULL. */
int value_propagate(util_state *s, int32_t *assignment, solve_result *res);

void util_state_free(util_state *s);

/* ------------------------------------------------------ staged interface */

/* Host planning only (ordering, buckets, mini-bucket partition, levels,
 * kernel work decomposition); no GPU needed.  kind: enum gpube_kind;
 * i_bound is used by GPUBE_KIND_MBE and GPUBE_KIND_SUM_MBE; parent by
 * GPUBE_KIND_DPOP.  For the sum-product kinds util_value_launch performs the
 * root reduction only (bound = -log Z, as logz_solve). */
int util_plan(wcsp *w, int32_t kind, int32_t i_bound, const int32_t *parent,
              const solve_opts *opts, util_state **out);
int util_plan_info(const util_state *s, gpube_plan_info *info);
int util_task_info(const util_state *s, int32_t t, gpube_task_info *info);
/* The elimination order of the plan (host, n entries). */
int util_order(const util_state *s, int32_t *order);

/* Bind device memory (arena == NULL: the library allocates) and upload the
 * tables and the kernel plan.  Must precede util_run. */
int util_bind(util_state *s, void *arena, size_t arena_bytes, void *stream);

/* Run the UTIL phase on the bound stream (asynchronous: returns after the
 * launches are queued).  Re-runnable: every run recomputes all tables. */
int util_run(util_state *s);

/* Queue the VALUE phase (root reduction, assignment, Eq. 1 cost of the
 * assignment) on the device; value_propagate = value_launch + copy back. */
int util_value_launch(util_state *s);

/* Wait for the bound stream and report a device-side status (ETIMEDOUT if a
 * bounded wait gave up). */
int util_sync(util_state *s);

/* Copy one task's output (cost table and argmin table, rows entries each) to
 * host buffers (either may be NULL); synchronous.  For a task that writes no
 * argmin table (solve_opts.argmin_tables) arg_host receives zeros. */
int util_fetch_table(util_state *s, int32_t t, void *cost_host, uint8_t *arg_host);

/* The launch configuration of a state (what util_autotune chooses). */
typedef struct gpube_launch_config {
    int32_t block_threads;     /* UTIL kernel CTA size                                    */
    int32_t rows_per_item;     /* separator rows of one work item per thread (target)     */
    int32_t lo_target;         /* minimum extent of a work item's inner row block         */
    int32_t stage_max_entries; /* tables up to this many entries staged in shared memory (0: none) */
    int32_t pipeline;          /* 1: a task's group input is prefetched by the per-thread
                                  cp.async pipeline (4-12 groups in flight) where the task
                                  allows it; 0: register variants (1-2 groups in flight)  */
    int32_t launch_mode;       /* solve_opts.batched: 0 per bucket, 1 per level, 2 fused  */
    int32_t vector_rows;       /* 1: four consecutive rows per thread where a task allows it */
} gpube_launch_config;

/* Measure candidate launch configurations on this state's own UTIL phase and
 * keep the fastest (each candidate: the median of enough runs for about 4 ms
 * of timing): CTA size x rows per item, then the lo extent target, then two
 * passes over the launch mode with every lo target (per level or one launch
 * over all levels; a per-bucket state keeps its mode), the staging limit with
 * the group-input pipeline on and off, the four-rows-per-thread variant, the
 * launch shape and the lo target, each varied around the best so far; the
 * three fastest are timed again with three times the runs.  Changing
 * the lo target or the staging limit re-shapes the tasks and rebuilds the
 * offset tables in the bound arena (candidates that do not fit it are
 * skipped); the tables computed by later runs are unchanged (bit for bit for
 * integer costs).  The choice is appended to opts.autotune_cache when given
 * and read back from it for the same plan.  Writes the chosen CTA size and
 * rows per item to *threads and *rows_per_item (either may be NULL); the
 * whole configuration is available from util_launch_config. */
int util_autotune(util_state *s, int32_t *threads, int32_t *rows_per_item);
int util_launch_config(const util_state *s, gpube_launch_config *out);

/* Conditioning: clamp variables to values for the following runs of the same
 * plan, without planning or binding again (evidence in a Bayesian network,
 * Section 3; the repeated mini-bucket bounds of a search that conditions on
 * partial assignments, Section 9).  Each variable must be one of the
 * evidence_vars the plan was made with: the plan holds, per such variable, a
 * unary function in that variable's bucket, all zero while the variable is
 * free; clamping x_v to a sets it to 0 at a and to the top cost (fp32:
 * +inf) elsewhere.  vals[i] = -1 frees vars[i]; variables not listed keep
 * their state.  On a bound state the new tables are copied on the bound
 * stream (ordered after the work already queued there), so the next
 * util_run uses them, graph replays included.  EINVAL for an undeclared
 * variable or a value outside its domain (nothing is changed then). */
int util_condition(util_state *s, int32_t n, const int32_t *vars, const int32_t *vals);

/* Device time in ms of the last util_run / VALUE phase (after util_sync). */
int util_last_times(util_state *s, double *util_ms, double *value_ms);

/* ---------------------------------------------------- single-bucket kernel */

/* One (mini-)bucket on the GPU: the fused aggregation + elimination of
 * Section 6.3-6.4 (Procedures Gpu::Aggregate, Gpu::Eliminate), also writing
 * the first argmin.  The joint scope is m separator variables (domains
 * sep_dom[0..m-1], host) followed by the eliminated variable (domain d).
 * Input i is a device table row-major over its scope: the separator
 * variables at positions in_pos[in_pos_off[i] .. in_pos_off[i+1]) (host,
 * ascending, each in 0..m-1) followed by the eliminated variable.  in_tables
 * (host array of n_in device pointers, 16-byte aligned) point to int32
 * (WCSP_INT32_SAT) or float (WCSP_FP32_LOG) data.  out (device, rows
 * entries of the same type) and arg (device, rows bytes) receive the
 * bucket function and its argmin, rows = product of sep_dom.  Scratch
 * (plan tables) comes from a per-device buffer the library keeps and grows
 * with cudaMalloc.  Asynchronous on stream. */
int util_bucket(int32_t cost_type, int32_t top_k, int32_t m, const int32_t *sep_dom, int32_t d,
                int32_t n_in, const void *const *in_tables, const int32_t *in_pos_off,
                const int32_t *in_pos, void *out, uint8_t *arg, void *stream);

/* The same single-bucket computation for callers that cannot allocate
 * device memory: loops that forbid allocation once they run (an allocation
 * may block or fail at a moment nobody chose), and processes whose device
 * memory is entirely owned by another allocator (a framework's caching
 * allocator, a pre-reserved pool), where a cudaMalloc from this library
 * would compete for memory that allocator does not know about.  The paper
 * has no counterpart; it is a service of this library.  Its scratch (offset
 * tables, descriptors, work counter) is a fixed 4 MiB array inside the
 * library, present on every device the library is used on from load until
 * process exit; nothing is allocated and nothing is freed.  Arguments as
 * util_bucket.  A bucket whose scratch would exceed the array fails with
 * GPUBE_ENOMEM before any CUDA call (util_bucket takes it;
 * util_bucket_scratch_bytes tells beforehand).  The first call on a device,
 * with that device current, looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the process: after cudaDeviceReset
 * that address is stale and the entry point must not be called again.  All
 * calls share the array and it keeps the last call's contents (each call
 * clears its counter and status first): calls that may overlap on the GPU
 * (different streams, or threads) race and must be serialised by the
 * caller.  Asynchronous on stream. */
int util_bucket_noalloc(int32_t cost_type, int32_t top_k, int32_t m, const int32_t *sep_dom, int32_t d,
                        int32_t n_in, const void *const *in_tables, const int32_t *in_pos_off,
                        const int32_t *in_pos, void *out, uint8_t *arg, void *stream);

/* Scratch bytes util_bucket and util_bucket_noalloc need for a bucket of
 * this shape (arguments as util_bucket, without tables), into *bytes, and
 * the size of util_bucket_noalloc's fixed array into *noalloc_limit (may be
 * NULL).  Host only: no CUDA call, no GPU needed.  EINVAL on a malformed
 * shape, ENOMEM when the output would exceed 2^31 entries.  The paper has
 * no counterpart. */
int util_bucket_scratch_bytes(int32_t m, const int32_t *sep_dom, int32_t d, int32_t n_in,
                              const int32_t *in_pos_off, const int32_t *in_pos, size_t *bytes,
                              size_t *noalloc_limit);

/* Diagnostic: launch one CTA that waits, with the same time-bounded wait the
 * UTIL kernel uses on its TMA barriers, on a barrier that nothing completes.
 * Returns GPUBE_ETIMEDOUT after about timeout_ns (the failure path ends in a
 * status, not a hang or a trap; the context stays usable), GPUBE_ECUDA on a
 * CUDA error.  Synchronous on stream.  The paper has no counterpart. */
int util_selftest_wait(uint64_t timeout_ns, void *stream);

/* Diagnostic: one thread runs the wait of a launch over all levels
 * (solve_opts.batched = 2) for a producing bucket that never completes.
 * Returns GPUBE_ETIMEDOUT after about timeout_ns, GPUBE_ECUDA on a CUDA
 * error; the context stays usable.  Synchronous on stream.  The paper has
 * no counterpart. */
int util_selftest_dep_wait(uint64_t timeout_ns, void *stream);

/* ---------------------------------------------------------------- serving */

/* A continuous-batching server for streams of problems (DCOP or WCSP) on one
 * GPU.  Requests are admitted while their device-memory need (from the plan,
 * before any allocation) fits in budget_bytes and a slot is free; the
 * elimination-tree levels of all admitted requests are merged into shared
 * persistent launches, so requests that arrive while others run join the
 * next launch.  The arena (device, arena_bytes >= budget_bytes) is the
 * caller's; NULL = the library allocates budget_bytes. */
typedef struct gpube_server gpube_server;

int srv_create(size_t budget_bytes, int32_t max_slots, void *arena, size_t arena_bytes,
               void *stream, gpube_server **out);
/* Submit a problem (kind as in util_plan): copies parent[] and the options'
 * arrays, takes a reference to the problem (wcsp_free may be called right
 * away; the problem is released once no request needs it) and queues the
 * request for the server's planner threads, which plan requests in parallel
 * with each other and with srv_step.  Returns a request id >= 0, or EINVAL.
 * A request whose plan fails, or that can never fit the budget (ENOMEM),
 * ends in that status (srv_result returns it). */
int64_t srv_submit(gpube_server *s, wcsp *w, int32_t kind, int32_t i_bound,
                   const int32_t *parent, const solve_opts *opts);
/* Advance the server by one iteration: take finished plans, admit what
 * fits, launch one merged level step, retire finished requests.  Returns the
 * number of requests still being planned, queued or in flight. */
int srv_step(gpube_server *s);
/* Result of a finished request: 0 with res filled (assignment copied when
 * non-NULL), EAGAIN if not finished. */
int srv_result(gpube_server *s, int64_t id, int32_t *assignment, solve_result *res);
/* Host times of a finished request (seconds on the server's monotonic
 * clock): submit, admit, done. */
int srv_times(gpube_server *s, int64_t id, double *t_submit, double *t_admit, double *t_done);
int srv_stats(gpube_server *s, int64_t *launches, int64_t *peak_bytes, int64_t *max_inflight);
void srv_free(gpube_server *s);

#ifdef __cplusplus
}
#endif

#endif /* GPUBE_H */
