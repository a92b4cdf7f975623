// C ABI of the library (include/gpube.h): problem loading, planning, arena
// layout, upload, launches (plain per bucket, or batched per elimination-tree
// level, optionally captured once in a CUDA graph), the VALUE phase, and the
// one-call solvers of Algorithms 1-2 and DPOP.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <fstream>
#include <map>
#include <mutex>
#include <numeric>
#include <sstream>
#include <string>

#include "gpube_internal.h"

using namespace gpube;

double gpube::now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

namespace {

size_t al(size_t x, size_t a) { return (x + a - 1) / a * a; }

#define CUDA_TRY(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);    \
    } while (0)

// Sequential byte layout with alignment.
struct Cursor {
    size_t off = 0;
    size_t take(size_t bytes, size_t align = 16)
    {
        off = al(off, align);
        size_t r = off;
        off += bytes;
        return r;
    }
};

}  // namespace

static DescLayout &layout_of(util_state *s) { return s->dl; }
static const DescLayout &layout_of(const util_state *s) { return s->dl; }

// ------------------------------------------------------------------ misc
extern "C" const char *wcsp_last_error(void) { return gpube::last_error(); }

extern "C" void solve_opts_init(solve_opts *o)
{
    memset(o, 0, sizeof(*o));
    o->order_kind = GPUBE_ORDER_MINFILL;
    o->ibound_mode = GPUBE_IB_SEP_VARS;
    o->batched = 1;
    o->use_graph = 0;
}

// ---------------------------------------------------------------- problem
extern "C" int wcsp_load(const wcsp_desc *d, wcsp **out)
{
    if (!d || !out) return set_error(GPUBE_EINVAL, "null argument");
    *out = nullptr;
    if (d->n_vars < 0 || d->n_funcs < 0) return set_error(GPUBE_EINVAL, "negative sizes");
    if (d->cost_type != WCSP_INT32_SAT && d->cost_type != WCSP_FP32_LOG)
        return set_error(GPUBE_EINVAL, "unknown cost type %d", d->cost_type);
    if (d->cost_type == WCSP_INT32_SAT && d->top_k < 1)
        return set_error(GPUBE_EINVAL, "top_k must be in [1, 2^31-1]");
    if (d->n_vars > 0 && !d->dom) return set_error(GPUBE_EINVAL, "dom is NULL");
    if (d->n_funcs > 0 && (!d->scope_off || !d->tab_off || !d->costs))
        return set_error(GPUBE_EINVAL, "function arrays are NULL");
    wcsp *w = new wcsp();
    w->n = d->n_vars;
    w->nf = d->n_funcs;
    w->cost_type = d->cost_type;
    w->top_k = static_cast<uint32_t>(d->cost_type == WCSP_INT32_SAT ? d->top_k : 1);
    w->dom.assign(d->dom, d->dom + d->n_vars);
    for (int v = 0; v < w->n; ++v)
        if (w->dom[v] < 1 || w->dom[v] > 255) {
            delete w;
            return set_error(GPUBE_EINVAL, "domain of variable %d is %d (must be 1..255)", v, d->dom[v]);
        }
    w->scope.resize(w->nf);
    if (w->cost_type == WCSP_INT32_SAT) w->itab.resize(w->nf);
    else w->ftab.resize(w->nf);
    w->adj.assign(w->n, {});
    if (d->n_funcs > 0 && d->scope_off[0] != 0) {
        delete w;
        return set_error(GPUBE_EINVAL, "scope_off[0] must be 0");
    }
    for (int j = 0; j < w->nf; ++j) {
        const int32_t a = d->scope_off[j], b = d->scope_off[j + 1];
        if (b < a || (b > a && !d->scope)) {
            delete w;
            return set_error(GPUBE_EINVAL, "bad scope offsets of function %d", j);
        }
        std::vector<int32_t> s(d->scope + a, d->scope + b);
        int64_t size = 1;
        for (size_t x = 0; x < s.size(); ++x) {
            if (s[x] < 0 || s[x] >= w->n) {
                delete w;
                return set_error(GPUBE_EINVAL, "function %d mentions variable %d", j, s[x]);
            }
            for (size_t y = 0; y < x; ++y)
                if (s[x] == s[y]) {
                    delete w;
                    return set_error(GPUBE_EINVAL, "function %d repeats variable %d", j, s[x]);
                }
            size *= w->dom[s[x]];
            if (size > INT32_MAX) {
                delete w;
                return set_error(GPUBE_ENOMEM, "table of function %d has more than 2^31 entries", j);
            }
        }
        const int64_t t0 = d->tab_off[j], t1 = d->tab_off[j + 1];
        if (t1 - t0 != size) {
            delete w;
            return set_error(GPUBE_EINVAL, "function %d: table has %lld entries, scope needs %lld", j,
                             static_cast<long long>(t1 - t0), static_cast<long long>(size));
        }
        if (w->cost_type == WCSP_INT32_SAT) {
            const int32_t *c = static_cast<const int32_t *>(d->costs) + t0;
            auto &t = w->itab[j];
            t.resize(size);
            for (int64_t i = 0; i < size; ++i) {
                if (c[i] < 0) {
                    delete w;
                    return set_error(GPUBE_EINVAL, "function %d has a negative cost", j);
                }
                t[i] = static_cast<uint32_t>(c[i]) > w->top_k ? static_cast<int32_t>(w->top_k) : c[i];
            }
        } else {
            const float *c = static_cast<const float *>(d->costs) + t0;
            auto &t = w->ftab[j];
            t.assign(c, c + size);
            for (float x : t)
                if (!(x >= 0.0f)) {
                    delete w;
                    return set_error(GPUBE_EINVAL, "function %d has a negative or NaN cost", j);
                }
        }
        for (int32_t x : s)
            for (int32_t y : s)
                if (x != y) w->adj[x].push_back(y);
        w->scope[j] = std::move(s);
    }
    for (auto &a : w->adj) {
        std::sort(a.begin(), a.end());
        a.erase(std::unique(a.begin(), a.end()), a.end());
    }
    *out = w;
    return GPUBE_OK;
}

extern "C" void wcsp_free(wcsp *w) { wcsp_unref(w); }

// ---------------------------------------------------------------- planning
static std::vector<int32_t> row_strides(const wcsp &w, const std::vector<int32_t> &scope)
{
    std::vector<int32_t> st(scope.size());
    int64_t s = 1;
    for (int k = static_cast<int>(scope.size()) - 1; k >= 0; --k) {
        st[k] = static_cast<int32_t>(s);
        s *= w.dom[scope[k]];
    }
    return st;
}

// VALUE plan: per variable, the argmin table of its bucket (BE, DPOP) or all
// functions of its bucket (MBE); variables grouped by dependency level.
static void build_value_plan(const wcsp &w, Plan &P)
{
    const int n = w.n;
    ValuePlanH &V = P.value;
    V = ValuePlanH();
    if (kind_sum(P.kind)) {
        // sum-product: no assignment and no Eq. 1 evaluation, only the sum
        // of the root constants (-log Z of each component)
        V.n_levels = 0;
        V.lev_off.assign(1, 0);
        V.vinfo.assign(n, ValueVar{0, 1, 0, 0});
        for (int v = 0; v < n; ++v) V.vinfo[v].d = w.dom[v];
        for (const Task &T : P.tasks)
            if (T.sep.empty()) V.roots.push_back(T.out_off);
        return;
    }
    std::vector<std::vector<int32_t>> tasks_of(n);
    for (size_t t = 0; t < P.tasks.size(); ++t) tasks_of[P.tasks[t].var].push_back(static_cast<int32_t>(t));
    std::vector<int32_t> vlev(n, 0);
    int maxlev = -1;
    for (int t = n - 1; t >= 0; --t) {
        const int v = P.order[t];
        int lev = 0;
        for (int tk : tasks_of[v])
            for (int u : P.tasks[tk].sep) lev = std::max(lev, vlev[u] + 1);
        vlev[v] = lev;
        maxlev = std::max(maxlev, lev);
    }
    V.n_levels = maxlev + 1;
    V.lev_off.assign(V.n_levels + 1, 0);
    for (int v = 0; v < n; ++v) V.lev_off[vlev[v] + 1]++;
    for (int l = 0; l < V.n_levels; ++l) V.lev_off[l + 1] += V.lev_off[l];
    std::vector<int32_t> fillp(V.lev_off.begin(), V.lev_off.end() - 1);
    V.vorder.assign(n, 0);
    for (int t = n - 1; t >= 0; --t) {
        const int v = P.order[t];
        V.vorder[fillp[vlev[v]]++] = v;
    }
    V.vinfo.assign(n, ValueVar{0, 1, 0, 0});
    for (int v = 0; v < n; ++v) {
        ValueVar &vi = V.vinfo[v];
        vi.d = w.dom[v];
        if (tasks_of[v].empty()) continue;
        vi.term_off = static_cast<int32_t>(V.terms.size());
        if (!kind_mbe(P.kind)) {
            const Task &T = P.tasks[tasks_of[v][0]];
            vi.mode = 1;
            vi.n_terms = 1;
            ValueTermH th{T.arg_off, static_cast<int32_t>(T.sep.size()), static_cast<int32_t>(V.vvars.size())};
            std::vector<int32_t> st = row_strides(w, T.sep);
            V.vvars.insert(V.vvars.end(), T.sep.begin(), T.sep.end());
            V.vstrides.insert(V.vstrides.end(), st.begin(), st.end());
            V.terms.push_back(th);
        } else {
            vi.mode = 2;
            for (int tk : tasks_of[v])
                for (int fid : P.tasks[tk].inputs) {
                    const Func &f = P.funcs[fid];
                    std::vector<int32_t> st = row_strides(w, f.scope);
                    const int nv = static_cast<int>(f.scope.size()) - 1;  // v is last
                    ValueTermH th{f.off, nv, static_cast<int32_t>(V.vvars.size())};
                    V.vvars.insert(V.vvars.end(), f.scope.begin(), f.scope.begin() + nv);
                    V.vstrides.insert(V.vstrides.end(), st.begin(), st.begin() + nv);
                    V.terms.push_back(th);
                    vi.n_terms++;
                }
        }
    }
    for (int j = 0; j < w.nf; ++j) {
        const Func &f = P.funcs[j];
        if (f.scope.empty() || f.ext) continue;
        std::vector<int32_t> st = row_strides(w, f.scope);
        ValueTermH th{f.off, static_cast<int32_t>(f.scope.size()), static_cast<int32_t>(V.vvars.size())};
        V.vvars.insert(V.vvars.end(), f.scope.begin(), f.scope.end());
        V.vstrides.insert(V.vstrides.end(), st.begin(), st.end());
        V.evals.push_back(th);
    }
    for (const Task &T : P.tasks)
        if (T.sep.empty()) V.roots.push_back(T.out_off);
}

// Arena layout: originals | bucket functions | argmins | A/B tables |
// descriptors | value plan | counters, status, result, assignment.
void gpube_layout(util_state *s)
{
    const wcsp &w = *s->w;
    Plan &P = s->plan;
    Cursor c;
    for (int j = 0; j < w.nf; ++j)
        if (!P.funcs[j].scope.empty() && !P.funcs[j].ext) P.funcs[j].off = c.take(P.funcs[j].size * 4, 16);
    c.off = al(c.off, 256);
    s->upload_bytes = c.off;
    // (tables the caller owns, single-bucket calls, take no arena space)
    for (size_t t = 0; t < P.tasks.size(); ++t) {
        Task &T = P.tasks[t];
        T.out_off = T.ext_out ? 0 : c.take(T.rows * 4, 128);
        P.funcs[w.nf + t].off = T.out_off;
    }
    for (Task &T : P.tasks) T.arg_off = (T.ext_arg || !T.keep_arg) ? 0 : c.take(T.rows, 128);
    for (Task &T : P.tasks) {
        T.A_off = c.take(static_cast<size_t>(T.G + 1) * T.sa * 4, 128);
        T.B_off = c.take(static_cast<size_t>(T.P_lo) * T.sb * 4, 128);
    }
    // the value plan refers to table offsets, so it is built after them
    build_value_plan(w, P);
    DescLayout &D = layout_of(s);
    const size_t nt = P.tasks.size();
    D.n_in = 0;
    D.n_pool = 0;
    for (const Task &T : P.tasks) {
        D.n_in += T.inputs.size();
        const size_t m = T.sep.size();
        D.n_pool += m + T.hperm.size() + (T.inputs.size() + 1) * m;
    }
    D.n_prefix = 3 * nt + P.n_levels + 2;
    c.off = al(c.off, 256);
    s->desc_off = c.off;
    D.taskdev = c.take(sizeof(TaskDev) * nt, 16);
    D.indev = c.take(sizeof(InDev) * D.n_in, 16);
    D.prefix = c.take(4 * D.n_prefix, 16);
    D.expand = c.take(sizeof(ExpandDev) * nt, 16);
    D.exp_prefix = c.take(8 * (nt + 1), 16);
    D.pool = c.take(4 * D.n_pool, 16);
    D.dep_off = c.take(4 * (nt + 1), 16);
    D.deps = c.take(4 * std::max<size_t>(D.n_in, 1), 16);
    s->desc_bytes = c.off - s->desc_off;
    const ValuePlanH &V = P.value;
    s->value_off = al(c.off, 16);
    D.lev_off = c.take(4 * V.lev_off.size(), 16);
    D.vorder = c.take(4 * V.vorder.size(), 16);
    D.vinfo = c.take(sizeof(ValueVar) * V.vinfo.size(), 16);
    D.terms = c.take(sizeof(ValueTerm) * V.terms.size(), 16);
    D.vvars = c.take(4 * V.vvars.size(), 16);
    D.vstrides = c.take(4 * V.vstrides.size(), 16);
    D.evals = c.take(sizeof(ValueTerm) * V.evals.size(), 16);
    D.roots = c.take(8 * V.roots.size(), 16);
    s->value_bytes = c.off - s->value_off;
    // queue heads (one per launch), or one head and a completion count per
    // task for a launch over all levels
    const size_t n_counters = std::max<size_t>(std::max<size_t>(nt + 1, P.n_levels), 1);
    s->counters_off = c.take(4 * n_counters, 256);
    s->status_off = c.take(8, 16);
    s->result_off = s->status_off + 8;
    c.off = s->result_off;
    c.take(16, 8);
    s->sigma_off = c.take(4 * std::max(w.n, 1), 4);
    s->work_off = s->counters_off;
    s->arena_bytes = al(c.off, 256);
    // live bytes: the largest footprint along the plain order when the cost
    // tables of BE / DPOP messages are released once their bucket is done
    size_t fixed = s->upload_bytes + (s->arena_bytes - s->desc_off);
    size_t live = fixed, peak = fixed;
    for (const Task &T : P.tasks)
        live += (T.keep_arg ? al(T.rows, 128) : 0) + al((T.G + 1) * T.sa * 4, 128) + al(T.P_lo * T.sb * 4, 128);
    peak = live;
    for (const Task &T : P.tasks) {
        live += al(T.rows * 4, 128);
        peak = std::max(peak, live);
        if (!kind_mbe(P.kind))
            for (int fid : T.inputs)
                if (P.funcs[fid].task >= 0) live -= al(P.funcs[fid].size * 4, 128);
    }
    P.peak_live_bytes = peak;
}

extern "C" int util_plan(wcsp *w, int32_t kind, int32_t i_bound, const int32_t *parent, const solve_opts *opts,
                         util_state **out)
{
    if (!w || !out) return set_error(GPUBE_EINVAL, "null argument");
    *out = nullptr;
    if (kind < GPUBE_KIND_BE || kind > GPUBE_KIND_SUM_MBE) return set_error(GPUBE_EINVAL, "unknown kind %d", kind);
    solve_opts o;
    if (opts) o = *opts;
    else solve_opts_init(&o);
    const double t0 = now_ms();
    if (o.n_evidence_vars < 0 || (o.n_evidence_vars > 0 && !o.evidence_vars))
        return set_error(GPUBE_EINVAL, "bad evidence_vars");
    {
        std::vector<char> seen(w->n, 0);
        for (int i = 0; i < o.n_evidence_vars; ++i) {
            const int v = o.evidence_vars[i];
            if (v < 0 || v >= w->n || seen[v]) return set_error(GPUBE_EINVAL, "evidence variable %d", v);
            seen[v] = 1;
        }
    }
    util_state *s = new util_state();
    s->w = w;
    s->ktype = w->cost_type == WCSP_FP32_LOG ? kKTypeFloat : kKTypeInt;
    if (kind_sum(kind)) {
        s->ktype = kKTypeSum;
        if (w->cost_type == WCSP_INT32_SAT) {
            // solution counting: weight 1 (-log 0) below the top cost, weight 0
            // (+inf) at it
            s->own_w.reset(new wcsp(*w));
            wcsp &c = *s->own_w;
            c.cost_type = WCSP_FP32_LOG;
            c.top_k = 1;
            c.ftab.resize(c.nf);
            for (int j = 0; j < c.nf; ++j) {
                c.ftab[j].resize(c.itab[j].size());
                for (size_t e = 0; e < c.itab[j].size(); ++e)
                    c.ftab[j][e] = static_cast<uint32_t>(c.itab[j][e]) >= w->top_k ? INFINITY : 0.0f;
            }
            c.itab.clear();
            c.itab.shrink_to_fit();
            s->w = &c;
        }
    }
    if (o.n_evidence_vars > 0) {
        // one unary function per evidence variable, appended after the
        // problem's functions, all zero (free) until util_condition
        if (!s->own_w) s->own_w.reset(new wcsp(*w));
        wcsp &c = *s->own_w;
        s->ev_fid0 = c.nf;
        for (int i = 0; i < o.n_evidence_vars; ++i) {
            const int v = o.evidence_vars[i];
            c.scope.push_back({v});
            if (c.cost_type == WCSP_FP32_LOG) c.ftab.emplace_back(c.dom[v], 0.0f);
            else c.itab.emplace_back(c.dom[v], 0);
            s->ev_vars.push_back(v);
            s->ev_val.push_back(-1);
        }
        c.nf += o.n_evidence_vars;
        s->w = &c;
    }
    s->opts = o;
    s->opts.evidence_vars = nullptr;  // not kept: the caller owns the array
    if (o.batched < kLaunchPerTask || o.batched > kLaunchFused) {
        delete s;
        return set_error(GPUBE_EINVAL, "batched must be 0 (per bucket), 1 (per level) or 2 (all levels in one launch)");
    }
    s->launch_mode = o.batched;
    s->use_graph = o.use_graph != 0;
    s->device = o.device;
    if (o.block_threads) {
        if (o.block_threads < 32 || o.block_threads > kMaxThreads || o.block_threads % 32) {
            delete s;
            return set_error(GPUBE_EINVAL, "block_threads must be a multiple of 32 in [32, %d]", kMaxThreads);
        }
        s->cfg.threads = o.block_threads;
    }
    if (o.rows_per_item < 0) {
        delete s;
        return set_error(GPUBE_EINVAL, "rows_per_item must be >= 0");
    }
    if (o.rows_per_item) s->cfg.rows_per_item = o.rows_per_item;
    int rc = build_plan(*s->w, kind, i_bound, parent, o, s->plan);
    if (rc) {
        delete s;
        return rc;
    }
    shape_tasks(*s->w, s->plan);
    gpube_layout(s);
    if (w->n > 200 * 1024) {
        delete s;
        return set_error(GPUBE_EINVAL, "more than 204800 variables are not supported by the VALUE kernel");
    }
    s->plan_ms = now_ms() - t0;
    *out = s;
    return GPUBE_OK;
}

extern "C" int util_plan_info(const util_state *s, gpube_plan_info *info)
{
    if (!s || !info) return set_error(GPUBE_EINVAL, "null argument");
    const Plan &P = s->plan;
    info->n_vars = s->w->n;
    info->n_tasks = static_cast<int32_t>(P.tasks.size());
    info->n_levels = P.n_levels;
    info->induced_width = P.width;
    info->util_entries = P.util_entries;
    info->out_entries = P.out_entries;
    info->in_entries = P.in_entries;
    info->alg_bytes = alg_bytes_of(P);
    info->arena_bytes = s->arena_bytes;
    info->peak_live_bytes = P.peak_live_bytes;
    info->max_sep = P.width;
    info->max_inputs = P.max_inputs;
    info->n_argmin_tables = 0;
    for (const Task &T : P.tasks) info->n_argmin_tables += T.keep_arg ? 1 : 0;
    return GPUBE_OK;
}

extern "C" int util_task_info(const util_state *s, int32_t t, gpube_task_info *info)
{
    if (!s || !info) return set_error(GPUBE_EINVAL, "null argument");
    if (t < 0 || t >= static_cast<int32_t>(s->plan.tasks.size())) return set_error(GPUBE_EINVAL, "no task %d", t);
    const Task &T = s->plan.tasks[t];
    info->var = T.var;
    info->level = T.level;
    info->n_sep = static_cast<int32_t>(T.sep.size());
    info->n_inputs = static_cast<int32_t>(T.inputs.size());
    info->rows = T.rows;
    if (info->sep) std::copy(T.sep.begin(), T.sep.end(), info->sep);
    if (info->inputs) std::copy(T.inputs.begin(), T.inputs.end(), info->inputs);
    info->lo_extent = T.P_lo;
    info->groups = T.G;
    info->r0 = T.R0;
    info->n_lo = T.n_lo;
    info->n_group = T.n_gi;
    info->n_uonly = T.n_uo;
    info->staged_bytes = T.stage_bytes;
    info->argmin = T.keep_arg ? 1 : 0;
    return GPUBE_OK;
}

extern "C" int util_order(const util_state *s, int32_t *order)
{
    if (!s || !order) return set_error(GPUBE_EINVAL, "null argument");
    std::copy(s->plan.order.begin(), s->plan.order.end(), order);
    return GPUBE_OK;
}

// ------------------------------------------------------------ descriptors
// Distinct runs of input f that the first `lanes` rows of a lo chunk (one
// warp) read.  The cp.async pipeline copies every lane's run on its own, and
// copies of one global address into many lanes' slots take several
// shared-memory wavefronts each (on GB300 about 11 per instruction when 4-8
// distinct runs feed a warp), so an input that a warp reads mostly
// duplicated is read with plain loads instead, which broadcast.
static int warp_distinct_runs(const wcsp &w, const Task &T, const std::vector<int32_t> &st, int f, int lanes)
{
    const int m = static_cast<int>(T.sep.size());
    std::vector<int64_t> off(static_cast<size_t>(lanes));
    for (int lo = 0; lo < lanes; ++lo) {
        int64_t r = lo, o = 0;
        for (int j = m - 1; j >= m - T.L; --j) {
            const int dj = w.dom[T.sep[j]];
            o += (r % dj) * st[static_cast<size_t>(f) * m + j];
            r /= dj;
        }
        off[static_cast<size_t>(lo)] = o;
    }
    std::sort(off.begin(), off.end());
    return static_cast<int>(std::unique(off.begin(), off.end()) - off.begin());
}

static const void *func_ptr(const util_state *s, int fid)
{
    const Func &f = s->plan.funcs[fid];
    if (f.ext) return f.ext;
    if (f.task >= 0) {
        const Task &T = s->plan.tasks[f.task];
        if (T.ext_out) return T.ext_out;
    }
    return s->base + f.off;
}

// Rebuild the launch-configuration-dependent descriptors (TaskDev, InDev,
// work-item prefixes) and the static ones (expansion plan, value plan) into
// the host blob that mirrors [desc_off, value_off + value_bytes).
// Upper bounds of every function's entries (integer costs): an original's
// largest entry, a bucket function's min(k, sum of its inputs' bounds) (its
// entries are minima of such sums).  Tables the library cannot read (caller
// device tables) and the evidence tables (rewritten after binding) are
// bounded by k.
static std::vector<uint64_t> upper_bounds(const util_state *s)
{
    const wcsp &w = *s->w;
    const Plan &P = s->plan;
    const uint64_t k = w.top_k;
    std::vector<uint64_t> ub(P.funcs.size(), k);
    if (w.cost_type != WCSP_INT32_SAT) return ub;
    const int ev0 = s->ev_vars.empty() ? w.nf : s->ev_fid0;
    for (int j = 0; j < w.nf && j < ev0; ++j) {
        if (P.funcs[j].ext || static_cast<size_t>(j) >= w.itab.size() || w.itab[j].empty()) continue;
        uint64_t m = 0;
        for (int32_t v : w.itab[j]) m = std::max<uint64_t>(m, static_cast<uint32_t>(v));
        ub[j] = std::min(m, k);
    }
    for (size_t t = 0; t < P.tasks.size(); ++t) {  // inputs are originals or earlier tasks
        uint64_t sum = 0;
        for (int fid : P.tasks[t].inputs) sum += ub[fid];
        ub[w.nf + t] = std::min(sum, k);
    }
    return ub;
}

int gpube_build_descriptors(util_state *s)
{
    const wcsp &w = *s->w;
    Plan &P = s->plan;
    const DescLayout &D = layout_of(s);
    const size_t nt = P.tasks.size();
    const std::vector<uint64_t> ub = upper_bounds(s);
    const int NT = s->cfg.threads;
    const size_t blob_bytes = s->value_off + s->value_bytes - s->desc_off;
    s->host_blob.assign(blob_bytes, 0);
    unsigned char *hb = s->host_blob.data();
    auto at = [&](size_t off) { return hb + (off - s->desc_off); };
    unsigned char *B = s->base;
    TaskDev *td = reinterpret_cast<TaskDev *>(at(D.taskdev));
    InDev *ind = reinterpret_cast<InDev *>(at(D.indev));
    int32_t *pre = reinterpret_cast<int32_t *>(at(D.prefix));
    std::vector<int32_t> slot(nt);  // task -> index in level order
    size_t in_pos = 0;
    for (size_t i = 0; i < nt; ++i) {
        const int t = P.level_order[i];
        slot[t] = static_cast<int32_t>(i);
        const Task &T = P.tasks[t];
        TaskDev &x = td[i];
        x.A = reinterpret_cast<const int32_t *>(B + T.A_off);
        x.B = reinterpret_cast<const int32_t *>(B + T.B_off);
        x.in = reinterpret_cast<const InDev *>(B + D.indev) + in_pos;
        x.out = T.ext_out ? T.ext_out : static_cast<void *>(B + T.out_off);
        // (null only for shapes whose kernel variants leave the argmin out)
        x.arg = !T.keep_arg ? nullptr : T.ext_arg ? T.ext_arg : B + T.arg_off;
        x.F = static_cast<int32_t>(T.inputs.size());
        x.d = T.d;
        x.sa = T.sa;
        x.sb = T.sb;
        x.P_lo = static_cast<int32_t>(T.P_lo);
        x.G = static_cast<int32_t>(T.G);
        x.R0 = T.R0;
        // rows_per_item counts separator rows; an item spans whole groups
        const int64_t groups = std::max<int64_t>(1, s->cfg.rows_per_item / std::max(T.R0, 1));
        x.hc = static_cast<int32_t>(std::min<int64_t>(groups, T.G));
        // four consecutive rows per thread: domains 2..4, at most 3 inputs,
        // lo extent a multiple of 4, and (single-bucket calls) caller output
        // tables aligned for the 16-byte and 4-byte stores
        const bool out_ok = !T.ext_out || (reinterpret_cast<uintptr_t>(T.ext_out) % 16 == 0 &&
                                           reinterpret_cast<uintptr_t>(T.ext_arg) % 4 == 0);
        x.v4 = (P.allow_v4 && T.d >= 2 && T.d <= 3 && x.F <= 3 && T.P_lo % 4 == 0 && out_ok) ? 1 : 0;
        x.lin = 0;
        x.uni = 0;
        if (x.v4) {
            // input f is read in blocks when its strides of the lo digits are d
            // times the output's (its layout ends with the lo digits and x_i);
            // it has one offset per aligned block of four rows when it mentions
            // no lo digit j whose lower digits' product P_j is not a multiple of
            // 4 (exactly the digits that change inside some aligned block)
            std::vector<int32_t> st;
            task_strides(w, P, T, st);
            const int m = static_cast<int>(T.sep.size());
            for (int f = 0; f < x.F; ++f) {
                bool lin = true, uni = true;
                int64_t pj = 1;
                for (int j = m - 1; j >= m - T.L; --j) {
                    const int64_t sf = st[static_cast<size_t>(f) * m + j];
                    lin = lin && sf == static_cast<int64_t>(T.d) * st[static_cast<size_t>(x.F) * m + j];
                    if (sf != 0 && pj % 4 != 0) uni = false;
                    pj *= w.dom[T.sep[j]];
                }
                if (lin) x.lin |= 1 << f;
                else if (uni) x.uni |= 1 << f;
            }
        }
        // lo chunks: NT rows (one per thread), 4 NT rows (four per thread), or
        // NT / 32 rows for wide domains (one per warp)
        const int64_t chunk = dclass_of(T.d) == kDClassWide ? NT / 32 : x.v4 ? 4 * NT : NT;
        x.nlc = static_cast<int32_t>((T.P_lo + chunk - 1) / chunk);
        const int64_t items = static_cast<int64_t>(x.nlc) * ((T.G + x.hc - 1) / x.hc);
        if (items > INT32_MAX / 2) return set_error(GPUBE_ENOMEM, "task %d has too many work items", t);
        x.n_items = static_cast<int32_t>(items);
        x.variant = dclass_of(T.d) * kNumFClass + fclass_of(x.F);
        x.stage_bytes = T.stage_bytes;
        x.cin = 1;
        for (size_t f = 0; f < T.inputs.size(); ++f)
            if (T.stage_off[f] >= 0 && P.funcs[T.inputs[f]].task >= 0) x.cin = 0;
        x.n_lo = T.n_lo;
        x.n_gi = T.n_gi;
        // one global group input, at most 3 inputs, a fixed-domain variant:
        // prefetch that input with the per-thread cp.async pipeline, unless
        // a warp's lanes mostly read the same runs of it
        x.pipe = (!x.v4 && P.allow_pipe && x.F <= 3 && T.d >= 2 && T.d <= 8 && T.n_gi - T.n_lo == 1 && T.stage_off[T.n_lo] < 0 &&
                  T.G > 1)
                     ? 1
                     : 0;
        if (x.pipe) {
            std::vector<int32_t> st;
            task_strides(w, P, T, st);
            const int lanes = static_cast<int>(std::min<int64_t>(32, T.P_lo));
            if (2 * warp_distinct_runs(w, T, st, T.n_lo, lanes) < lanes) x.pipe = 0;
        }
        x.n_uo = T.n_uo;
        uint64_t sum_ub = 0;
        for (int fid : T.inputs) sum_ub += ub[fid];
        x.nosat = (w.cost_type == WCSP_INT32_SAT && sum_ub < w.top_k && sum_ub < (1ull << 30)) ? 1 : 0;
        for (size_t f = 0; f < T.inputs.size(); ++f) {
            InDev &in = ind[in_pos + f];
            in.ptr = func_ptr(s, T.inputs[f]);
            in.stage_off = T.stage_off[f];
            in.bytes16 = static_cast<int32_t>(al(P.funcs[T.inputs[f]].size * 4, kStageAlign));
        }
        in_pos += T.inputs.size();
    }
    // work-item prefixes: batched (per level) first, then plain (per task)
    s->launches.clear();
    s->launch_grid.clear();
    s->launch_smem.clear();
    s->launch_ktype.clear();
    int32_t *counters = reinterpret_cast<int32_t *>(B + s->counters_off);
    int32_t *status = reinterpret_cast<int32_t *>(B + s->status_off);
    const int32_t *pre_dev = reinterpret_cast<const int32_t *>(B + D.prefix);
    const TaskDev *td_dev = reinterpret_cast<const TaskDev *>(B + D.taskdev);
    size_t pp = 0;
    std::map<int, int> occ;
    auto blocks_per_sm = [&](int smem) {
        auto it = occ.find(smem);
        if (it != occ.end()) return it->second;
        int nb = util_max_blocks_per_sm(s->ktype, NT, smem);
        occ[smem] = nb;
        return nb;
    };
    // shared memory of a launch over tasks [first, first + count): staged
    // tables | the item's A rows | pipeline slots and four per-u partial sums
    // per thread (cp.async path)
    const int smem_cap = max_dynamic_smem() - 256;  // static shared memory of the kernel
    auto launch_smem = [&](int first, int count, LaunchDev &L) {
        int smem = 0, pipe_b = 0;
        for (int i = 0; i < count; ++i) {
            const TaskDev &x = td[first + i];
            smem = std::max(smem, x.stage_bytes);
            if (x.pipe) pipe_b = std::max(pipe_b, pipe_bytes_per_thread(x.d));
        }
        L.arows_off = static_cast<int32_t>(al(smem, 16));
        L.pipe_off = L.arows_off + (pipe_b ? kMaxPipeRows * 16 : 0);
        if (pipe_b) smem = L.pipe_off + NT * pipe_b;
        return smem;
    };
    // work items of tasks [first, first + count) for cap resident CTAs: whole
    // waves of items of about equal size, near rows_per_item rows per thread;
    // their first items go to first_item[i], numbered from *tot on
    auto size_items = [&](int first, int count, int64_t cap, int64_t *tot, int32_t *first_item) {
        double work = 0.0;  // thread-rows, idle lanes of partial lo chunks included
        for (int i = 0; i < count; ++i) {
            const TaskDev &x = td[first + i];
            work += static_cast<double>(x.nlc) * NT * x.G * x.R0 * (x.v4 ? 4 : 1);
        }
        const double pref = std::max(s->cfg.rows_per_item, 1);
        const double waves = std::max(1.0, std::round(work / (static_cast<double>(cap) * NT * pref)));
        const double rows_per_thread = work / (waves * cap * NT);
        for (int i = 0; i < count; ++i) {
            TaskDev &x = td[first + i];
            const int64_t hc = std::llround(rows_per_thread / (std::max(x.R0, 1) * (x.v4 ? 4 : 1)));
            x.hc = static_cast<int32_t>(std::min<int64_t>(std::max<int64_t>(hc, 1), x.G));
            if (x.pipe) x.hc = std::min(x.hc, kMaxPipeRows);  // its A rows fit the shared-memory area
            const int64_t items = static_cast<int64_t>(x.nlc) * ((x.G + x.hc - 1) / x.hc);
            if (items > INT32_MAX / 2) return set_error(GPUBE_ENOMEM, "a task has too many work items");
            x.n_items = static_cast<int32_t>(items);
            first_item[i] = static_cast<int32_t>(*tot);
            *tot += items;
        }
        if (*tot > INT32_MAX / 2) return set_error(GPUBE_ENOMEM, "launch has too many work items");
        return GPUBE_OK;
    };
    auto add_launch = [&](int first, int count, int counter_idx) {
        LaunchDev L{};
        L.tasks = td_dev + first;
        L.prefix = pre_dev + pp;
        L.n_tasks = count;
        const int smem = place_prefix_smem(L, launch_smem(first, count, L));
        if (smem > smem_cap)
            return set_error(GPUBE_ENOMEM, "a launch needs %d bytes of shared memory, the device allows %d (lower "
                             "stage_max_entries or block_threads)", smem, smem_cap);
        const int64_t cap = static_cast<int64_t>(blocks_per_sm(smem)) * s->num_sms;
        int64_t tot = 0;
        int rc = size_items(first, count, cap, &tot, pre + pp);
        if (rc) return rc;
        pre[pp + count] = static_cast<int32_t>(tot);
        pp += count + 1;
        L.total_items = static_cast<int32_t>(tot);
        L.counter = counters + counter_idx;
        L.status = status;
        L.top_k = w.top_k;
        s->launches.push_back(L);
        s->launch_grid.push_back(static_cast<int32_t>(std::max<int64_t>(1, std::min<int64_t>(tot, cap))));
        s->launch_smem.push_back(smem);
        // int32 and sum-product launches whose tasks all take the two-term
        // rows of one domain D (2..4) run the instantiation compiled with
        // that body alone
        const bool pk = s->ktype == kKTypeInt;
        int rows_d = (pk || s->ktype == kKTypeSum) ? rows_spec_of(td[first], pk) : 0;
        for (int i = 1; i < count && rows_d; ++i)
            if (rows_spec_of(td[first + i], pk) != rows_d) rows_d = 0;
        s->launch_ktype.push_back(rows_d ? (pk ? kKTypeIntRows : kKTypeSumRows) + rows_d - 2 : s->ktype);
        return GPUBE_OK;
    };
    s->n_zero = 1;
    if (s->launch_mode == kLaunchFused) {
        // one persistent launch over all levels: tasks in level order, each
        // level's items sized for the launch's resident CTAs, a task's CTAs
        // wait on the device for the tasks that produce its inputs
        LaunchDev L{};
        L.tasks = td_dev;
        L.prefix = pre_dev + pp;
        L.n_tasks = static_cast<int32_t>(nt);
        const int smem = place_prefix_smem(L, launch_smem(0, static_cast<int>(nt), L));
        if (smem > smem_cap)
            return set_error(GPUBE_ENOMEM, "the launch needs %d bytes of shared memory, the device allows %d "
                             "(lower stage_max_entries or block_threads)", smem, smem_cap);
        const int64_t cap = static_cast<int64_t>(blocks_per_sm(smem)) * s->num_sms;
        int64_t tot = 0;
        for (int l = 0; l < P.n_levels; ++l) {
            const int first = P.level_off[l], count = P.level_off[l + 1] - P.level_off[l];
            int rc = size_items(first, count, cap, &tot, pre + pp + first);
            if (rc) return rc;
        }
        pre[pp + nt] = static_cast<int32_t>(tot);
        pp += nt + 1;
        int32_t *doff = reinterpret_cast<int32_t *>(at(D.dep_off));
        int32_t *dl = reinterpret_cast<int32_t *>(at(D.deps));
        size_t nd = 0;
        for (size_t i = 0; i < nt; ++i) {
            doff[i] = static_cast<int32_t>(nd);
            const size_t nd0 = nd;
            for (int fid : P.tasks[P.level_order[i]].inputs) {
                const int pt = P.funcs[fid].task;
                if (pt < 0) continue;
                const int ps = slot[pt];
                if (static_cast<size_t>(ps) >= i)
                    return set_error(GPUBE_EINVAL, "internal: task %d depends on a later task", static_cast<int>(i));
                if (std::find(dl + nd0, dl + nd, ps) == dl + nd) dl[nd++] = ps;
            }
        }
        doff[nt] = static_cast<int32_t>(nd);
        L.total_items = static_cast<int32_t>(tot);
        L.counter = counters;
        L.done = counters + 1;
        L.dep_off = reinterpret_cast<const int32_t *>(B + D.dep_off);
        L.deps = reinterpret_cast<const int32_t *>(B + D.deps);
        L.status = status;
        L.top_k = w.top_k;
        s->launches.push_back(L);
        s->launch_grid.push_back(static_cast<int32_t>(std::max<int64_t>(1, std::min<int64_t>(tot, cap))));
        s->launch_smem.push_back(smem);
        s->launch_ktype.push_back(s->ktype);
        s->n_zero = static_cast<int32_t>(nt + 1);
    } else if (s->launch_mode == kLaunchPerLevel) {
        for (int l = 0; l < P.n_levels; ++l) {
            int rc = add_launch(P.level_off[l], P.level_off[l + 1] - P.level_off[l], l);
            if (rc) return rc;
        }
        s->n_zero = std::max(P.n_levels, 1);
    } else {
        for (size_t t = 0; t < nt; ++t) {
            int rc = add_launch(slot[t], 1, static_cast<int>(t));
            if (rc) return rc;
        }
        s->n_zero = static_cast<int32_t>(std::max<size_t>(nt, 1));
    }
    // expansion plan
    ExpandDev *ex = reinterpret_cast<ExpandDev *>(at(D.expand));
    int64_t *exp_pre = reinterpret_cast<int64_t *>(at(D.exp_prefix));
    int32_t *pool = reinterpret_cast<int32_t *>(at(D.pool));
    size_t po = 0;
    int64_t tot = 0;
    std::vector<int32_t> st;
    for (size_t t = 0; t < nt; ++t) {
        const Task &T = P.tasks[t];
        ExpandDev &x = ex[t];
        const int m = static_cast<int>(T.sep.size());
        x.A = reinterpret_cast<int32_t *>(B + T.A_off);
        x.B = reinterpret_cast<int32_t *>(B + T.B_off);
        x.m = m;
        x.L = T.L;
        x.nh = static_cast<int32_t>(T.hperm.size());
        x.F = static_cast<int32_t>(T.inputs.size());
        x.sa = T.sa;
        x.sb = T.sb;
        x.G = static_cast<int32_t>(T.G);
        x.P_lo = static_cast<int32_t>(T.P_lo);
        x.rad_off = static_cast<int32_t>(po);
        for (int j = 0; j < m; ++j) pool[po++] = w.dom[T.sep[j]];
        x.perm_off = static_cast<int32_t>(po);
        for (int j : T.hperm) pool[po++] = j;
        x.stride_off = static_cast<int32_t>(po);
        task_strides(w, P, T, st);
        for (int32_t v : st) pool[po++] = v;
        exp_pre[t] = tot;
        tot += T.G + 1 + T.P_lo;
    }
    exp_pre[nt] = tot;
    // value plan
    const ValuePlanH &V = P.value;
    auto put = [&](size_t off, const void *src, size_t bytes) {
        if (bytes) memcpy(at(off), src, bytes);
    };
    put(D.lev_off, V.lev_off.data(), 4 * V.lev_off.size());
    put(D.vorder, V.vorder.data(), 4 * V.vorder.size());
    put(D.vinfo, V.vinfo.data(), sizeof(ValueVar) * V.vinfo.size());
    ValueTerm *terms = reinterpret_cast<ValueTerm *>(at(D.terms));
    for (size_t i = 0; i < V.terms.size(); ++i)
        terms[i] = ValueTerm{B + V.terms[i].tab_off, V.terms[i].nv, V.terms[i].var_off};
    put(D.vvars, V.vvars.data(), 4 * V.vvars.size());
    put(D.vstrides, V.vstrides.data(), 4 * V.vstrides.size());
    ValueTerm *evals = reinterpret_cast<ValueTerm *>(at(D.evals));
    for (size_t i = 0; i < V.evals.size(); ++i)
        evals[i] = ValueTerm{B + V.evals[i].tab_off, V.evals[i].nv, V.evals[i].var_off};
    const void **roots = reinterpret_cast<const void **>(at(D.roots));
    for (size_t i = 0; i < V.roots.size(); ++i) roots[i] = B + V.roots[i];
    ValueDev &vd = s->vdev;
    vd.lev_off = reinterpret_cast<const int32_t *>(B + D.lev_off);
    vd.vorder = reinterpret_cast<const int32_t *>(B + D.vorder);
    vd.vinfo = reinterpret_cast<const ValueVar *>(B + D.vinfo);
    vd.terms = reinterpret_cast<const ValueTerm *>(B + D.terms);
    vd.vvars = reinterpret_cast<const int32_t *>(B + D.vvars);
    vd.vstrides = reinterpret_cast<const int32_t *>(B + D.vstrides);
    vd.evals = reinterpret_cast<const ValueTerm *>(B + D.evals);
    vd.roots = reinterpret_cast<const void *const *>(B + D.roots);
    vd.n = w.n;
    vd.n_levels = V.n_levels;
    vd.n_evals = static_cast<int32_t>(V.evals.size());
    vd.n_roots = static_cast<int32_t>(V.roots.size());
    vd.const_sum = P.const_sum;
    vd.top_k = w.top_k;
    vd.is_float = w.cost_type == WCSP_FP32_LOG;
    vd.result = reinterpret_cast<double *>(B + s->result_off);
    vd.sigma = reinterpret_cast<int32_t *>(B + s->sigma_off);
    vd.n_terms = static_cast<int32_t>(V.terms.size());
    vd.n_vv = static_cast<int32_t>(V.vvars.size());
    vd.smem_sig = static_cast<int32_t>(al(std::max(w.n, 1), 16));
    const size_t plan_bytes = sizeof(ValueVar) * static_cast<size_t>((w.n + 1) & ~1) + sizeof(ValueTerm) * V.terms.size() +
                              8 * V.vvars.size();
    vd.plan_in_smem = (vd.smem_sig + plan_bytes <= 160 * 1024) ? 1 : 0;
    s->value_smem = vd.smem_sig + (vd.plan_in_smem ? static_cast<int32_t>(plan_bytes) : 0);
    // a chain (one variable per level, argmin lookups, two preceding domains
    // of at most 32 value pairs) runs on one warp with its loads issued early
    bool chain = vd.plan_in_smem && V.n_levels == w.n && w.n > 0 && s->value_smem + 4 * w.n <= 160 * 1024;
    for (int v = 0; chain && v < w.n; ++v) chain = V.vinfo[v].mode <= 1 && w.dom[v] <= 5;
    vd.chain = chain ? 1 : 0;
    vd.smem_step = static_cast<int32_t>(al(s->value_smem, 16));
    if (chain) s->value_smem = vd.smem_step + 4 * w.n;
    return GPUBE_OK;
}

static void drop_graph(util_state *s)
{
    if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
}

static int upload_descriptors(util_state *s)
{
    int rc = gpube_build_descriptors(s);
    if (rc) return rc;
    drop_graph(s);
    CUDA_TRY(cudaMemcpyAsync(s->base + s->desc_off, s->host_blob.data(), s->host_blob.size(),
                             cudaMemcpyHostToDevice, s->stream));
    return GPUBE_OK;
}

// Originals in canonical scope order (descending elimination position).
static void pack_originals(const util_state *s, std::vector<unsigned char> &buf)
{
    const wcsp &w = *s->w;
    const Plan &P = s->plan;
    buf.assign(s->upload_bytes, 0);
    for (int j = 0; j < w.nf; ++j) {
        const Func &f = P.funcs[j];
        if (f.scope.empty()) continue;
        const auto &g = w.scope[j];
        const size_t a = g.size();
        std::vector<int32_t> cst = row_strides(w, f.scope), gst(a);
        for (size_t k = 0; k < a; ++k)
            for (size_t q = 0; q < a; ++q)
                if (f.scope[q] == g[k]) gst[k] = cst[q];
        std::vector<int32_t> dig(a, 0);
        int64_t ci = 0;
        for (int64_t i = 0; i < f.size; ++i) {
            if (w.cost_type == WCSP_FP32_LOG)
                reinterpret_cast<float *>(buf.data() + f.off)[ci] = w.ftab[j][i];
            else
                reinterpret_cast<int32_t *>(buf.data() + f.off)[ci] = w.itab[j][i];
            for (int k = static_cast<int>(a) - 1; k >= 0; --k) {  // odometer over the given layout
                ci += gst[k];
                if (++dig[k] < w.dom[g[k]]) break;
                ci -= static_cast<int64_t>(gst[k]) * dig[k];
                dig[k] = 0;
            }
        }
    }
}

extern "C" int util_bind(util_state *s, void *arena, size_t arena_bytes, void *stream)
{
    if (!s) return set_error(GPUBE_EINVAL, "null state");
    if (s->bound) return set_error(GPUBE_EINVAL, "state is already bound");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0)
        return set_error(GPUBE_ENODEV, "no CUDA device");
    CUDA_TRY(cudaSetDevice(s->device));
    CUDA_TRY(cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device));
    CUDA_TRY(kernels_init_device());
    if (!arena) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, s->arena_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(GPUBE_ENOMEM, "cudaMalloc of %zu bytes failed: %s", s->arena_bytes,
                             cudaGetErrorString(e));
        }
        s->base = static_cast<unsigned char *>(p);
        s->owns_arena = true;
        s->arena_cap = s->arena_bytes;
    } else {
        if (arena_bytes < s->arena_bytes)
            return set_error(GPUBE_ENOMEM, "arena of %zu bytes, the plan needs %zu", arena_bytes, s->arena_bytes);
        if (reinterpret_cast<uintptr_t>(arena) % 256)
            return set_error(GPUBE_EINVAL, "arena must be 256-byte aligned");
        s->base = static_cast<unsigned char *>(arena);
        s->arena_cap = arena_bytes;
    }
    s->stream = static_cast<cudaStream_t>(stream);
    // (timing events and the capture stream are created when first needed)
    if (s->orig_blob.empty()) pack_originals(s, s->orig_blob);
    if (!s->orig_blob.empty())
        CUDA_TRY(cudaMemcpyAsync(s->base, s->orig_blob.data(), s->orig_blob.size(), cudaMemcpyHostToDevice, s->stream));
    std::vector<unsigned char>().swap(s->orig_blob);  // staged by the copy; not needed again
    int rc = upload_descriptors(s);
    if (rc) return rc;
    CUDA_TRY(cudaMemsetAsync(s->base + s->status_off, 0, 8, s->stream));
    const DescLayout &D = layout_of(s);
    CUDA_TRY(launch_expand(reinterpret_cast<const ExpandDev *>(s->base + D.expand),
                           reinterpret_cast<const int64_t *>(s->base + D.exp_prefix),
                           static_cast<int>(s->plan.tasks.size()),
                           reinterpret_cast<const int64_t *>(s->host_blob.data() + (D.exp_prefix - s->desc_off))
                               [s->plan.tasks.size()],
                           reinterpret_cast<const int32_t *>(s->base + D.pool), s->num_sms, s->stream));
    s->bound = true;
    return GPUBE_OK;
}

// The host copy of the original tables in their device layout, made ahead of
// util_bind (e.g. by a planner thread; the layout does not depend on where
// the arena is).
void gpube_prepack(util_state *s) { pack_originals(s, s->orig_blob); }

static int ensure_events(util_state *s)
{
    for (auto &e : s->ev)
        if (!e) CUDA_TRY(cudaEventCreate(&e));
    return GPUBE_OK;
}

int gpube_enqueue_util(util_state *s, cudaStream_t st)
{
    CUDA_TRY(cudaMemsetAsync(s->base + s->counters_off, 0, 4 * static_cast<size_t>(s->n_zero), st));
    // consecutive levels: each launch may be scheduled while the previous one
    // drains (it waits for it before reading any table)
    for (size_t i = 0; i < s->launches.size(); ++i)
        CUDA_TRY(launch_util(s->launches[i], s->launch_ktype[i], s->launch_grid[i], s->cfg.threads,
                             s->launch_smem[i], st, i > 0));
    return GPUBE_OK;
}

extern "C" int util_run(util_state *s)
{
    if (!s || !s->bound) return set_error(GPUBE_EINVAL, "state is not bound");
    if (int rc = ensure_events(s)) return rc;
    if (s->use_graph) {
        if (!s->graph) {
            if (!s->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
            int rc = gpube_enqueue_util(s, s->cap_stream);
            cudaError_t e = cudaStreamEndCapture(s->cap_stream, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&s->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
        }
        CUDA_TRY(cudaEventRecord(s->ev[0], s->stream));
        CUDA_TRY(cudaGraphLaunch(s->graph, s->stream));
        CUDA_TRY(cudaEventRecord(s->ev[1], s->stream));
    } else {
        CUDA_TRY(cudaEventRecord(s->ev[0], s->stream));
        int rc = gpube_enqueue_util(s, s->stream);
        if (rc) return rc;
        CUDA_TRY(cudaEventRecord(s->ev[1], s->stream));
    }
    s->ran = true;
    return GPUBE_OK;
}

extern "C" int util_value_launch(util_state *s)
{
    if (!s || !s->bound) return set_error(GPUBE_EINVAL, "state is not bound");
    if (!s->ran) return set_error(GPUBE_EINVAL, "VALUE phase before the UTIL phase");
    if (int rc = ensure_events(s)) return rc;
    CUDA_TRY(cudaEventRecord(s->ev[2], s->stream));
    CUDA_TRY(launch_value(s->vdev, s->ktype, s->value_smem, s->stream));
    CUDA_TRY(cudaEventRecord(s->ev[3], s->stream));
    s->value_ran = true;
    return GPUBE_OK;
}

extern "C" int util_sync(util_state *s)
{
    if (!s || !s->bound) return set_error(GPUBE_EINVAL, "state is not bound");
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    int32_t status = 0;
    CUDA_TRY(cudaMemcpy(&status, s->base + s->status_off, 4, cudaMemcpyDeviceToHost));
    if (status == kStatusTimeout) return set_error(GPUBE_ETIMEDOUT, "a bounded device-side wait gave up");
    if (status == kStatusBadSpec) return set_error(GPUBE_EINVAL, "internal: a task reached a specialised kernel");
    return GPUBE_OK;
}

extern "C" int util_condition(util_state *s, int32_t n, const int32_t *vars, const int32_t *vals)
{
    if (!s || n < 0 || (n > 0 && (!vars || !vals))) return set_error(GPUBE_EINVAL, "bad argument");
    if (s->ev_vars.empty()) {
        if (n == 0) return GPUBE_OK;
        return set_error(GPUBE_EINVAL, "the plan has no evidence variables");
    }
    wcsp &c = *s->own_w;  // present whenever ev_vars is non-empty
    std::vector<int> slot(n);
    for (int i = 0; i < n; ++i) {
        auto it = std::find(s->ev_vars.begin(), s->ev_vars.end(), vars[i]);
        if (it == s->ev_vars.end()) return set_error(GPUBE_EINVAL, "variable %d is not an evidence variable", vars[i]);
        slot[i] = static_cast<int>(it - s->ev_vars.begin());
        if (vals[i] < -1 || vals[i] >= c.dom[vars[i]])
            return set_error(GPUBE_EINVAL, "value %d outside the domain of variable %d", vals[i], vars[i]);
    }
    for (int i = 0; i < n; ++i) {
        const int e = slot[i], j = s->ev_fid0 + e, a = vals[i];
        s->ev_val[e] = a;
        if (c.cost_type == WCSP_FP32_LOG)
            for (int l = 0; l < c.dom[vars[i]]; ++l) c.ftab[j][l] = (a < 0 || l == a) ? 0.0f : INFINITY;
        else
            for (int l = 0; l < c.dom[vars[i]]; ++l)
                c.itab[j][l] = (a < 0 || l == a) ? 0 : static_cast<int32_t>(c.top_k);
    }
    if (!s->bound) {
        std::vector<unsigned char>().swap(s->orig_blob);  // util_bind packs the current tables
        return GPUBE_OK;
    }
    // the evidence tables are the last originals of the arena: one copy of
    // their span (the host buffer is staged before cudaMemcpyAsync returns)
    const Plan &P = s->plan;
    const int j0 = s->ev_fid0, j1 = c.nf - 1;
    const size_t a0 = P.funcs[j0].off, a1 = P.funcs[j1].off + static_cast<size_t>(P.funcs[j1].size) * 4;
    std::vector<unsigned char> buf(a1 - a0, 0);
    for (int j = j0; j <= j1; ++j) {
        const size_t d = static_cast<size_t>(P.funcs[j].size) * 4;
        memcpy(buf.data() + (P.funcs[j].off - a0),
               c.cost_type == WCSP_FP32_LOG ? static_cast<const void *>(c.ftab[j].data())
                                            : static_cast<const void *>(c.itab[j].data()),
               d);
    }
    CUDA_TRY(cudaSetDevice(s->device));
    CUDA_TRY(cudaMemcpyAsync(s->base + a0, buf.data(), buf.size(), cudaMemcpyHostToDevice, s->stream));
    return GPUBE_OK;
}

extern "C" int util_last_times(util_state *s, double *util_ms, double *value_ms)
{
    if (!s || !s->bound) return set_error(GPUBE_EINVAL, "state is not bound");
    float a = 0.f, b = 0.f;
    if (s->ran && s->ev[1]) CUDA_TRY(cudaEventElapsedTime(&a, s->ev[0], s->ev[1]));
    if (s->value_ran && s->ev[3]) CUDA_TRY(cudaEventElapsedTime(&b, s->ev[2], s->ev[3]));
    if (util_ms) *util_ms = a;
    if (value_ms) *value_ms = b;
    return GPUBE_OK;
}

static void fill_stats(const util_state *s, solve_result *res)
{
    const Plan &P = s->plan;
    res->induced_width = P.width;
    res->n_tasks = static_cast<int32_t>(P.tasks.size());
    res->n_levels = P.n_levels;
    res->n_launches = static_cast<int32_t>(s->launches.size());
    res->util_entries = P.util_entries;
    res->alg_bytes = alg_bytes_of(P);
    res->plan_ms = s->plan_ms;
}

extern "C" int value_propagate(util_state *s, int32_t *assignment, solve_result *res)
{
    int rc = util_value_launch(s);
    if (rc) return rc;
    const int n = s->w->n;
    std::vector<unsigned char> buf(8 + 16 + 4 * static_cast<size_t>(std::max(n, 1)));
    CUDA_TRY(cudaMemcpyAsync(buf.data(), s->base + s->status_off, buf.size(), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    int32_t status;
    memcpy(&status, buf.data(), 4);
    if (status == kStatusTimeout) return set_error(GPUBE_ETIMEDOUT, "a bounded device-side wait gave up");
    if (status == kStatusBadSpec) return set_error(GPUBE_EINVAL, "internal: a task reached a specialised kernel");
    const bool sum = kind_sum(s->plan.kind);  // no assignment, no Eq. 1 cost
    if (assignment && !sum) memcpy(assignment, buf.data() + 24, 4 * static_cast<size_t>(n));
    if (res) {
        double r[2];
        memcpy(r, buf.data() + 8, 16);
        res->bound = r[0];
        res->cost = sum ? NAN : r[1];
        if (!sum && res->assignment && res->assignment != assignment)
            memcpy(res->assignment, buf.data() + 24, 4 * static_cast<size_t>(n));
        fill_stats(s, res);
        float a = 0.f, b = 0.f;
        if (s->ev[1]) cudaEventElapsedTime(&a, s->ev[0], s->ev[1]);
        if (s->ev[3]) cudaEventElapsedTime(&b, s->ev[2], s->ev[3]);
        res->util_ms = a;
        res->value_ms = b;
    }
    return GPUBE_OK;
}

extern "C" int util_fetch_table(util_state *s, int32_t t, void *cost_host, uint8_t *arg_host)
{
    if (!s || !s->bound) return set_error(GPUBE_EINVAL, "state is not bound");
    if (t < 0 || t >= static_cast<int32_t>(s->plan.tasks.size())) return set_error(GPUBE_EINVAL, "no task %d", t);
    const Task &T = s->plan.tasks[t];
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (cost_host) CUDA_TRY(cudaMemcpy(cost_host, s->base + T.out_off, T.rows * 4, cudaMemcpyDeviceToHost));
    if (arg_host) {
        if (T.keep_arg) CUDA_TRY(cudaMemcpy(arg_host, s->base + T.arg_off, T.rows, cudaMemcpyDeviceToHost));
        else memset(arg_host, 0, static_cast<size_t>(T.rows));  // the task keeps no argmin table
    }
    return GPUBE_OK;
}

extern "C" void util_state_free(util_state *s)
{
    if (!s) return;
    if (s->base && s->sync_on_free) cudaStreamSynchronize(s->stream);
    drop_graph(s);
    for (auto &e : s->ev)
        if (e) cudaEventDestroy(e);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->owns_arena && s->base) cudaFree(s->base);
    delete s;
}

// ---------------------------------------------------------------- autotune
// The launch configuration of a state: the kernel launch shape (CTA size,
// rows per work item), the work decomposition (lo extent target, staging
// limit), the group-input pipeline and the launch mode.
namespace {
struct TuneCfg {
    int32_t threads, rows, lo, stage, pipe, mode, v4;
    bool operator==(const TuneCfg &o) const
    {
        return threads == o.threads && rows == o.rows && lo == o.lo && stage == o.stage && pipe == o.pipe &&
               mode == o.mode && v4 == o.v4;
    }
};

TuneCfg current_cfg(const util_state *s)
{
    return TuneCfg{s->cfg.threads,         s->cfg.rows_per_item, s->plan.lo_target, s->plan.stage_max_entries,
                   s->plan.allow_pipe ? 1 : 0, s->launch_mode,   s->plan.allow_v4 ? 1 : 0};
}

// Expand the offset tables of a bound state on its stream (after the
// descriptors are uploaded).
int expand_tables(util_state *s)
{
    const DescLayout &D = layout_of(s);
    CUDA_TRY(launch_expand(reinterpret_cast<const ExpandDev *>(s->base + D.expand),
                           reinterpret_cast<const int64_t *>(s->base + D.exp_prefix),
                           static_cast<int>(s->plan.tasks.size()),
                           reinterpret_cast<const int64_t *>(s->host_blob.data() + (D.exp_prefix - s->desc_off))
                               [s->plan.tasks.size()],
                           reinterpret_cast<const int32_t *>(s->base + D.pool), s->num_sms, s->stream));
    return GPUBE_OK;
}
}  // namespace

// Apply a configuration to a bound state.  A new lo target or staging limit
// re-shapes the tasks (decomposition, input classes, staged tables) and lays
// the arena out again: the original tables, bucket functions and argmin
// tables keep their offsets (they come first and do not depend on the
// shape); the offset tables, descriptors and value plan after them are
// rebuilt and expanded again.  ENOMEM (state unchanged) when the new layout
// does not fit the bound arena.
static int apply_cfg(util_state *s, const TuneCfg &c)
{
    Plan &P = s->plan;
    const TuneCfg old = current_cfg(s);
    const bool reshape = c.lo != P.lo_target || c.stage != P.stage_max_entries;
    const bool was_stale = s->tables_stale;
    if (reshape) {
        P.lo_target = c.lo;
        P.stage_max_entries = c.stage;
        shape_tasks(*s->w, P);
        gpube_layout(s);
        s->tables_stale = true;
        if (s->arena_bytes > s->arena_cap) {
            P.lo_target = old.lo;
            P.stage_max_entries = old.stage;
            shape_tasks(*s->w, P);
            gpube_layout(s);
            s->tables_stale = was_stale;  // back to the shape the arena's tables were in before
            return set_error(GPUBE_ENOMEM, "the re-shaped plan does not fit the bound arena");
        }
    }
    s->cfg.threads = c.threads;
    s->cfg.rows_per_item = c.rows;
    P.allow_pipe = c.pipe != 0;
    P.allow_v4 = c.v4 != 0;
    s->launch_mode = c.mode;
    int rc = upload_descriptors(s);
    if (rc) return rc;
    // the status word may have moved with a layout (this one's, or that of a
    // configuration tried before and refused): it starts at zero again
    CUDA_TRY(cudaMemsetAsync(s->base + s->status_off, 0, 8, s->stream));
    // after a refused configuration the offset tables may belong to another
    // shape: expand whenever the shape changed since they were last written
    if (reshape || s->tables_stale) {
        rc = expand_tables(s);
        if (!rc) s->tables_stale = false;
        return rc;
    }
    return GPUBE_OK;
}

static std::string tune_key(const util_state *s)
{
    const Plan &P = s->plan;
    std::ostringstream k;
    k << "k" << P.kind << "_t" << P.tasks.size() << "_l" << P.n_levels << "_e" << P.util_entries << "_c"
      << s->ktype << "_w" << P.width << "_m" << (s->launch_mode == kLaunchPerTask ? 0 : 1);
    return k.str();
}

extern "C" int util_launch_config(const util_state *s, gpube_launch_config *out)
{
    if (!s || !out) return set_error(GPUBE_EINVAL, "null argument");
    const TuneCfg c = current_cfg(s);
    out->block_threads = c.threads;
    out->rows_per_item = c.rows;
    out->lo_target = c.lo;
    out->stage_max_entries = c.stage;
    out->pipeline = c.pipe;
    out->launch_mode = c.mode;
    out->vector_rows = c.v4;
    return GPUBE_OK;
}

extern "C" int util_autotune(util_state *s, int32_t *threads, int32_t *rows_per_item)
{
    if (!s || !s->bound) return set_error(GPUBE_EINVAL, "state is not bound");
    const std::string key = tune_key(s);
    const char *cache = s->opts.autotune_cache;
    auto report = [&]() {
        if (threads) *threads = s->cfg.threads;
        if (rows_per_item) *rows_per_item = s->cfg.rows_per_item;
        return GPUBE_OK;
    };
    if (cache) {
        std::ifstream in(cache);
        std::string line;
        while (std::getline(in, line)) {
            std::istringstream ls(line);
            std::string k;
            TuneCfg c{};
            double ms;
            if (ls >> k >> c.threads >> c.rows >> c.lo >> c.stage >> c.pipe >> c.mode >> c.v4 >> ms && k == key) {
                int rc = apply_cfg(s, c);
                if (rc == GPUBE_ENOMEM) break;  // measured with a larger arena: tune here
                if (rc) return rc;
                return report();
            }
        }
    }
    // time one configuration: the mean of two runs after one warm-up run
    // time one configuration: the median of n runs after one warm-up run, n
    // enough for about 4 ms of timed runs (2 to 15; short runs are noisier),
    // times the given factor
    auto measure = [&](const TuneCfg &c, double *ms, int factor) {
        int rc = apply_cfg(s, c);
        if (rc) return rc;
        std::vector<double> t;
        int n = 2;
        for (int rep = 0; rep <= n; ++rep) {
            rc = util_run(s);
            if (!rc) rc = util_sync(s);
            if (rc) return rc;
            double x;
            util_last_times(s, &x, nullptr);
            if (rep == 0) {
                n = factor * std::max(2, std::min(15, static_cast<int>(4.0 / std::max(x, 1e-3))));
                continue;
            }
            t.push_back(x);
        }
        std::nth_element(t.begin(), t.begin() + t.size() / 2, t.end());
        *ms = t[t.size() / 2];
        return GPUBE_OK;
    };
    TuneCfg best = current_cfg(s);
    double best_ms = 1e30;
    std::vector<TuneCfg> seen;
    std::vector<std::pair<double, int>> timed;  // (ms, index into seen) of every configuration run
    // coordinate descent: each stage varies one part of the configuration
    // around the best one so far (a candidate already timed is skipped)
    auto try_all = [&](const std::vector<TuneCfg> &cands) {
        for (const TuneCfg &c : cands) {
            if (std::find(seen.begin(), seen.end(), c) != seen.end()) continue;
            seen.push_back(c);
            double ms;
            int rc = measure(c, &ms, 1);
            if (rc == GPUBE_ENOMEM) continue;  // does not fit the bound arena
            if (rc) return rc;
            timed.push_back({ms, static_cast<int>(seen.size()) - 1});
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        return GPUBE_OK;
    };
    const int cand_t[] = {128, 256, 512};
    const int cand_r[] = {16, 32, 64, 128, 256};
    auto shapes = [&]() {
        std::vector<TuneCfg> v;
        for (int th : cand_t)
            for (int rp : cand_r) {
                TuneCfg c = best;
                c.threads = th;
                c.rows = rp;
                v.push_back(c);
            }
        return v;
    };
    // lo extent target of the work decomposition
    auto los = [&]() {
        std::vector<TuneCfg> v;
        for (int lo : {128, 256, 512, 1024, 2048}) {
            TuneCfg c = best;
            c.lo = lo;
            v.push_back(c);
        }
        return v;
    };
    int rc = try_all(shapes());
    if (!rc) rc = try_all(los());
    // two passes over the other dimensions, each around the best so far (one
    // pass can stop in a corner: a staging limit that only pays with the
    // pipeline on, kept after the pipeline is switched off)
    for (int pass = 0; pass < 2 && !rc; ++pass) {
        if (s->plan.n_levels > 1 && s->launch_mode != kLaunchPerTask) {
            // one launch per level, or one over all levels, each with every lo
            // target (the best target differs between the two forms)
            std::vector<TuneCfg> v;
            for (int mode : {kLaunchPerLevel, kLaunchFused})
                for (int lo : {128, 256, 512, 1024, 2048}) {
                    TuneCfg c = best;
                    c.mode = mode;
                    c.lo = lo;
                    v.push_back(c);
                }
            rc = try_all(v);
        }
        if (!rc) {  // staging limit (0: no table staged) and the group-input pipeline
            std::vector<TuneCfg> v;
            for (int st : {0, 1024, 4096, 32768})
                for (int pipe : {0, 1}) {
                    TuneCfg c = best;
                    c.stage = st;
                    c.pipe = pipe;
                    v.push_back(c);
                }
            rc = try_all(v);
        }
        if (!rc) {  // four rows per thread where a task allows it
            TuneCfg c = best;
            c.v4 = 1 - c.v4;
            rc = try_all({c});
        }
        if (!rc) rc = try_all(shapes());  // the launch shape again, for the chosen decomposition
        if (!rc) rc = try_all(los());       // and the lo target for that shape
    }
    if (rc) return rc;
    // the three fastest configurations timed again with three times the runs
    std::sort(timed.begin(), timed.end());
    best_ms = 1e30;
    for (size_t i = 0; i < timed.size() && i < 3; ++i) {
        double ms;
        rc = measure(seen[timed[i].second], &ms, 3);
        if (rc) return rc;
        if (ms < best_ms) {
            best_ms = ms;
            best = seen[timed[i].second];
        }
    }
    rc = apply_cfg(s, best);
    if (rc) return rc;
    if (cache) {
        std::ofstream out(cache, std::ios::app);
        out << key << " " << best.threads << " " << best.rows << " " << best.lo << " " << best.stage << " "
            << best.pipe << " " << best.mode << " " << best.v4 << " " << best_ms << "\n";
    }
    return report();
}

// ---------------------------------------------------------- one-call solvers
static int solve_common(wcsp *w, int kind, int32_t i_bound, const int32_t *parent, const solve_opts *opts,
                        solve_result *res)
{
    if (!w) return set_error(GPUBE_EINVAL, "null problem");
    solve_opts o;
    if (opts) o = *opts;
    else solve_opts_init(&o);
    util_state *s = nullptr;
    int rc = util_plan(w, kind, i_bound, parent, &o, &s);
    if (rc) return rc;
    rc = util_bind(s, o.arena, o.arena_bytes, o.stream);
    if (!rc) rc = util_run(s);
    if (!rc) rc = value_propagate(s, res ? res->assignment : nullptr, res);
    util_state_free(s);
    return rc;
}

extern "C" int be_solve(wcsp *w, const solve_opts *opts, solve_result *res)
{
    return solve_common(w, GPUBE_KIND_BE, 0, nullptr, opts, res);
}

extern "C" int mbe_solve(wcsp *w, int32_t i_bound, const solve_opts *opts, solve_result *res)
{
    return solve_common(w, GPUBE_KIND_MBE, i_bound, nullptr, opts, res);
}

extern "C" int logz_solve(wcsp *w, int32_t i_bound, const solve_opts *opts, solve_result *res)
{
    return solve_common(w, i_bound > 0 ? GPUBE_KIND_SUM_MBE : GPUBE_KIND_SUM, i_bound, nullptr, opts, res);
}

extern "C" int dpop_util(wcsp *w, const int32_t *parent, const solve_opts *opts, util_state **out)
{
    if (!w || !out) return set_error(GPUBE_EINVAL, "null argument");
    solve_opts o;
    if (opts) o = *opts;
    else solve_opts_init(&o);
    util_state *s = nullptr;
    int rc = util_plan(w, GPUBE_KIND_DPOP, 0, parent, &o, &s);
    if (rc) return rc;
    rc = util_bind(s, o.arena, o.arena_bytes, o.stream);
    if (!rc) rc = util_run(s);
    if (rc) {
        util_state_free(s);
        return rc;
    }
    *out = s;
    return GPUBE_OK;
}

// ------------------------------------------------------ single bucket
namespace {
struct Scratch {
    void *p = nullptr;
    size_t bytes = 0;
};
std::mutex g_scratch_mu;
std::map<int, Scratch> g_scratch;
}  // namespace

extern "C" int util_bucket(int32_t cost_type, int32_t top_k, int32_t m, const int32_t *sep_dom, int32_t d,
                           int32_t n_in, const void *const *in_tables, const int32_t *in_pos_off,
                           const int32_t *in_pos, void *out, uint8_t *arg, void *stream)
{
    if (cost_type != WCSP_INT32_SAT && cost_type != WCSP_FP32_LOG)
        return set_error(GPUBE_EINVAL, "unknown cost type");
    if (cost_type == WCSP_INT32_SAT && top_k < 1) return set_error(GPUBE_EINVAL, "top_k must be >= 1");
    if (m < 0 || d < 1 || d > 255 || n_in < 1 || (m > 0 && !sep_dom) || !in_tables || !in_pos_off || !out || !arg)
        return set_error(GPUBE_EINVAL, "bad argument");
    // a problem whose variables are the joint scope: separator position j is
    // variable j, the eliminated variable is m; it is eliminated first, the
    // separator from the last position to the first
    wcsp w;
    w.n = m + 1;
    w.cost_type = cost_type;
    w.top_k = static_cast<uint32_t>(cost_type == WCSP_INT32_SAT ? top_k : 1);
    w.dom.resize(m + 1);
    for (int j = 0; j < m; ++j) {
        if (sep_dom[j] < 1 || sep_dom[j] > 255) return set_error(GPUBE_EINVAL, "bad domain at %d", j);
        w.dom[j] = sep_dom[j];
    }
    w.dom[m] = d;
    util_state s;
    s.w = &w;
    s.ktype = cost_type == WCSP_FP32_LOG ? kKTypeFloat : kKTypeInt;
    Plan &P = s.plan;
    P.kind = GPUBE_KIND_BE;
    P.order.resize(m + 1);
    P.pos.resize(m + 1);
    P.order[0] = m;
    for (int j = 0; j < m; ++j) P.order[1 + j] = m - 1 - j;
    for (int t = 0; t <= m; ++t) P.pos[P.order[t]] = t;
    Task T;
    T.var = m;
    T.d = d;
    T.rows = 1;
    for (int j = 0; j < m; ++j) {
        T.sep.push_back(j);
        T.rows *= sep_dom[j];
        if (T.rows > INT32_MAX) return set_error(GPUBE_ENOMEM, "output of more than 2^31 entries");
    }
    for (int i = 0; i < n_in; ++i) {
        Func f;
        const int a = in_pos_off[i], b = in_pos_off[i + 1];
        if (b < a) return set_error(GPUBE_EINVAL, "bad in_pos_off");
        int prev = -1;
        for (int k = a; k < b; ++k) {
            if (in_pos[k] <= prev || in_pos[k] >= m) return set_error(GPUBE_EINVAL, "in_pos must ascend in [0, m)");
            prev = in_pos[k];
            f.scope.push_back(in_pos[k]);
            f.size *= sep_dom[in_pos[k]];
        }
        f.scope.push_back(m);
        f.size *= d;
        if (!in_tables[i] || reinterpret_cast<uintptr_t>(in_tables[i]) % 16)
            return set_error(GPUBE_EINVAL, "input %d is NULL or not 16-byte aligned", i);
        f.ext = in_tables[i];
        P.funcs.push_back(f);
        T.inputs.push_back(i);
    }
    T.ext_out = out;
    T.ext_arg = arg;
    P.tasks.push_back(T);
    Func o;
    o.scope = P.tasks[0].sep;
    o.size = P.tasks[0].rows;
    o.task = 0;
    P.funcs.push_back(o);
    w.nf = n_in;  // the inputs stand as the originals; they stay in the caller's memory
    P.n_levels = 1;
    P.level_order = {0};
    P.level_off = {0, 1};
    shape_tasks(w, P);
    gpube_layout(&s);
    s.launch_mode = kLaunchPerTask;
    s.use_graph = false;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    s.device = dev;
    CUDA_TRY(cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(kernels_init_device());
    s.stream = static_cast<cudaStream_t>(stream);
    // scratch: everything of the layout except the (external) tables
    std::lock_guard<std::mutex> g(g_scratch_mu);
    Scratch &sc = g_scratch[dev];
    if (sc.bytes < s.arena_bytes) {
        if (sc.p) {
            cudaStreamSynchronize(s.stream);
            cudaFree(sc.p);
        }
        sc.p = nullptr;
        sc.bytes = 0;
        cudaError_t e = cudaMalloc(&sc.p, s.arena_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(GPUBE_ENOMEM, "scratch of %zu bytes: %s", s.arena_bytes, cudaGetErrorString(e));
        }
        sc.bytes = s.arena_bytes;
    }
    s.base = static_cast<unsigned char *>(sc.p);
    int rc = gpube_build_descriptors(&s);
    if (!rc) {
        const DescLayout &D = layout_of(&s);
        cudaError_t e = cudaMemcpyAsync(s.base + s.desc_off, s.host_blob.data(), s.host_blob.size(),
                                        cudaMemcpyHostToDevice, s.stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(s.base + s.status_off, 0, 8, s.stream);
        if (e == cudaSuccess)
            e = launch_expand(reinterpret_cast<const ExpandDev *>(s.base + D.expand),
                              reinterpret_cast<const int64_t *>(s.base + D.exp_prefix), 1,
                              P.tasks[0].G + 1 + P.tasks[0].P_lo, reinterpret_cast<const int32_t *>(s.base + D.pool),
                              s.num_sms, s.stream);
        if (e != cudaSuccess) rc = cuda_error(e, "util_bucket upload");
        else rc = gpube_enqueue_util(&s, s.stream);
    }
    return rc;
}
