// Host planning: elimination order (Definition 1, min-fill / natural /
// given / DFS pseudo-tree post-order, Sections 2 and 6.2), buckets and
// mini-bucket partitions (Algorithms 1-2), elimination-tree levels, the work
// decomposition of each bucket for the UTIL kernel, the VALUE plan and the
// arena layout.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdint>
#include <numeric>

#include "gpube_internal.h"

namespace gpube {

static thread_local char g_err[512];

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

const char *last_error() { return g_err; }

int cuda_error(cudaError_t e, const char *what)
{
    return set_error(GPUBE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ----------------------------------------------------------- orderings
namespace {

struct Bits {
    int n = 0, words = 0;
    std::vector<uint64_t> w;  // n rows of `words` 64-bit words
    void init(int n_)
    {
        n = n_;
        words = (n + 63) / 64;
        w.assign(static_cast<size_t>(n) * words, 0);
    }
    uint64_t *row(int v) { return w.data() + static_cast<size_t>(v) * words; }
    bool test(int v, int u) const { return (w[static_cast<size_t>(v) * words + u / 64] >> (u % 64)) & 1; }
    void set(int v, int u) { row(v)[u / 64] |= 1ULL << (u % 64); }
};

}  // namespace

// Greedy min-fill: eliminate the variable whose remaining neighbours have the
// fewest unconnected pairs; ties: fewer remaining neighbours, then lower id.
// fill[] and deg[] are kept up to date edge by edge: removing v drops, for
// each neighbour a, the missing pairs (v, x) of a's neighbourhood; adding a
// fill edge (a, b) removes one missing pair from every common neighbour and
// adds to a (b) the pairs (b, x) ((a, x)) that are still missing.
std::vector<int32_t> order_minfill(const wcsp &w, int32_t *width, int32_t give_up_above)
{
    const int n = w.n;
    Bits adj;
    adj.init(n);
    for (int v = 0; v < n; ++v)
        for (int u : w.adj[v]) adj.set(v, u);
    const int W = adj.words;
    std::vector<uint64_t> alive(W, 0);
    for (int v = 0; v < n; ++v) alive[v / 64] |= 1ULL << (v % 64);
    // |N(a) \ N[b]| among alive vertices (b itself excluded)
    auto missing_from = [&](int a, int b) {
        const uint64_t *ra = adj.row(a), *rb = adj.row(b);
        int64_t c = 0;
        for (int k = 0; k < W; ++k) c += __builtin_popcountll(ra[k] & alive[k] & ~rb[k]);
        const bool b_counted = adj.test(a, b) && ((alive[b / 64] >> (b % 64)) & 1);
        return c - (b_counted ? 1 : 0);
    };
    std::vector<int64_t> fill(n, 0);
    std::vector<int32_t> deg(n, 0);
    for (int v = 0; v < n; ++v) {
        int64_t m = 0;
        for (int a : w.adj[v]) m += missing_from(v, a);  // ordered pairs (a, x), x in N(v) \ N[a]
        fill[v] = m / 2;
        deg[v] = static_cast<int32_t>(w.adj[v].size());
    }
    std::vector<int32_t> order;
    order.reserve(n);
    std::vector<char> gone(n, 0);
    std::vector<int> nb;
    int32_t wmax = 0;
    for (int t = 0; t < n; ++t) {
        int best = -1;
        for (int v = 0; v < n; ++v) {
            if (gone[v]) continue;
            if (best < 0 || fill[v] < fill[best] || (fill[v] == fill[best] && deg[v] < deg[best])) best = v;
        }
        nb.clear();
        {
            const uint64_t *r = adj.row(best);
            for (int k = 0; k < W; ++k) {
                uint64_t x = r[k] & alive[k];
                while (x) {
                    nb.push_back(k * 64 + __builtin_ctzll(x));
                    x &= x - 1;
                }
            }
        }
        wmax = std::max<int32_t>(wmax, static_cast<int32_t>(nb.size()));
        if (wmax > give_up_above) {  // the caller has an order at least this good
            if (width) *width = wmax;
            return {};
        }
        gone[best] = 1;
        order.push_back(best);
        // 1. best leaves the graph
        alive[best / 64] &= ~(1ULL << (best % 64));
        for (int a : nb) {
            fill[a] -= missing_from(a, best);
            deg[a] -= 1;
        }
        // 2. its neighbours become a clique, one fill edge at a time
        for (size_t i = 0; i < nb.size(); ++i)
            for (size_t j2 = i + 1; j2 < nb.size(); ++j2) {
                const int a = nb[i], b = nb[j2];
                if (adj.test(a, b)) continue;
                const uint64_t *ra = adj.row(a), *rb = adj.row(b);
                for (int k = 0; k < W; ++k) {
                    uint64_t x = ra[k] & rb[k] & alive[k];
                    while (x) {
                        fill[k * 64 + __builtin_ctzll(x)] -= 1;
                        x &= x - 1;
                    }
                }
                fill[a] += missing_from(a, b);
                fill[b] += missing_from(b, a);
                deg[a] += 1;
                deg[b] += 1;
                adj.set(a, b);
                adj.set(b, a);
            }
    }
    if (width) *width = wmax;
    return order;
}

// Induced width along an order (Definition 1): the largest number of
// remaining neighbours of a variable when it is eliminated, its remaining
// neighbours connected pairwise after each elimination (adjacency bit rows).
int32_t induced_width(const wcsp &w, const std::vector<int32_t> &order)
{
    const int n = w.n;
    Bits adj;
    adj.init(n);
    for (int v = 0; v < n; ++v)
        for (int u : w.adj[v]) adj.set(v, u);
    const int W = adj.words;
    std::vector<uint64_t> alive(W, 0), nbm(W);
    for (int v = 0; v < n; ++v) alive[v / 64] |= 1ULL << (v % 64);
    int32_t wmax = 0;
    std::vector<int> nb;
    for (int v : order) {
        alive[v / 64] &= ~(1ULL << (v % 64));
        const uint64_t *r = adj.row(v);
        nb.clear();
        for (int k = 0; k < W; ++k) {
            nbm[k] = r[k] & alive[k];
            for (uint64_t x = nbm[k]; x; x &= x - 1) nb.push_back(k * 64 + __builtin_ctzll(x));
        }
        wmax = std::max<int32_t>(wmax, static_cast<int32_t>(nb.size()));
        for (int a : nb) {  // a gains every other remaining neighbour of v
            uint64_t *ra = adj.row(a);
            for (int k = 0; k < W; ++k) ra[k] |= nbm[k];
            ra[a / 64] &= ~(1ULL << (a % 64));
        }
    }
    return wmax;
}

// Vertices by (degree descending, id ascending): the pseudo-tree priority of
// Section 6.2.
static std::vector<int32_t> degree_rank(const wcsp &w)
{
    std::vector<int32_t> r(w.n);
    std::iota(r.begin(), r.end(), 0);
    std::stable_sort(r.begin(), r.end(), [&](int a, int b) { return w.adj[a].size() > w.adj[b].size(); });
    return r;
}

// DFS pseudo-tree (Definition 2): every non-tree edge of a DFS tree joins an
// ancestor and a descendant.  Roots and children by degree_rank.
std::vector<int32_t> dfs_pseudotree(const wcsp &w)
{
    const int n = w.n;
    std::vector<int32_t> rank = degree_rank(w), where(n);
    for (int i = 0; i < n; ++i) where[rank[i]] = i;
    std::vector<std::vector<int32_t>> nbr(n);
    for (int v = 0; v < n; ++v) {
        nbr[v] = w.adj[v];
        std::sort(nbr[v].begin(), nbr[v].end(), [&](int a, int b) { return where[a] < where[b]; });
    }
    std::vector<int32_t> parent(n, -1);
    std::vector<char> seen(n, 0);
    std::vector<std::pair<int, size_t>> st;
    for (int r : rank) {
        if (seen[r]) continue;
        seen[r] = 1;
        st.push_back({r, 0});
        while (!st.empty()) {
            auto &top = st.back();
            if (top.second < nbr[top.first].size()) {
                int u = nbr[top.first][top.second++];
                if (!seen[u]) {
                    seen[u] = 1;
                    parent[u] = top.first;
                    st.push_back({u, 0});
                }
            } else {
                st.pop_back();
            }
        }
    }
    return parent;
}

// Post-order of a pseudo-tree (children and roots by degree_rank), after
// checking that parent[] is a forest on which every constraint lies on one
// root-to-leaf path.
int pseudotree_order(const wcsp &w, const int32_t *parent, std::vector<int32_t> &order)
{
    const int n = w.n;
    for (int v = 0; v < n; ++v)
        if (parent[v] < -1 || parent[v] >= n || parent[v] == v)
            return set_error(GPUBE_EINVAL, "parent[%d] = %d is not a variable", v, parent[v]);
    std::vector<int32_t> rank = degree_rank(w), where(n);
    for (int i = 0; i < n; ++i) where[rank[i]] = i;
    std::vector<std::vector<int32_t>> kids(n);
    std::vector<int32_t> roots;
    for (int r : rank) {
        if (parent[r] < 0) roots.push_back(r);
        else kids[parent[r]].push_back(r);
    }
    order.clear();
    std::vector<int32_t> tin(n, -1), tout(n, -1);
    int clock = 0;
    std::vector<std::pair<int, size_t>> st;
    for (int r : roots) {
        st.push_back({r, 0});
        tin[r] = clock++;
        while (!st.empty()) {
            auto &top = st.back();
            if (top.second < kids[top.first].size()) {
                int c = kids[top.first][top.second++];
                tin[c] = clock++;
                st.push_back({c, 0});
            } else {
                tout[top.first] = clock++;
                order.push_back(top.first);
                st.pop_back();
            }
        }
    }
    if (static_cast<int>(order.size()) != n)
        return set_error(GPUBE_EINVAL, "parent[] has a cycle (%zu of %d nodes reachable)", order.size(), n);
    auto is_anc = [&](int a, int b) { return tin[a] <= tin[b] && tout[b] <= tout[a]; };
    for (int j = 0; j < w.nf; ++j) {
        const auto &s = w.scope[j];
        for (size_t x = 0; x < s.size(); ++x)
            for (size_t y = x + 1; y < s.size(); ++y)
                if (!is_anc(s[x], s[y]) && !is_anc(s[y], s[x]))
                    return set_error(GPUBE_EINVAL,
                                     "constraint %d joins %d and %d on different branches of the pseudo-tree",
                                     j, s[x], s[y]);
    }
    return GPUBE_OK;
}

// ------------------------------------------------------------- planning
static bool mb_fits(const wcsp &w, int mode, int z, const std::vector<int32_t> &u)
{
    const int k = static_cast<int>(u.size());
    if (mode == GPUBE_IB_SEP_VARS) return k - 1 <= z;
    if (mode == GPUBE_IB_JOINT_VARS) return k <= z;
    // product of the domains <= 2^z, exactly
    if (z < 0) return false;
    unsigned __int128 p = 1, lim = (z >= 120) ? ~static_cast<unsigned __int128>(0) : (static_cast<unsigned __int128>(1) << z);
    for (int v : u) {
        p *= static_cast<unsigned>(w.dom[v]);
        if (p > lim) return false;
    }
    return true;
}

int build_plan(const wcsp &w, int kind, int i_bound, const int32_t *parent, const solve_opts &o, Plan &P)
{
    const int n = w.n;
    P = Plan();
    P.kind = kind;
    P.i_bound = i_bound;
    P.ibound_mode = o.ibound_mode;
    if (kind_mbe(kind) && (o.ibound_mode < 0 || o.ibound_mode > 2))
        return set_error(GPUBE_EINVAL, "unknown ibound_mode %d", o.ibound_mode);
    if (o.lo_target > 0) P.lo_target = o.lo_target;
    if (o.stage_max_entries > 0) P.stage_max_entries = o.stage_max_entries;
    if (o.stage_max_entries < 0) P.stage_max_entries = 0;
    P.allow_pipe = o.pipeline >= 0;
    P.allow_v4 = o.vector_rows > 0;
    P.keep_arg = !kind_mbe(kind) || o.argmin_tables > 0;

    // 1. elimination order
    int okind = o.order_kind;
    if (kind == GPUBE_KIND_DPOP) okind = GPUBE_ORDER_PSEUDOTREE;
    const int32_t *tree = (kind == GPUBE_KIND_DPOP) ? parent : o.parent;
    switch (okind) {
    case GPUBE_ORDER_MINFILL: P.order = order_minfill(w, nullptr); break;
    case GPUBE_ORDER_NATURAL:
        P.order.resize(n);
        std::iota(P.order.begin(), P.order.end(), 0);
        break;
    case GPUBE_ORDER_BEST: {
        // the natural order unless min-fill is at least as good (min-fill is
        // abandoned as soon as its width exceeds the natural order's)
        std::vector<int32_t> nat(n);
        std::iota(nat.begin(), nat.end(), 0);
        const int32_t wn = induced_width(w, nat);
        int32_t wm = 0;
        P.order = order_minfill(w, &wm, wn);
        if (P.order.empty()) P.order = nat;
        break;
    }
    case GPUBE_ORDER_GIVEN: {
        if (!o.order) return set_error(GPUBE_EINVAL, "GPUBE_ORDER_GIVEN without an order");
        P.order.assign(o.order, o.order + n);
        std::vector<char> seen(n, 0);
        for (int v : P.order) {
            if (v < 0 || v >= n || seen[v]) return set_error(GPUBE_EINVAL, "order is not a permutation");
            seen[v] = 1;
        }
        break;
    }
    case GPUBE_ORDER_PSEUDOTREE: {
        std::vector<int32_t> pt;
        if (!tree) {
            pt = dfs_pseudotree(w);
            tree = pt.data();
        }
        int rc = pseudotree_order(w, tree, P.order);
        if (rc) return rc;
        break;
    }
    default: return set_error(GPUBE_EINVAL, "unknown order kind %d", okind);
    }
    P.pos.assign(n, 0);
    for (int t = 0; t < n; ++t) P.pos[P.order[t]] = t;

    // 2. original functions in canonical scope order (descending position)
    auto canonical = [&](std::vector<int32_t> s) {
        std::sort(s.begin(), s.end(), [&](int a, int b) { return P.pos[a] > P.pos[b]; });
        return s;
    };
    std::vector<std::vector<int32_t>> bucket(n);
    P.funcs.reserve(static_cast<size_t>(w.nf) + n);
    P.tasks.reserve(n);
    P.funcs.resize(w.nf);
    for (int j = 0; j < w.nf; ++j) {
        Func &f = P.funcs[j];
        f.scope = canonical(w.scope[j]);
        f.size = 1;
        for (int v : f.scope) f.size *= w.dom[v];
        if (f.scope.empty()) {
            P.const_sum += (w.cost_type == WCSP_FP32_LOG) ? static_cast<double>(w.ftab[j][0])
                                                          : static_cast<double>(w.itab[j][0]);
        } else {
            bucket[f.scope.back()].push_back(j);
        }
    }

    // 3. Algorithm 1 / 2: buckets, partitions, bucket functions
    const bool mbe = kind_mbe(kind);
    std::vector<char> in_union(n, 0);  // BE: variables of the bucket's single mini-bucket
    // scratch reused across buckets: mini-bucket variable sets and function
    // lists (the first nmb entries are live), a separator, a scope union
    std::vector<std::vector<int32_t>> mb_funcs, mb_vars;
    std::vector<int32_t> sep, fv, uni;
    for (int t = 0; t < n; ++t) {
        const int v = P.order[t];
        std::vector<int32_t> &B = bucket[v];
        if (B.empty()) {
            // a variable in no function: nothing to minimise; in the sum each
            // of its values counts, a factor |D_v| of Z
            if (kind_sum(kind)) P.const_sum += -std::log(static_cast<double>(w.dom[v]));
            continue;
        }
        // arity descending, then creation order (a total order: the sort is stable)
        std::sort(B.begin(), B.end(), [&](int a, int b) {
            if (P.funcs[a].scope.size() != P.funcs[b].scope.size())
                return P.funcs[a].scope.size() > P.funcs[b].scope.size();
            return a < b;
        });
        size_t nmb = 0;  // mini-buckets of this bucket; their variables kept sorted by id
        auto open_mb = [&]() {
            if (mb_vars.size() <= nmb) {
                mb_vars.emplace_back();
                mb_funcs.emplace_back();
            }
            mb_vars[nmb].clear();
            mb_funcs[nmb].clear();
            return nmb++;
        };
        if (!mbe) {
            // one bucket: the union of the scopes by marks, no partition
            const size_t b0 = open_mb();
            mb_funcs[b0] = B;
            for (int fid : B)
                for (int u : P.funcs[fid].scope)
                    if (!in_union[u]) {
                        in_union[u] = 1;
                        mb_vars[b0].push_back(u);
                    }
            for (int u : mb_vars[b0]) in_union[u] = 0;
            std::sort(mb_vars[b0].begin(), mb_vars[b0].end());
        }
        for (size_t k = 0; mbe && k < B.size(); ++k) {  // Algorithm 2: first fit under the bound
            const int fid = B[k];
            fv.assign(P.funcs[fid].scope.begin(), P.funcs[fid].scope.end());
            std::sort(fv.begin(), fv.end());
            size_t placed = SIZE_MAX;
            for (size_t b = 0; b < nmb && placed == SIZE_MAX; ++b) {
                uni.clear();
                std::set_union(mb_vars[b].begin(), mb_vars[b].end(), fv.begin(), fv.end(), std::back_inserter(uni));
                if (mb_fits(w, o.ibound_mode, i_bound, uni)) {
                    mb_vars[b].swap(uni);
                    placed = b;
                }
            }
            if (placed == SIZE_MAX) {
                placed = open_mb();
                mb_vars[placed] = fv;
            }
            mb_funcs[placed].push_back(fid);
        }
        for (size_t b = 0; b < nmb; ++b) {
            Task T;
            T.var = v;
            T.d = w.dom[v];
            sep.clear();
            for (int u : mb_vars[b])
                if (u != v) sep.push_back(u);
            T.sep = canonical(sep);
            T.inputs = mb_funcs[b];
            T.rows = 1;
            for (int u : T.sep) {
                T.rows *= w.dom[u];
                if (T.rows > INT32_MAX)
                    return set_error(GPUBE_ENOMEM, "bucket of variable %d needs a table of more than 2^31 entries", v);
            }
            int lev = 0;
            for (int fid : T.inputs)
                if (P.funcs[fid].task >= 0) lev = std::max(lev, P.tasks[P.funcs[fid].task].level + 1);
            T.level = lev;
            const int tid = static_cast<int>(P.tasks.size());
            P.width = std::max<int32_t>(P.width, static_cast<int32_t>(T.sep.size()));
            P.max_inputs = std::max<int32_t>(P.max_inputs, static_cast<int32_t>(T.inputs.size()));
            P.util_entries += T.rows * T.d;
            P.out_entries += T.rows;
            for (int fid : T.inputs) P.in_entries += P.funcs[fid].size;
            Func out;
            out.scope = T.sep;
            out.size = T.rows;
            out.task = tid;
            P.tasks.push_back(std::move(T));
            P.funcs.push_back(std::move(out));
            if (!P.tasks.back().sep.empty()) bucket[P.tasks.back().sep.back()].push_back(w.nf + tid);
        }
    }

    // 4. elimination-tree levels
    P.n_levels = 0;
    for (const Task &T : P.tasks) P.n_levels = std::max(P.n_levels, T.level + 1);
    P.level_order.resize(P.tasks.size());
    std::iota(P.level_order.begin(), P.level_order.end(), 0);
    std::stable_sort(P.level_order.begin(), P.level_order.end(),
                     [&](int a, int b) { return P.tasks[a].level < P.tasks[b].level; });
    P.level_off.assign(P.n_levels + 1, 0);
    for (const Task &T : P.tasks) P.level_off[T.level + 1]++;
    for (int l = 0; l < P.n_levels; ++l) P.level_off[l + 1] += P.level_off[l];
    return GPUBE_OK;
}

// ------------------------------------------------- work decomposition
// Stride of each separator digit in each input's canonical layout (0 when
// the input does not mention it), plus the output's own strides (slot F).
void task_strides(const wcsp &w, const Plan &P, const Task &T, std::vector<int32_t> &st)
{
    const int m = static_cast<int>(T.sep.size());
    const int F = static_cast<int>(T.inputs.size());
    st.assign(static_cast<size_t>(F + 1) * m, 0);
    for (int f = 0; f < F; ++f) {
        const Func &fn = P.funcs[T.inputs[f]];
        int64_t s = 1;
        for (int k = static_cast<int>(fn.scope.size()) - 1; k >= 0; --k) {
            const int u = fn.scope[k];
            for (int j = 0; j < m; ++j)
                if (T.sep[j] == u) st[static_cast<size_t>(f) * m + j] = static_cast<int32_t>(s);
            s *= w.dom[u];
        }
    }
    int64_t s = 1;
    for (int j = m - 1; j >= 0; --j) {
        st[static_cast<size_t>(F) * m + j] = static_cast<int32_t>(s);
        s *= w.dom[T.sep[j]];
    }
}

// Split every task's rows into (hi, lo), choose the hi iteration order
// (its fastest digit u, then the groups), order the inputs by how often
// they are read, and choose the staged inputs.
void shape_tasks(const wcsp &w, Plan &P)
{
    // staged bytes per task: the byte limit, or room for one table at the
    // entry limit when that is larger (up to 160 KB, which leaves shared
    // memory for the pipeline slots of a 128-thread CTA)
    const int64_t stage_cap = std::min<int64_t>(std::max<int64_t>(P.stage_max_bytes, 4LL * P.stage_max_entries),
                                                160 * 1024);
    // scratch lists reused across tasks (cleared per task)
    std::vector<int32_t> absent, present, lo_only, group, u_only, row;
    std::vector<int> idx;
    for (Task &T : P.tasks) {
        const int m = static_cast<int>(T.sep.size());
        const int F = static_cast<int>(T.inputs.size());
        T.L = 0;
        T.P_lo = 1;
        for (int j = m - 1; j >= 0 && T.P_lo < P.lo_target; --j) {
            T.P_lo *= w.dom[T.sep[j]];
            T.L++;
        }
        T.H = T.rows / T.P_lo;
        // hi digits absent from the largest input iterate fastest: consecutive
        // rows then share that input's entries
        int big = 0;
        for (int f = 1; f < F; ++f)
            if (P.funcs[T.inputs[f]].size > P.funcs[T.inputs[big]].size) big = f;
        const auto &bs = P.funcs[T.inputs[big]].scope;
        absent.clear();
        present.clear();
        for (int j = m - T.L - 1; j >= 0; --j) {
            bool in = std::find(bs.begin(), bs.end(), T.sep[j]) != bs.end();
            (in ? present : absent).push_back(j);
        }
        T.hperm = absent;
        T.hperm.insert(T.hperm.end(), present.begin(), present.end());
        T.R0 = T.hperm.empty() ? 1 : w.dom[T.sep[T.hperm[0]]];
        T.G = T.H / T.R0;
        // inputs: lo digits only | hi digits but not u | u as the only hi digit | u and others
        {
            lo_only.clear();
            group.clear();
            u_only.clear();
            row.clear();
            for (int fid : T.inputs) {
                const auto &fs = P.funcs[fid].scope;
                auto has = [&](int j) { return std::find(fs.begin(), fs.end(), T.sep[j]) != fs.end(); };
                int nhi = 0;
                for (int j = 0; j < m - T.L; ++j) nhi += has(j);
                if (nhi == 0) lo_only.push_back(fid);
                else if (!has(T.hperm[0])) group.push_back(fid);
                else if (nhi == 1) u_only.push_back(fid);
                else row.push_back(fid);
            }
            T.n_lo = static_cast<int32_t>(lo_only.size());
            T.n_gi = static_cast<int32_t>(lo_only.size() + group.size());
            T.n_uo = static_cast<int32_t>(T.n_gi + u_only.size());
            T.inputs = lo_only;
            T.inputs.insert(T.inputs.end(), group.begin(), group.end());
            T.inputs.insert(T.inputs.end(), u_only.begin(), u_only.end());
            T.inputs.insert(T.inputs.end(), row.begin(), row.end());
        }
        T.sa = arow_of(F);
        T.sb = brow_of(F);
        // stage the smallest inputs while they fit
        T.stage_off.assign(F, -1);
        T.stage_bytes = 0;
        idx.resize(F);
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(),
                         [&](int a, int b) { return P.funcs[T.inputs[a]].size < P.funcs[T.inputs[b]].size; });
        for (int f : idx) {
            const Func &fn = P.funcs[T.inputs[f]];
            const int64_t sz = fn.size;
            if (sz > P.stage_max_entries) break;
            if (fn.ext && (sz * 4) % kStageAlign) continue;  // a copy would read past the caller's table
            const int64_t bytes = static_cast<int64_t>(align_up(sz * 4, kStageAlign));
            if (T.stage_bytes + bytes > stage_cap) break;
            T.stage_off[f] = T.stage_bytes;
            T.stage_bytes += static_cast<int32_t>(bytes);
        }
        T.keep_arg = task_keeps_arg(w.cost_type, P, T);
    }
}

}  // namespace gpube
