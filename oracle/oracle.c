/*
 * CPU oracle for Bucket Elimination, Mini-Bucket Elimination and DPOP's
 * UTIL / VALUE phases (arXiv 1608.05288, Sections 2-4 and 6).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may link, load or
 * call this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA path.
 *
 * Everything here is written for clarity, not speed:
 *   - costs are held in double.  Integer WCSP costs (<= 2^30) and their sums
 *     are exact in double, so the integer semantics "sum, then saturate at
 *     the top cost k" (Section 2: k stands for infinity) are reproduced
 *     exactly; real (-log p) costs are fp64.
 *   - a cost function is evaluated on a full assignment by the row-major rule
 *     of the bucket-table definition (Section 6.1: rows in lexicographic
 *     order, the first scope variable varies slowest).
 *   - the elimination loop follows Algorithm 1 / Algorithm 2 step by step.
 *
 * Readings of points the paper leaves open (each one is a decision shared by
 * the oracle and the library; see the design notes):
 *   - bucket of a function = its first-eliminated variable (Algorithm 1
 *     picks the bucket by a minimum in the paper's reverse numbering; the
 *     text of Section 2.1 and the worked example fix the meaning);
 *   - a bucket function's scope is its separator ordered by descending
 *     elimination position, the eliminated variable last (Section 6.2);
 *   - ties in min / argmin: the first minimum by ascending domain value;
 *   - the mini-bucket bound z is applied in one of three modes (separator
 *     arity, joint arity, log2 of joint entries), partition = first fit of the
 *     functions sorted by arity (descending) then creation index;
 *   - MBE value assignment minimises the sum of all functions of the bucket
 *     (all mini-buckets), Section 2.2's example.
 *   - sum-product (the weighted-counting / partition-function problem the
 *     conclusions name, and the solution count of Section 2.1): the same
 *     buckets, with the min over the eliminated variable replaced by
 *     -log sum_l exp(-s_l), so that the root constants add up to -log Z,
 *     Z = sum over all assignments of exp(-Eq. 1 cost).  Costs are real
 *     (-log weights, +inf = weight 0); a WCSP's solutions are counted by
 *     giving each entry below the top cost weight 1 and the rest weight 0
 *     (a solution is consistent when no function is at the top cost).  A
 *     mini-bucket partition eliminates each mini-bucket by its own sum, which
 *     can only make Z larger (sum_l prod_j g_j <= prod_j sum_l g_j for
 *     g_j >= 0), so the mini-bucket -log Z is a lower bound, as for min-sum.
 *     There is no value phase.
 *
 * Parity pins: brute force on tiny instances (minimum and -log Z), the worked examples of
 * Sections 2 and 6 (structure and Eq. 3), invariants (BE = optimum, MBE lower
 * bound, cost of the returned assignment), a transfer-matrix DP for grids,
 * component additivity.  The example's optimum value (cost 4, bound 2) is
 * parity unpinned: its cost tables are only in a figure.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ problem */
typedef struct {
    int n;                    /* number of variables                          */
    const int *dom;           /* dom[v] = |D_v|                               */
    int nf;                   /* number of cost functions                     */
    const int *scope_off;     /* [nf+1] offsets into scope                    */
    const int *scope;         /* variable ids, each function's scope as given */
    const long long *tab_off; /* [nf+1] offsets into cost                     */
    const double *cost;       /* table entries, row-major over the scope      */
    int saturate;             /* 1: integer WCSP costs, saturate at top       */
    double top;               /* the top cost k (infeasible)                  */
} orc_problem;

static int g_threads = 1;

void orc_set_threads(int t) { g_threads = t > 0 ? t : 1; }

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}

/* A cost function: an ordered scope and a row-major table over it. */
typedef struct {
    int nv;
    int *vars;
    long long *stride; /* stride[j] = product of dom of vars[j+1..] */
    const double *tab;
    double *owned;     /* non-NULL when the table belongs to the oracle */
} func;

static void func_init(func *f, const orc_problem *P, int nv, const int *vars, const double *tab)
{
    f->nv = nv;
    f->vars = (int *)malloc(sizeof(int) * (nv > 0 ? nv : 1));
    f->stride = (long long *)malloc(sizeof(long long) * (nv > 0 ? nv : 1));
    memcpy(f->vars, vars, sizeof(int) * nv);
    long long s = 1;
    for (int j = nv - 1; j >= 0; --j) {
        f->stride[j] = s;
        s *= P->dom[vars[j]];
    }
    f->tab = tab;
    f->owned = NULL;
}

/* f(asg): the entry of f's table selected by the full assignment asg. */
static double func_eval(const func *f, const int *asg)
{
    long long idx = 0;
    for (int j = 0; j < f->nv; ++j) idx += (long long)asg[f->vars[j]] * f->stride[j];
    return f->tab[idx];
}

static double clamp_top(const orc_problem *P, double s)
{
    if (P->saturate && s > P->top) return P->top;
    return s;
}

/* Eq. 1: the cost of a complete assignment, sum over all cost functions. */
double orc_eval(const orc_problem *P, const int *sigma)
{
    double s = 0.0;
    for (int i = 0; i < P->nf; ++i) {
        func f;
        func_init(&f, P, P->scope_off[i + 1] - P->scope_off[i], P->scope + P->scope_off[i],
                  P->cost + P->tab_off[i]);
        s += func_eval(&f, sigma);
        free(f.vars);
        free(f.stride);
    }
    return clamp_top(P, s);
}

/* Exhaustive minimisation of Eq. 1 (tiny instances only).  Assignments are
 * enumerated with variable 0 slowest; the first minimum is returned. */
double orc_bruteforce(const orc_problem *P, int *sigma_out)
{
    int n = P->n;
    int *asg = (int *)calloc(n > 0 ? n : 1, sizeof(int));
    double best = INFINITY;
    for (;;) {
        double c = orc_eval(P, asg);
        if (c < best) {
            best = c;
            memcpy(sigma_out, asg, sizeof(int) * n);
        }
        int j = n - 1;
        while (j >= 0) {
            if (++asg[j] < P->dom[j]) break;
            asg[j] = 0;
            --j;
        }
        if (j < 0) break;
    }
    free(asg);
    return best;
}

/* -log Z by enumeration (tiny instances only): Z = sum over every complete
 * assignment of exp(-cost), cost = Eq. 1 (real costs, no saturation).  The
 * smallest cost c0 is taken out first, -log Z = c0 - log sum exp(c0 - cost),
 * so that no term underflows as a whole; an instance with no finite-cost
 * assignment has Z = 0 and -log Z = +inf. */
double orc_sum_bruteforce(const orc_problem *P)
{
    int n = P->n;
    int *asg = (int *)calloc(n > 0 ? n : 1, sizeof(int));
    double c0 = INFINITY, z = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        memset(asg, 0, sizeof(int) * (n > 0 ? n : 1));
        for (;;) {
            double c = orc_eval(P, asg);
            if (pass == 0) {
                if (c < c0) c0 = c;
            } else {
                z += exp(c0 - c);
            }
            int j = n - 1;
            while (j >= 0) {
                if (++asg[j] < P->dom[j]) break;
                asg[j] = 0;
                --j;
            }
            if (j < 0) break;
        }
        if (pass == 0 && !(c0 < INFINITY)) break;
    }
    free(asg);
    return c0 < INFINITY ? c0 - log(z) : INFINITY;
}

/* ------------------------------------------------------------ primal graph */
static unsigned char *primal_graph(const orc_problem *P)
{
    int n = P->n;
    unsigned char *adj = (unsigned char *)calloc((size_t)n * n + 1, 1);
    for (int i = 0; i < P->nf; ++i) {
        const int *s = P->scope + P->scope_off[i];
        int a = P->scope_off[i + 1] - P->scope_off[i];
        for (int x = 0; x < a; ++x)
            for (int y = 0; y < a; ++y)
                if (s[x] != s[y]) adj[(size_t)s[x] * n + s[y]] = 1;
    }
    return adj;
}

/* Induced width along an elimination order (order[0] eliminated first):
 * the largest number of not-yet-eliminated neighbours a variable has when it
 * is eliminated, neighbours being connected to each other as it goes
 * (Definition 1). */
int orc_induced_width(const orc_problem *P, const int *order)
{
    int n = P->n, w = 0;
    unsigned char *adj = primal_graph(P);
    unsigned char *gone = (unsigned char *)calloc(n + 1, 1);
    int *nb = (int *)malloc(sizeof(int) * (n + 1));
    for (int t = 0; t < n; ++t) {
        int v = order[t], k = 0;
        for (int u = 0; u < n; ++u)
            if (!gone[u] && adj[(size_t)v * n + u]) nb[k++] = u;
        if (k > w) w = k;
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b)
                if (a != b) adj[(size_t)nb[a] * n + nb[b]] = 1;
        gone[v] = 1;
    }
    free(adj);
    free(gone);
    free(nb);
    return w;
}

/* Greedy min-fill elimination order: repeatedly eliminate the variable whose
 * elimination adds the fewest fill edges; ties go to the fewest remaining
 * neighbours, then to the lowest id.  Returns the induced width. */
int orc_minfill(const orc_problem *P, int *order)
{
    int n = P->n, w = 0;
    unsigned char *adj = primal_graph(P);
    unsigned char *gone = (unsigned char *)calloc(n + 1, 1);
    int *nb = (int *)malloc(sizeof(int) * (n + 1));
    for (int t = 0; t < n; ++t) {
        int best = -1;
        long long bfill = 0;
        int bdeg = 0;
        for (int v = 0; v < n; ++v) {
            if (gone[v]) continue;
            int k = 0;
            for (int u = 0; u < n; ++u)
                if (!gone[u] && adj[(size_t)v * n + u]) nb[k++] = u;
            long long fill = 0;
            for (int a = 0; a < k; ++a)
                for (int b = a + 1; b < k; ++b)
                    if (!adj[(size_t)nb[a] * n + nb[b]]) ++fill;
            if (best < 0 || fill < bfill || (fill == bfill && k < bdeg)) {
                best = v;
                bfill = fill;
                bdeg = k;
            }
        }
        int k = 0;
        for (int u = 0; u < n; ++u)
            if (!gone[u] && adj[(size_t)best * n + u]) nb[k++] = u;
        if (k > w) w = k;
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b)
                if (a != b) adj[(size_t)nb[a] * n + nb[b]] = 1;
        gone[best] = 1;
        order[t] = best;
    }
    free(adj);
    free(gone);
    free(nb);
    return w;
}

/* ------------------------------------------------------------ pseudo-trees */
static int *g_deg; /* degree table for the comparator below */

/* (degree descending, id ascending): the priority of Section 6.2
 * (x_i before x_j iff |N(x_i)| > |N(x_j)|), ties to the lowest id. */
static int by_degree(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    if (g_deg[x] != g_deg[y]) return g_deg[y] - g_deg[x];
    return x - y;
}

static void dfs_visit(int u, int n, const unsigned char *adj, unsigned char *seen, int *parent,
                      const int *rank)
{
    seen[u] = 1;
    for (int i = 0; i < n; ++i) {
        int w = rank[i];
        if (adj[(size_t)u * n + w] && !seen[w]) {
            parent[w] = u;
            dfs_visit(w, n, adj, seen, parent, rank);
        }
    }
}

/* DFS pseudo-tree (Definition 2): roots and children are taken by
 * (degree descending, id ascending).  parent[v] = -1 for roots. */
void orc_dfs_pseudotree(const orc_problem *P, int *parent)
{
    int n = P->n;
    unsigned char *adj = primal_graph(P);
    int *deg = (int *)calloc(n + 1, sizeof(int));
    int *rank = (int *)malloc(sizeof(int) * (n + 1));
    unsigned char *seen = (unsigned char *)calloc(n + 1, 1);
    for (int v = 0; v < n; ++v) {
        for (int u = 0; u < n; ++u) deg[v] += adj[(size_t)v * n + u];
        rank[v] = v;
        parent[v] = -1;
    }
    g_deg = deg;
    qsort(rank, n, sizeof(int), by_degree);
    for (int i = 0; i < n; ++i)
        if (!seen[rank[i]]) dfs_visit(rank[i], n, adj, seen, parent, rank);
    free(adj);
    free(deg);
    free(rank);
    free(seen);
}

static void post_visit(int u, int n, const int *parent, const int *rank, int *order, int *t)
{
    for (int i = 0; i < n; ++i)
        if (parent[rank[i]] == u) post_visit(rank[i], n, parent, rank, order, t);
    order[(*t)++] = u;
}

/* Elimination order of a pseudo-tree: its post-order (every node after all of
 * its descendants), children and roots taken by (degree descending, id
 * ascending).  DPOP's UTIL messages are BE's bucket functions on this order
 * (Section 4.1). */
void orc_pseudotree_order(const orc_problem *P, const int *parent, int *order)
{
    int n = P->n, t = 0;
    unsigned char *adj = primal_graph(P);
    int *deg = (int *)calloc(n + 1, sizeof(int));
    int *rank = (int *)malloc(sizeof(int) * (n + 1));
    for (int v = 0; v < n; ++v) {
        for (int u = 0; u < n; ++u) deg[v] += adj[(size_t)v * n + u];
        rank[v] = v;
    }
    g_deg = deg;
    qsort(rank, n, sizeof(int), by_degree);
    for (int i = 0; i < n; ++i)
        if (parent[rank[i]] == -1) post_visit(rank[i], n, parent, rank, order, &t);
    free(adj);
    free(deg);
    free(rank);
}

/* ----------------------------------------------------------------- Eq. 3 */
/* Eq. 3 of Section 6.3: the row of an input bucket-table that matches row
 * r_out of the output bucket-table.  The output scope has m variables with
 * domains out_dom[0..m-1]; the input scope is the subsequence at positions
 * phi[0..s-1] (ascending) of it, and both end with the same variable
 * (phi[s-1] = m-1).  mul[k] = product of the input domains after k,
 * div[k] = product of the output domains after phi[k], mod[k] = the input
 * domain of k. */
long long orc_project_index(int m, const int *out_dom, int s, const int *phi, long long r_out)
{
    long long r_in = 0;
    for (int k = 0; k < s - 1; ++k) {
        long long mul = 1, div = 1;
        for (int j = k + 1; j < s; ++j) mul *= out_dom[phi[j]];
        for (int j = phi[k] + 1; j < m; ++j) div *= out_dom[j];
        long long mod = out_dom[phi[k]];
        r_in += mul * ((r_out / div) % mod);
    }
    r_in += r_out % out_dom[phi[s - 1]];
    return r_in;
}

/* One bucket, as Section 6 computes it: aggregate every input table into a
 * zero-initialised joint table (Procedure Gpu::Aggregate, rows matched by
 * Eq. 3), then eliminate the last variable by a min over its contiguous rows
 * (Procedure Gpu::Eliminate), also recording the first argmin.
 * Joint scope: the m-1 separator variables (domains sep_dom) then the
 * eliminated variable (domain d).  Input i has ns[i] separator positions
 * (ascending) listed in pos[], plus the eliminated variable last. */
void orc_util_bucket(int m1, const int *sep_dom, int d, int nin, const double *const *tabs,
                     const int *ns, const int *pos, int saturate, double top, double *out,
                     unsigned char *arg)
{
    int m = m1 + 1;
    int *jdom = (int *)malloc(sizeof(int) * m);
    for (int j = 0; j < m1; ++j) jdom[j] = sep_dom[j];
    jdom[m1] = d;
    long long rows = 1;
    for (int j = 0; j < m1; ++j) rows *= sep_dom[j];
    long long jrows = rows * d;
    double *joint = (double *)calloc((size_t)(jrows > 0 ? jrows : 1), sizeof(double));
    int *phi = (int *)malloc(sizeof(int) * m);
    const int *p = pos;
    for (int i = 0; i < nin; ++i) {
        for (int k = 0; k < ns[i]; ++k) phi[k] = p[k];
        phi[ns[i]] = m1;
        for (long long r = 0; r < jrows; ++r)
            joint[r] += tabs[i][orc_project_index(m, jdom, ns[i] + 1, phi, r)];
        p += ns[i];
    }
    for (long long r = 0; r < rows; ++r) {
        double best = 0.0;
        int bl = 0;
        for (int l = 0; l < d; ++l) {
            double c = joint[r * d + l];
            if (saturate && c > top) c = top;
            if (l == 0 || c < best) {
                best = c;
                bl = l;
            }
        }
        out[r] = best;
        arg[r] = (unsigned char)bl;
    }
    free(jdom);
    free(joint);
    free(phi);
}

/* ------------------------------------------------------ (mini-)bucket run */
typedef struct {
    int var;         /* eliminated variable                      */
    int nsep;        /* separator size                           */
    int *sep;        /* separator, descending elimination order  */
    int nin;         /* number of functions in the mini-bucket   */
    int *in_ids;     /* their creation ids                       */
    long long rows;  /* output entries                           */
    double *out;     /* the bucket function's table              */
    unsigned char *arg;
} task;

typedef struct {
    int n, ntasks;
    task *tasks;
    double bound;    /* sum of the root constants (saturated)    */
    int *sigma;      /* VALUE phase assignment                   */
    double cost;     /* Eq. 1 cost of sigma                      */
    int width;       /* largest separator                        */
} orc_run;

enum { ORC_BE = 0, ORC_MBE_SEP = 1, ORC_MBE_JOINT = 2, ORC_MBE_LOG2 = 3 };
enum { ORC_MIN_SUM = 0, ORC_SUM_PRODUCT = 1 };

static int fits(const orc_problem *P, int mode, int z, const unsigned char *in_u)
{
    int k = 0;
    double entries = 1.0;
    for (int v = 0; v < P->n; ++v)
        if (in_u[v]) {
            ++k;
            entries *= P->dom[v];
        }
    if (mode == ORC_BE) return 1;
    if (mode == ORC_MBE_SEP) return k - 1 <= z;
    if (mode == ORC_MBE_JOINT) return k <= z;
    return entries <= ldexp(1.0, z);
}

static int *g_ar, *g_id; /* arity / creation id, for the partition sort */
static int by_arity(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    if (g_ar[x] != g_ar[y]) return g_ar[y] - g_ar[x];
    return g_id[x] - g_id[y];
}

/* Algorithm 1 (mode ORC_BE) / Algorithm 2 (the other modes) along the given
 * elimination order.  semiring ORC_MIN_SUM eliminates by min and is followed
 * by the value-assignment phase; ORC_SUM_PRODUCT eliminates by
 * -log sum exp(-.) and has no value phase (sigma stays 0, cost is NaN). */
orc_run *orc_eliminate_sr(const orc_problem *P, const int *order, int mode, int z, int semiring)
{
    int n = P->n;
    /* A mini-bucket turns one or more live functions into at most one new
     * one, so at most nf functions are live at any time (bucket sizes are
     * bounded by nf); the total number of functions and tasks is not, and
     * those arrays grow on demand. */
    int live_cap = P->nf + 1;
    int cap = P->nf + n + 8;
    func *fs = (func *)calloc(cap, sizeof(func));
    int *alive = (int *)calloc(cap, sizeof(int));
    int *fid = (int *)calloc(cap, sizeof(int)); /* creation id of fs[i] */
    int nfs = 0;
    int *pos = (int *)malloc(sizeof(int) * (n + 1));
    for (int t = 0; t < n; ++t) pos[order[t]] = t;

    orc_run *R = (orc_run *)calloc(1, sizeof(orc_run));
    R->n = n;
    R->tasks = (task *)calloc(cap, sizeof(task));
    R->sigma = (int *)calloc(n + 1, sizeof(int));
    double bound = 0.0;

    for (int i = 0; i < P->nf; ++i) {
        int a = P->scope_off[i + 1] - P->scope_off[i];
        func_init(&fs[nfs], P, a, P->scope + P->scope_off[i], P->cost + P->tab_off[i]);
        fid[nfs] = i;
        if (a == 0) { /* a constant: part of every solution's cost */
            bound += fs[nfs].tab[0];
            alive[nfs] = 0;
        } else {
            alive[nfs] = 1;
        }
        ++nfs;
    }

    /* bucket membership kept for the value phase: vb[v] lists the bucket's
     * functions, vbm[v] the mini-bucket each of them went to */
    int **vb = (int **)calloc(n + 1, sizeof(int *));
    int **vbm = (int **)calloc(n + 1, sizeof(int *));
    int *nvb = (int *)calloc(n + 1, sizeof(int));
    unsigned char *in_u = (unsigned char *)calloc(n + 1, 1);
    unsigned char *tmp_u = (unsigned char *)calloc(n + 1, 1);
    int *members = (int *)malloc(sizeof(int) * live_cap);
    int *mb_of = (int *)malloc(sizeof(int) * live_cap);
    unsigned char *mb_u = (unsigned char *)calloc((size_t)live_cap * (n + 1), 1);

    for (int t = 0; t < n; ++t) {
        int v = order[t];
        /* B_v: every live function mentioning v (its first-eliminated variable) */
        int nb = 0;
        for (int i = 0; i < nfs; ++i) {
            if (!alive[i]) continue;
            for (int j = 0; j < fs[i].nv; ++j)
                if (fs[i].vars[j] == v) {
                    members[nb++] = i;
                    break;
                }
        }
        vb[v] = (int *)malloc(sizeof(int) * (nb > 0 ? nb : 1));
        vbm[v] = (int *)calloc(nb > 0 ? nb : 1, sizeof(int));
        nvb[v] = nb;
        memcpy(vb[v], members, sizeof(int) * nb);
        for (int k = 0; k < nb; ++k) alive[members[k]] = 0;
        if (nb == 0) {
            /* an empty bucket: min-sum adds nothing; for the sum every value of
             * v is free, a factor |D_v| of Z */
            if (semiring == ORC_SUM_PRODUCT) bound += -log((double)P->dom[v]);
            continue;
        }

        /* partition into mini-buckets: sort by arity desc, creation id asc,
         * then first fit under the bound z */
        if (nfs + nb + 1 > cap) { /* room for this bucket's new functions and tasks */
            int ncap = 2 * (nfs + nb + 1);
            fs = (func *)realloc(fs, sizeof(func) * ncap);
            alive = (int *)realloc(alive, sizeof(int) * ncap);
            fid = (int *)realloc(fid, sizeof(int) * ncap);
            R->tasks = (task *)realloc(R->tasks, sizeof(task) * ncap);
            memset(R->tasks + cap, 0, sizeof(task) * (ncap - cap));
            cap = ncap;
        }
        int *ar = (int *)malloc(sizeof(int) * cap);
        for (int i = 0; i < nfs; ++i) ar[i] = fs[i].nv;
        g_ar = ar;
        g_id = fid;
        qsort(members, nb, sizeof(int), by_arity);
        int nmb = 0;
        for (int k = 0; k < nb; ++k) {
            func *f = &fs[members[k]];
            int placed = -1;
            for (int b = 0; b < nmb && placed < 0; ++b) {
                unsigned char *u = mb_u + (size_t)b * (n + 1);
                memcpy(tmp_u, u, n + 1);
                for (int j = 0; j < f->nv; ++j) tmp_u[f->vars[j]] = 1;
                if (fits(P, mode, z, tmp_u)) {
                    memcpy(u, tmp_u, n + 1);
                    placed = b;
                }
            }
            if (placed < 0) {
                placed = nmb++;
                unsigned char *u = mb_u + (size_t)placed * (n + 1);
                memset(u, 0, n + 1);
                for (int j = 0; j < f->nv; ++j) u[f->vars[j]] = 1;
            }
            mb_of[k] = placed;
        }
        free(ar);
        for (int k = 0; k < nb; ++k)
            for (int q = 0; q < nb; ++q)
                if (vb[v][q] == members[k]) vbm[v][q] = mb_of[k];

        for (int b = 0; b < nmb; ++b) {
            unsigned char *u = mb_u + (size_t)b * (n + 1);
            task *T = &R->tasks[R->ntasks];
            T->var = v;
            /* separator: the union minus v, by descending elimination position */
            T->sep = (int *)malloc(sizeof(int) * (n + 1));
            T->nsep = 0;
            for (int tt = n - 1; tt > t; --tt)
                if (u[order[tt]]) T->sep[T->nsep++] = order[tt];
            T->in_ids = (int *)malloc(sizeof(int) * (nb + 1));
            T->nin = 0;
            for (int k = 0; k < nb; ++k)
                if (mb_of[k] == b) T->in_ids[T->nin++] = fid[members[k]];
            int *mbf = (int *)malloc(sizeof(int) * (nb + 1));
            int nm = 0;
            for (int k = 0; k < nb; ++k)
                if (mb_of[k] == b) mbf[nm++] = members[k];
            long long rows = 1;
            for (int j = 0; j < T->nsep; ++j) rows *= P->dom[T->sep[j]];
            T->rows = rows;
            T->out = (double *)malloc(sizeof(double) * rows);
            T->arg = (unsigned char *)malloc(rows);
            if (T->nsep > R->width) R->width = T->nsep;
            /* h(sep) = min over v of the sum of the mini-bucket's functions
             * (sum-product: -log of the sum over v of exp(-sum)) */
#pragma omp parallel num_threads(g_threads)
            {
            int *asg = (int *)calloc(n + 1, sizeof(int));
            double *sv = (double *)malloc(sizeof(double) * P->dom[v]);
#pragma omp for schedule(static)
            for (long long r = 0; r < rows; ++r) {
                long long rem = r;
                for (int j = T->nsep - 1; j >= 0; --j) {
                    asg[T->sep[j]] = (int)(rem % P->dom[T->sep[j]]);
                    rem /= P->dom[T->sep[j]];
                }
                double best = 0.0;
                int bl = 0;
                for (int l = 0; l < P->dom[v]; ++l) {
                    asg[v] = l;
                    double s = 0.0;
                    for (int k = 0; k < nm; ++k) s += func_eval(&fs[mbf[k]], asg);
                    s = clamp_top(P, s);
                    sv[l] = s;
                    if (l == 0 || s < best) {
                        best = s;
                        bl = l;
                    }
                }
                if (semiring == ORC_SUM_PRODUCT && best < INFINITY) {
                    /* -log sum_l exp(-sv[l]), with the smallest term taken out */
                    double acc = 0.0;
                    for (int l = 0; l < P->dom[v]; ++l) acc += exp(best - sv[l]);
                    best = best - log(acc);
                }
                T->out[r] = best;
                T->arg[r] = (unsigned char)bl;
            }
            free(sv);
            free(asg);
            }
            free(mbf);
            if (T->nsep == 0) {
                bound += T->out[0]; /* a root constant (Section 6.2, components add up) */
            } else {
                func_init(&fs[nfs], P, T->nsep, T->sep, T->out);
                fid[nfs] = P->nf + R->ntasks;
                alive[nfs] = 1;
                ++nfs;
            }
            R->ntasks++;
        }
    }
    R->bound = clamp_top(P, bound);

    /* value assignment: reverse elimination order, first argmin of the sum of
     * every function that was in the variable's bucket */
    int *asg = R->sigma;
    for (int t = n - 1; t >= 0 && semiring == ORC_MIN_SUM; --t) {
        int v = order[t];
        double best = 0.0;
        int bl = 0;
        for (int l = 0; l < P->dom[v]; ++l) {
            asg[v] = l;
            double s = 0.0;
            for (int k = 0; k < nvb[v]; ++k) s += func_eval(&fs[vb[v][k]], asg);
            s = clamp_top(P, s);
            if (l == 0 || s < best) {
                best = s;
                bl = l;
            }
        }
        asg[v] = bl;
    }
    R->cost = semiring == ORC_MIN_SUM ? orc_eval(P, R->sigma) : NAN;

    for (int i = 0; i < nfs; ++i) {
        free(fs[i].vars);
        free(fs[i].stride);
    }
    for (int v = 0; v < n; ++v) {
        free(vb[v]);
        free(vbm[v]);
    }
    free(vb);
    free(vbm);
    free(nvb);
    free(fs);
    free(alive);
    free(fid);
    free(pos);
    free(in_u);
    free(tmp_u);
    free(members);
    free(mb_of);
    free(mb_u);
    return R;
}

orc_run *orc_eliminate(const orc_problem *P, const int *order, int mode, int z)
{
    return orc_eliminate_sr(P, order, mode, z, ORC_MIN_SUM);
}

int orc_run_ntasks(const orc_run *R) { return R->ntasks; }
double orc_run_bound(const orc_run *R) { return R->bound; }
double orc_run_cost(const orc_run *R) { return R->cost; }
int orc_run_width(const orc_run *R) { return R->width; }
void orc_run_sigma(const orc_run *R, int *sigma) { memcpy(sigma, R->sigma, sizeof(int) * R->n); }

void orc_run_task(const orc_run *R, int t, int *var, int *nsep, int *sep, int *nin, int *in_ids,
                  long long *rows)
{
    const task *T = &R->tasks[t];
    *var = T->var;
    *nsep = T->nsep;
    if (sep) memcpy(sep, T->sep, sizeof(int) * T->nsep);
    *nin = T->nin;
    if (in_ids) memcpy(in_ids, T->in_ids, sizeof(int) * T->nin);
    *rows = T->rows;
}

void orc_run_table(const orc_run *R, int t, double *out, unsigned char *arg)
{
    const task *T = &R->tasks[t];
    if (out) memcpy(out, T->out, sizeof(double) * T->rows);
    if (arg) memcpy(arg, T->arg, T->rows);
}

void orc_run_free(orc_run *R)
{
    if (!R) return;
    for (int t = 0; t < R->ntasks; ++t) {
        free(R->tasks[t].sep);
        free(R->tasks[t].in_ids);
        free(R->tasks[t].out);
        free(R->tasks[t].arg);
    }
    free(R->tasks);
    free(R->sigma);
    free(R);
}
