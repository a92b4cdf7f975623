"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses an independent
computation (exhaustive search, a transfer-matrix DP, a closed form, values
printed in the paper) or an invariant the paper proves.
"""
import itertools
import json
import os

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ------------------------------------------------------------------ Eq. 3
def test_eq3_worked_example(orc):
    g = _gold("eq3_example.json")
    got = [orc.project_index(g["out_dom"], g["phi"], r) for r in g["r_out"]]
    assert got == g["r_in"]


def test_eq3_is_mixed_radix_projection(orc):
    # closed form: r_in is the row-major index of the projected digits
    rng = np.random.default_rng(1)
    for _ in range(50):
        m = int(rng.integers(1, 6))
        dom = rng.integers(1, 5, size=m).tolist()
        keep = sorted(set(rng.choice(m - 1, size=int(rng.integers(0, m)), replace=True).tolist())) if m > 1 else []
        phi = keep + [m - 1]
        for r in range(int(np.prod(dom))):
            digits = np.unravel_index(r, dom)
            want = np.ravel_multi_index([digits[p] for p in phi], [dom[p] for p in phi])
            assert orc.project_index(dom, phi, r) == want


# ------------------------------------------------------------- brute force
def test_bruteforce_unary_closed_form(orc):
    # with unary functions only, the optimum is the sum of the unary minima
    rng = np.random.default_rng(2)
    dom = np.array([3, 2, 4], dtype=np.int32)
    scopes = [np.array([v], dtype=np.int32) for v in range(3)] + [np.array([1], dtype=np.int32)]
    tables = [rng.integers(0, 50, size=int(dom[s[0]])) for s in scopes]
    inst = synth.Instance("unary", dom, scopes, tables, "int", 1 << 30)
    best, sig = orc.bruteforce(inst)
    want = tables[0].min() + (tables[1] + tables[3]).min() + tables[2].min()
    assert best == want
    assert orc.evaluate(inst, sig) == best


def test_eval_matches_numpy_broadcast(orc):
    # Eq. 1 on every assignment against a dense numpy evaluation
    for seed in range(5):
        inst = synth.random_small(seed, n=4, dmax=3, n_funcs=6)
        dense = np.zeros(tuple(int(d) for d in inst.dom))
        for s, t in zip(inst.scopes, inst.tables):
            shape = [1] * inst.n
            for v in s:
                shape[v] = int(inst.dom[v])
            arr = np.asarray(t, dtype=np.float64).reshape([int(inst.dom[v]) for v in s])
            order = np.argsort(s)
            arr = np.transpose(arr, order).reshape(shape) if len(s) else arr.reshape(shape)
            dense = dense + arr
        dense = np.minimum(dense, inst.top_k)
        for a in itertools.product(*[range(int(d)) for d in inst.dom]):
            assert orc.evaluate(inst, np.array(a)) == dense[a]


# ------------------------------------------------------ worked example (Sec. 2)
def _structure(run):
    return [{"var": int(t.var), "sep": [int(x) for x in t.sep], "inputs": sorted(int(x) for x in t.inputs)}
            for t in run.tasks]


def test_paper_example_structure(orc):
    g = _gold("paper_example_structure.json")
    inst = synth.paper_example()
    order = np.array(g["elimination_order"], dtype=np.int32)
    assert orc.induced_width(inst, order) == g["induced_width"]
    be = orc.eliminate(inst, order, "be")
    assert _structure(be) == g["be_tasks"]
    mbe = orc.eliminate(inst, order, "sep", 1)
    assert _structure(mbe) == g["mbe_z1_tasks"]
    # MBE gives a lower bound, its assignment an upper bound (Section 2.2)
    assert mbe.bound <= be.bound <= mbe.cost
    assert be.cost == be.bound



# ---------------------------------- mini-bucket partition and value (Sec. 2.2)
def _golden_instance(case, name):
    dom = np.array(case["dom"], dtype=np.int32)
    scopes = [np.array(s, dtype=np.int32) for s in case["scopes"]]
    if "tables" in case:
        tables = [np.array(t, dtype=np.int64) for t in case["tables"]]
    else:  # the partition depends on the scopes only
        tables = [np.zeros(int(np.prod([dom[v] for v in s])), dtype=np.int64) for s in scopes]
    return synth.Instance(name, dom, scopes, tables, "int", 1 << 30)


def test_mbe_partition_golden(orc):
    # hand-derived first-fit partitions of mixed-arity buckets (R13), with
    # unions exactly on the joint and log2 bounds
    for case in _gold("mbe_partition.json")["cases"]:
        inst = _golden_instance(case, case["name"])
        run = orc.eliminate(inst, np.array(case["order"], dtype=np.int32), case["mode"], case["z"])
        got = [{"sep": [int(x) for x in t.sep], "inputs": sorted(int(x) for x in t.inputs)}
               for t in run.tasks if int(t.var) == 0]
        assert got == case["tasks_of_var0"], case["name"]


def test_mbe_value_sums_every_minibucket(orc):
    # R11: the value of x_i minimises the sum of every function of its bucket
    g = _gold("mbe_value_example.json")
    inst = _golden_instance(g, "mbe_value")
    order = np.array(g["order"], dtype=np.int32)
    run = orc.eliminate(inst, order, g["mode"], g["z"])
    got = [{"var": int(t.var), "sep": [int(x) for x in t.sep], "inputs": [int(x) for x in t.inputs],
            "out": [int(x) for x in t.out], "arg": [int(x) for x in t.arg]} for t in run.tasks]
    assert got == g["tasks"]
    assert run.bound == g["bound"]
    assert [int(x) for x in run.sigma] == g["sigma"]
    assert run.cost == g["cost"]
    assert orc.bruteforce(inst)[0] == g["optimum"]

# ------------------------------------------------------ BE = exhaustive optimum
@pytest.mark.parametrize("cost_type", ["int", "real"])
@pytest.mark.parametrize("seed", range(12))
def test_be_equals_bruteforce(orc, seed, cost_type):
    inst = synth.random_small(seed, n=6, dmax=3, n_funcs=9, max_arity=3, cost_type=cost_type)
    best, _ = orc.bruteforce(inst)
    rng = np.random.default_rng(seed)
    orders = [orc.minfill(inst)[0], np.arange(inst.n), rng.permutation(inst.n)]
    for order in orders:
        run = orc.eliminate(inst, order, "be")
        if cost_type == "int":
            assert run.bound == best
            assert run.cost == best
        else:
            assert run.bound == pytest.approx(best, rel=1e-12, abs=1e-12)
            assert run.cost == pytest.approx(best, rel=1e-12, abs=1e-12)
        assert orc.evaluate(inst, run.sigma) == run.cost


@pytest.mark.parametrize("seed", range(8))
def test_mbe_bounds_and_exactness(orc, seed):
    inst = synth.random_small(seed + 100, n=7, dmax=3, n_funcs=10, max_arity=3)
    best, _ = orc.bruteforce(inst)
    order, w = orc.minfill(inst)
    be = orc.eliminate(inst, order, "be")
    for mode in ("sep", "joint", "log2"):
        for z in range(0, 8):
            run = orc.eliminate(inst, order, mode, z)
            assert run.bound <= best <= run.cost
            assert orc.evaluate(inst, run.sigma) == run.cost
    # once the bound admits every bucket, MBE is BE: identical tables
    exact = orc.eliminate(inst, order, "sep", w)
    assert _structure(exact) == _structure(be)
    for a, b in zip(exact.tasks, be.tasks):
        assert np.array_equal(a.out, b.out) and np.array_equal(a.arg, b.arg)
    assert exact.bound == best


def test_saturation_at_top(orc):
    # every joint entry sums past k: the optimum saturates to k and argmin is 0
    k = 100
    dom = np.array([2, 2], dtype=np.int32)
    scopes = [np.array([0, 1], dtype=np.int32), np.array([1], dtype=np.int32)]
    tables = [np.array([60, 70, 80, 90]), np.array([50, 45])]
    inst = synth.Instance("sat", dom, scopes, tables, "int", k)
    run = orc.eliminate(inst, np.array([1, 0]), "be")
    assert run.bound == k
    assert [int(x) for x in run.tasks[0].out] == [k, k]
    assert [int(x) for x in run.tasks[0].arg] == [0, 0]
    assert list(run.sigma) == [0, 0]


def test_argmin_first_minimum(orc):
    dom = np.array([3], dtype=np.int32)
    inst = synth.Instance("tie", dom, [np.array([0], dtype=np.int32)], [np.array([5, 2, 2])], "int", 1 << 30)
    run = orc.eliminate(inst, np.array([0]), "be")
    assert run.bound == 2 and int(run.tasks[0].arg[0]) == 1 and run.sigma[0] == 1


# --------------------------------------------- the two bucket formulations agree
def _to_joint(inst, f_scope, table, joint):
    """Re-lay a table row-major over its scope's subsequence of `joint`."""
    f_scope = [int(x) for x in f_scope]
    arr = np.asarray(table, dtype=np.float64).reshape([int(inst.dom[v]) for v in f_scope])
    keep = [v for v in joint if v in f_scope]
    return np.transpose(arr, [f_scope.index(v) for v in keep]).reshape(-1), keep


@pytest.mark.parametrize("seed", range(6))
def test_eq3_bucket_matches_assignment_form(orc, seed):
    inst = synth.random_small(seed + 7, n=6, dmax=3, n_funcs=9, with_constant=False)
    order, _ = orc.minfill(inst)
    run = orc.eliminate(inst, order, "sep", 2)
    funcs = {j: (inst.scopes[j], inst.tables[j]) for j in range(inst.n_funcs)}
    for t, T in enumerate(run.tasks):
        joint = [int(x) for x in T.sep] + [T.var]
        tabs, poss = [], []
        for i in T.inputs:
            s, tab = funcs[int(i)]
            flat, keep = _to_joint(inst, s, tab, joint)
            tabs.append(flat)
            poss.append([joint.index(v) for v in keep[:-1]])
            assert keep[-1] == T.var
        out, arg = orc.util_bucket([int(inst.dom[v]) for v in T.sep], int(inst.dom[T.var]),
                                   tabs, poss, True, inst.top_k)
        assert np.array_equal(out, T.out) and np.array_equal(arg, T.arg)
        funcs[inst.n_funcs + t] = (T.sep, T.out)


# ------------------------------------------------- grids: transfer-matrix DP
def _grid_dp(inst, rows, cols, d):
    """Row-by-row dynamic programme over all d**cols row states: an algorithm
    independent of variable elimination."""
    un = np.zeros((rows * cols, d))
    h = {}
    for s, t in zip(inst.scopes, inst.tables):
        s = [int(x) for x in s]
        if len(s) == 1:
            un[s[0]] += t
        else:
            h[tuple(s)] = np.asarray(t, dtype=np.float64).reshape(d, d)
    states = np.array(list(itertools.product(range(d), repeat=cols)))
    def row_cost(r):
        c = np.zeros(len(states))
        for j in range(cols):
            v = r * cols + j
            c += un[v][states[:, j]]
            if j + 1 < cols:
                c += h[(v, v + 1)][states[:, j], states[:, j + 1]]
        return c
    best = row_cost(0)
    for r in range(1, rows):
        trans = np.zeros((len(states), len(states)))
        for j in range(cols):
            v = (r - 1) * cols + j
            trans += h[(v, v + cols)][states[:, j][:, None], states[:, j][None, :]]
        best = (best[:, None] + trans).min(axis=0) + row_cost(r)
    return best.min()


def test_config0_transfer_matrix(orc):
    for seed in range(3):
        inst = synth.config_instance(0, seed)
        order, w = orc.minfill(inst)
        assert w == 4
        run = orc.eliminate(inst, order, "be")
        assert run.bound == _grid_dp(inst, 4, 5, 4)
        assert run.cost == run.bound


def test_grid_natural_order_width(orc):
    # row-major elimination of an r x c grid keeps c variables on the frontier
    for r, c in [(4, 5), (12, 12), (3, 7)]:
        inst = synth.grid_wcsp(r, c, 2, 0, unary=False)
        assert orc.induced_width(inst, np.arange(r * c)) == c


def test_minfill_small_graphs(orc):
    # a star has width 1 (leaves go first), a 5-cycle width 2
    star = synth.Instance("star", np.full(5, 2, np.int32),
                          [np.array([0, v], np.int32) for v in range(1, 5)],
                          [np.zeros(4, np.int64)] * 4, "int", 1 << 30)
    order, w = orc.minfill(star)
    assert w == 1 and int(order[-1]) in (0, 4) and sorted(order.tolist()) == list(range(5))
    cyc = synth.Instance("cyc", np.full(5, 2, np.int32),
                         [np.array(sorted((v, (v + 1) % 5)), np.int32) for v in range(5)],
                         [np.zeros(4, np.int64)] * 5, "int", 1 << 30)
    order, w = orc.minfill(cyc)
    assert w == 2 and int(order[0]) == 0


def test_minfill_tie_breaks(orc):
    # triangle 0-1-2 with a pendant 3 on 0: vertices 1, 2, 3 add no fill edge;
    # the fewest-neighbours rule picks 3, then the triangle by lowest id
    inst = synth.Instance("tri", np.full(4, 2, np.int32),
                          [np.array(p, np.int32) for p in ((0, 1), (1, 2), (0, 2), (0, 3))],
                          [np.zeros(4, np.int64)] * 4, "int", 1 << 30)
    order, w = orc.minfill(inst)
    assert list(order) == [3, 0, 1, 2] and w == 2


# ------------------------------------------------------ components (Sec. 6.2)
def test_components_add_up(orc):
    a = synth.random_small(31, n=5, dmax=3, n_funcs=6, with_constant=False)
    b = synth.random_small(32, n=4, dmax=3, n_funcs=5, with_constant=False)
    a.top_k = b.top_k = 10**6
    u = synth.disjoint_union(a, b)
    ra = orc.eliminate(a, orc.minfill(a)[0], "be").bound
    rb = orc.eliminate(b, orc.minfill(b)[0], "be").bound
    ru = orc.eliminate(u, orc.minfill(u)[0], "be").bound
    assert ru == ra + rb


# --------------------------------------------------------- DPOP (Section 4)
def _ancestors(parent, v):
    out = []
    v = int(parent[v])
    while v >= 0:
        out.append(v)
        v = int(parent[v])
    return out


def _descendants(parent, v):
    n = len(parent)
    return [u for u in range(n) if v in _ancestors(parent, u)]


@pytest.mark.parametrize("seed", range(4))
def test_dpop_separators(orc, seed):
    inst = synth.dcop_random(seed, n_range=(8, 14), d_range=(2, 3))
    for parent in (orc.dfs_pseudotree(inst), inst.parent):
        # every constraint joins an ancestor and a descendant (Definition 2)
        for s in inst.scopes:
            a, b = int(s[0]), int(s[1])
            assert a in _ancestors(parent, b) or b in _ancestors(parent, a)
        order = orc.pseudotree_order(inst, parent)
        run = orc.eliminate(inst, order, "be")
        linked = {v: set() for v in range(inst.n)}
        for s in inst.scopes:
            linked[int(s[0])].add(int(s[1]))
            linked[int(s[1])].add(int(s[0]))
        for T in run.tasks:
            sub = [T.var] + _descendants(parent, T.var)
            want = {a for a in _ancestors(parent, T.var) if any(a in linked[u] for u in sub)}
            assert set(int(x) for x in T.sep) == want
        best, _ = orc.bruteforce(inst) if np.prod(inst.dom.astype(float)) < 2e5 else (run.bound, None)
        assert run.bound == best


def test_dfs_pseudotree_root_and_order(orc):
    # root = highest degree; the post-order lists every node after its children
    inst = synth.dcop_random(3, n_range=(12, 12), d_range=(2, 2))
    par = orc.dfs_pseudotree(inst)
    deg = np.zeros(inst.n, int)
    for s in inst.scopes:
        deg[s] += 1
    roots = [v for v in range(inst.n) if par[v] == -1]
    assert roots[0] == int(np.argmax(deg))
    order = orc.pseudotree_order(inst, par)
    pos = {int(v): i for i, v in enumerate(order)}
    for v in range(inst.n):
        if par[v] >= 0:
            assert pos[v] < pos[int(par[v])]


# ----------------------------------------------------- MPE (Section 3)
def test_mpe_log_domain_bruteforce(orc):
    inst = synth.bayes_net_mpe(9, seed=4)
    best, sig = orc.bruteforce(inst)
    # the max-product optimum in probability space, by direct products
    pbest = 0.0
    for a in itertools.product(*[range(int(d)) for d in inst.dom]):
        p = 1.0
        for s, t in zip(inst.scopes, inst.tables):
            idx = np.ravel_multi_index([a[v] for v in s], [int(inst.dom[v]) for v in s])
            p *= np.exp(-t[idx])
        pbest = max(pbest, p)
    assert best == pytest.approx(-np.log(pbest), rel=1e-12)
    run = orc.eliminate(inst, orc.minfill(inst)[0], "be")
    assert run.bound == pytest.approx(best, rel=1e-12)


# ------------------------------------ sum-product (-log Z, solution counting)
def _z_direct(inst):
    """Z by direct products in probability space over every assignment."""
    z = 0.0
    for a in itertools.product(*[range(int(d)) for d in inst.dom]):
        p = 1.0
        for s, t in zip(inst.scopes, inst.tables):
            idx = np.ravel_multi_index([a[v] for v in s], [int(inst.dom[v]) for v in s]) if len(s) else 0
            p *= np.exp(-float(t[idx]))
        z += p
    return z


@pytest.mark.parametrize("seed", range(8))
def test_logz_bruteforce_is_the_partition_function(orc, seed):
    inst = synth.random_small(seed, n=6, dmax=3, n_funcs=8, max_arity=3, cost_type="real", p_top=0.05)
    z = _z_direct(inst)
    got = orc.logz_bruteforce(inst)
    if z == 0.0:
        assert got == np.inf
    else:
        assert got == pytest.approx(-np.log(z), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("seed", range(10))
def test_sum_elimination_equals_bruteforce(orc, seed):
    # exact BE with -log sum exp elimination reaches -log Z on any order;
    # the instances include variables in no function (a factor |D| each)
    inst = synth.random_small(seed + 100, n=7, dmax=3, n_funcs=7, max_arity=3, cost_type="real",
                              p_top=0.05)
    want = -np.log(_z_direct(inst)) if _z_direct(inst) > 0 else np.inf
    for order in (orc.minfill(inst)[0], np.arange(inst.n)[::-1]):
        run = orc.eliminate(inst, order, "be", semiring="sum")
        assert run.bound == pytest.approx(want, rel=1e-12, abs=1e-12)
        assert np.isnan(run.cost)


def test_bayes_net_partition_function_is_one(orc):
    # the CPTs of a Bayesian network multiply to a distribution: Z = 1
    inst = synth.bayes_net_mpe(40, seed=6)
    run = orc.eliminate(inst, orc.minfill(inst)[0], "be", semiring="sum")
    assert abs(run.bound) < 1e-9


def test_bayes_net_probability_of_evidence(orc):
    # evidence on x0 (no parents) and x1 (parents within {x0}):
    # P(x0 = a, x1 = b) = p(a) p(b | a), read off the two CPTs
    inst = synth.bayes_net_mpe(30, seed=2)
    assert list(inst.scopes[0]) == [0] and set(inst.scopes[1].tolist()) <= {0, 1}
    for a in range(int(inst.dom[0])):
        for b in range(int(inst.dom[1])):
            ev = synth.with_evidence(inst, {0: a, 1: b})
            run = orc.eliminate(ev, orc.minfill(ev)[0], "be", semiring="sum")
            c1 = inst.tables[1][a * int(inst.dom[1]) + b] if len(inst.scopes[1]) == 2 else inst.tables[1][b]
            assert run.bound == pytest.approx(inst.tables[0][a] + c1, rel=1e-10)


def test_ising_ring_closed_form(orc):
    # zero-field Ising ring: Z = (2 cosh J)^n + (2 sinh J)^n for the energy
    # -J sum s_v s_u; the tables add J per edge, so -log Z gains n J
    for n, J in ((8, 0.7), (11, 1.3)):
        inst = synth.ising_ring(n, J)
        want = n * J - np.log((2 * np.cosh(J)) ** n + (2 * np.sinh(J)) ** n)
        assert orc.logz_bruteforce(inst) == pytest.approx(want, rel=1e-12)
        run = orc.eliminate(inst, orc.minfill(inst)[0], "be", semiring="sum")
        assert run.bound == pytest.approx(want, rel=1e-12)


def test_coloring_counts_closed_forms(orc):
    # chromatic polynomials: cycle (q-1)^n + (-1)^n (q-1), path q (q-1)^(n-1),
    # complete graph q! / (q-n)!; an isolated vertex multiplies by q
    q = 3
    cyc = synth.coloring(7, [(v, (v + 1) % 7) for v in range(7)], q)
    path = synth.coloring(6, [(v, v + 1) for v in range(5)], q)
    k4 = synth.coloring(4, list(itertools.combinations(range(4), 2)), 5)
    iso = synth.coloring(5, [(0, 1), (1, 2), (2, 3)], q)  # vertex 4 in no constraint
    cases = [(cyc, (q - 1) ** 7 - (q - 1)), (path, q * (q - 1) ** 5), (k4, 120), (iso, q * q * (q - 1) ** 3)]
    for inst, count in cases:
        run = orc.eliminate(inst, orc.minfill(inst)[0], "be", semiring="sum")
        assert np.exp(-run.bound) == pytest.approx(count, rel=1e-12)
        assert orc.logz_bruteforce(orc.counting_instance(inst)) == pytest.approx(-np.log(count), rel=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_sum_minibuckets_bound_and_exactness(orc, seed):
    # each mini-bucket summed on its own can only enlarge Z: the mini-bucket
    # -log Z is a lower bound, exact once the bound admits the whole bucket
    inst = synth.random_small(seed + 200, n=9, dmax=3, n_funcs=12, max_arity=3, cost_type="real",
                              p_top=0.0)
    order, _ = orc.minfill(inst)
    exact = orc.eliminate(inst, order, "be", semiring="sum")
    assert exact.bound == pytest.approx(orc.logz_bruteforce(inst), rel=1e-11, abs=1e-11)
    for z in (1, 2, 3):
        mb = orc.eliminate(inst, order, "sep", z, semiring="sum")
        assert mb.bound <= exact.bound + 1e-9
    full = orc.eliminate(inst, order, "sep", exact.width, semiring="sum")
    assert full.bound == pytest.approx(exact.bound, rel=1e-12, abs=1e-12)


def test_sum_components_multiply(orc):
    # Z of a disjoint union is the product of the parts' Z
    a = synth.random_small(41, n=5, dmax=3, n_funcs=6, cost_type="real", p_top=0.0)
    b = synth.random_small(42, n=4, dmax=3, n_funcs=5, cost_type="real", p_top=0.0)
    u = synth.disjoint_union(a, b)
    za = orc.eliminate(a, orc.minfill(a)[0], "be", semiring="sum").bound
    zb = orc.eliminate(b, orc.minfill(b)[0], "be", semiring="sum").bound
    zu = orc.eliminate(u, orc.minfill(u)[0], "be", semiring="sum").bound
    assert zu == pytest.approx(za + zb, rel=1e-12)
