"""Seeded instance generators.

Every generator takes an integer seed and returns an :class:`Instance`.  The
instances follow the shapes of the paper's workloads (grid, Erdos-Renyi random,
scale-free networks, Section 8.1; Bayesian networks, Section 3; DCOPs,
Section 4) with the sizes of the five benchmark configurations.  Nothing here
orders, eliminates or evaluates anything: it only draws variables, domains,
scopes and cost tables.

Table layout: ``tables[j]`` is a flat array, row-major over ``scopes[j]`` as
given (the first scope variable varies slowest), so its length is the product
of the scope's domain sizes.  Integer instances hold costs in ``[0, top_k]``
(``top_k`` = infeasible); real instances hold ``-log p`` in float64 (``+inf``
where ``p = 0``).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

TOP_K = 1 << 30  # the WCSP top cost k used by every integer configuration


@dataclass
class Instance:
    name: str
    dom: np.ndarray                      # int32 [n]
    scopes: list                         # list of int32 arrays
    tables: list                         # list of int64 (int) / float64 (real) arrays
    cost_type: str = "int"               # "int" (saturating at top_k) or "real" (-log p)
    top_k: int = TOP_K
    parent: Optional[np.ndarray] = None  # pseudo-tree (DCOPs), -1 = root
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.dom.shape[0])

    @property
    def n_funcs(self) -> int:
        return len(self.scopes)

    def packed(self):
        """CSR arrays: scope_off[int32, F+1], scope[int32], tab_off[int64, F+1], costs."""
        F = len(self.scopes)
        scope_off = np.zeros(F + 1, dtype=np.int32)
        tab_off = np.zeros(F + 1, dtype=np.int64)
        for j, s in enumerate(self.scopes):
            scope_off[j + 1] = scope_off[j] + len(s)
            tab_off[j + 1] = tab_off[j] + len(self.tables[j])
        scope = (np.concatenate([np.asarray(s, dtype=np.int32) for s in self.scopes])
                 if F and scope_off[-1] > 0 else np.zeros(0, dtype=np.int32))
        if self.cost_type == "int":
            costs = (np.concatenate([np.asarray(t, dtype=np.int64) for t in self.tables])
                     if F else np.zeros(0, dtype=np.int64))
        else:
            costs = (np.concatenate([np.asarray(t, dtype=np.float64) for t in self.tables])
                     if F else np.zeros(0, dtype=np.float64))
        return scope_off, scope, tab_off, costs


def _table_size(dom, scope):
    size = 1
    for v in scope:
        size *= int(dom[v])
    return size


def _int_table(rng, dom, scope, lo, hi, p_top, top_k):
    t = rng.integers(lo, hi + 1, size=_table_size(dom, scope), dtype=np.int64)
    if p_top > 0:
        t[rng.random(t.shape[0]) < p_top] = top_k
    return t


# --------------------------------------------------------------------------- grid
def grid_wcsp(rows, cols, d, seed, lo=0, hi=100, unary=True, p_top=0.0,
              top_k=TOP_K, name=None):
    """Grid network (Section 8.1): node (r, c) has id r*cols + c and is linked to
    its right and lower neighbours; one binary table per edge, optional unary
    tables, integer costs uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    n = rows * cols
    dom = np.full(n, d, dtype=np.int32)
    scopes, tables = [], []
    if unary:
        for v in range(n):
            scopes.append(np.array([v], dtype=np.int32))
            tables.append(_int_table(rng, dom, [v], lo, hi, p_top, top_k))
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            if c + 1 < cols:
                scopes.append(np.array([v, v + 1], dtype=np.int32))
                tables.append(_int_table(rng, dom, [v, v + 1], lo, hi, p_top, top_k))
            if r + 1 < rows:
                scopes.append(np.array([v, v + cols], dtype=np.int32))
                tables.append(_int_table(rng, dom, [v, v + cols], lo, hi, p_top, top_k))
    return Instance(name or f"grid{rows}x{cols}_d{d}_s{seed}", dom, scopes, tables,
                    "int", top_k, meta={"rows": rows, "cols": cols, "seed": seed})


# --------------------------------------------------------------------------- Erdos-Renyi
def er_wcsp(n, seed, dmin=2, dmax=8, n_tables=1500, arity=3, lo=0, hi=500,
            p_top=0.05, top_k=TOP_K, name=None):
    """Random WCSP: ``n_tables`` cost tables on uniformly random distinct
    variable sets of size ``arity`` (scope order as drawn), domains uniform in
    {dmin..dmax}, costs uniform in [lo, hi] with a fraction ``p_top`` of the
    entries set to the top cost."""
    rng = np.random.default_rng(seed)
    dom = rng.integers(dmin, dmax + 1, size=n).astype(np.int32)
    seen = set()
    scopes, tables = [], []
    while len(scopes) < n_tables:
        s = rng.choice(n, size=arity, replace=False).astype(np.int32)
        key = tuple(sorted(int(x) for x in s))
        if key in seen:
            continue
        seen.add(key)
        scopes.append(s)
        tables.append(_int_table(rng, dom, s, lo, hi, p_top, top_k))
    return Instance(name or f"er{n}_t{n_tables}_s{seed}", dom, scopes, tables, "int",
                    top_k, meta={"seed": seed})


# --------------------------------------------------------------------------- Bayesian network
def bayes_net_mpe(n, seed, doms=(2, 3), max_parents=3, name=None):
    """Random Bayesian network (Section 3): variable v draws its number of
    parents uniformly in {0..min(max_parents, v)} and the parents uniformly
    among the earlier variables; each CPT row (one per parent configuration) is
    a Dirichlet(1) draw.  Costs are -log p in float64; the scope of CPT v is
    (sorted parents..., v), v varying fastest."""
    rng = np.random.default_rng(seed)
    dom = rng.choice(np.asarray(doms, dtype=np.int32), size=n).astype(np.int32)
    scopes, tables = [], []
    for v in range(n):
        k = int(rng.integers(0, min(max_parents, v) + 1))
        pa = np.sort(rng.choice(v, size=k, replace=False)).astype(np.int32) if k else \
            np.zeros(0, dtype=np.int32)
        scope = np.concatenate([pa, np.array([v], dtype=np.int32)])
        rows = _table_size(dom, pa)
        p = rng.dirichlet(np.ones(int(dom[v])), size=rows).reshape(-1)
        with np.errstate(divide="ignore"):
            cost = -np.log(p)
        scopes.append(scope)
        tables.append(cost.astype(np.float64))
    return Instance(name or f"bn{n}_s{seed}", dom, scopes, tables, "real", TOP_K,
                    meta={"seed": seed})


def bn_prefix(inst, m):
    """The first ``m`` variables of a Bayesian network and their CPTs (closed
    under parents, because parents always precede their child)."""
    keep = [j for j, s in enumerate(inst.scopes) if int(np.max(s)) < m]
    return Instance(f"{inst.name}_prefix{m}", inst.dom[:m].copy(),
                    [inst.scopes[j].copy() for j in keep],
                    [inst.tables[j].copy() for j in keep], inst.cost_type, inst.top_k,
                    meta=dict(inst.meta, prefix=m))


# --------------------------------------------------------------------------- DCOP
def dcop_random(seed, n_range=(20, 200), d_range=(5, 10), density=(0.1, 0.3),
                sep_cap=8, lo=0, hi=100, tree_window=None, top_k=TOP_K, name=None):
    """Random DCOP with a bounded separator.

    A random rooted tree is drawn (node v > 0 picks its parent uniformly among
    the ``tree_window`` previous nodes; all previous nodes when None).  Every
    tree edge is a binary constraint.  Each other ancestor/descendant pair is
    then considered in random order and linked with probability ``p`` (drawn
    uniformly from ``density``) unless the link would give some node more than
    ``sep_cap`` constrained ancestors in its subtree.  All links join an
    ancestor and a descendant, so the tree is a DFS pseudo-tree of the
    constraint graph; ``parent`` returns it.  Costs are uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    dom = rng.integers(d_range[0], d_range[1] + 1, size=n).astype(np.int32)
    p = float(rng.uniform(density[0], density[1]))
    parent = np.full(n, -1, dtype=np.int32)
    for v in range(1, n):
        w = v if tree_window is None else min(v, tree_window)
        parent[v] = int(rng.integers(v - w, v))
    # linked ancestors of every node's subtree (the separator of Section 4)
    sep = [set() for _ in range(n)]
    edges = []

    def path_to(u, a):
        out = []
        while u != a:
            out.append(u)
            u = int(parent[u])
        return out

    def add_edge(u, a):
        for w in path_to(u, a):
            sep[w].add(a)
        edges.append((a, u))

    for v in range(1, n):
        add_edge(v, int(parent[v]))
    if any(len(s) > sep_cap for s in sep):  # a tree alone has separators of size 1
        raise AssertionError("tree separators exceed the cap")
    cand = []
    for v in range(n):
        a = int(parent[v]) if v else -1
        a = int(parent[a]) if a >= 0 else -1
        while a >= 0:
            cand.append((v, a))
            a = int(parent[a])
    order = rng.permutation(len(cand))
    for i in order:
        u, a = cand[int(i)]
        if rng.random() >= p:
            continue
        if all(len(sep[w] | {a}) <= sep_cap for w in path_to(u, a)):
            add_edge(u, a)
    scopes, tables = [], []
    for a, u in edges:
        s = np.array(sorted((a, u)), dtype=np.int32)
        scopes.append(s)
        tables.append(_int_table(rng, dom, s, lo, hi, 0.0, top_k))
    achieved = len(edges) / (n * (n - 1) / 2)
    return Instance(name or f"dcop{n}_s{seed}", dom, scopes, tables, "int", top_k,
                    parent=parent,
                    meta={"seed": seed, "p": p, "density": achieved,
                          "max_sep": max(len(s) for s in sep)})


def dcop_stream(n_requests, seed, rate_per_s, **kw):
    """A Poisson stream: arrival times (seconds, exponential gaps of mean
    1/rate) and a seeded DCOP per request."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    seeds = rng.integers(0, 2**31 - 1, size=n_requests)
    return arrivals, [int(s) for s in seeds]


# --------------------------------------------------------------------------- paper sweeps
def random_network_wcsp(n, d, p1, seed, p2=0.5, lo=0, hi=100, top_k=TOP_K, name=None):
    """Random binary network (Section 8.1): floor(p1 * n(n-1)/2) distinct edges,
    redrawn until connected; a fraction p2 of each table's entries is
    infeasible, the rest uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    m = int(np.floor(p1 * n * (n - 1) / 2))
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    while True:
        pick = rng.choice(len(pairs), size=max(m, n - 1), replace=False)
        edges = [pairs[int(i)] for i in pick]
        if _connected(n, edges):
            break
    dom = np.full(n, d, dtype=np.int32)
    scopes = [np.array(e, dtype=np.int32) for e in edges]
    tables = [_int_table(rng, dom, s, lo, hi, p2, top_k) for s in scopes]
    return Instance(name or f"rand{n}_d{d}_p{p1}_s{seed}", dom, scopes, tables, "int",
                    top_k, meta={"seed": seed})


def scale_free_wcsp(n, d, seed, p2=0.5, lo=0, hi=100, top_k=TOP_K, name=None):
    """Barabasi-Albert network as in Section 8.1: start from one edge and add
    nodes linked to two distinct existing nodes drawn with probability
    proportional to their degree (2(n-2)+1 edges)."""
    rng = np.random.default_rng(seed)
    edges = [(0, 1)]
    deg = np.zeros(n, dtype=np.float64)
    deg[0] = deg[1] = 1
    for v in range(2, n):
        w = deg[:v] / deg[:v].sum()
        a, b = rng.choice(v, size=2, replace=False, p=w)
        edges += [(int(a), v), (int(b), v)]
        deg[a] += 1
        deg[b] += 1
        deg[v] = 2
    dom = np.full(n, d, dtype=np.int32)
    scopes = [np.array(e, dtype=np.int32) for e in edges]
    tables = [_int_table(rng, dom, s, lo, hi, p2, top_k) for s in scopes]
    return Instance(name or f"sf{n}_d{d}_s{seed}", dom, scopes, tables, "int", top_k,
                    meta={"seed": seed})


def _connected(n, edges):
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    seen = {0}
    stack = [0]
    while stack:
        u = stack.pop()
        for w in adj[u]:
            if w not in seen:
                seen.add(w)
                stack.append(w)
    return len(seen) == n


# --------------------------------------------------------------------------- small cases
def random_small(seed, n=6, dmax=3, n_funcs=8, max_arity=3, cost_type="int",
                 p_top=0.1, hi=20, with_constant=True, dmin=1, top_k=None):
    """Tiny random instance for exhaustive checks: mixed arities 0..max_arity
    (scope order as drawn, repeated scopes allowed), domains in {dmin..dmax}."""
    rng = np.random.default_rng(seed)
    dom = rng.integers(dmin, dmax + 1, size=n).astype(np.int32)
    k = top_k if top_k is not None else (hi * n_funcs + 1 if cost_type == "int" else TOP_K)
    scopes, tables = [], []
    for j in range(n_funcs):
        a = int(rng.integers(1, min(max_arity, n) + 1))
        if with_constant and j == 0:
            a = 0
        s = rng.choice(n, size=a, replace=False).astype(np.int32)
        scopes.append(s)
        size = _table_size(dom, s)
        if cost_type == "int":
            t = rng.integers(0, hi + 1, size=size, dtype=np.int64)
            t[rng.random(size) < p_top] = k
        else:
            t = -np.log(rng.uniform(0.02, 1.0, size=size))
            t[rng.random(size) < p_top] = np.inf
        tables.append(t)
    return Instance(f"small_s{seed}", dom, scopes, tables, cost_type, k, meta={"seed": seed})


def paper_example(seed=0, hi=9):
    """The 4-variable binary example of Section 2 (Example 1): constraints
    f(x1,x2), f(x1,x4), f(x2,x3), f(x2,x4), f(x3,x4); x1..x4 are ids 0..3.  The
    paper's cost tables are in a figure that is not available, so the costs
    are drawn at random."""
    rng = np.random.default_rng(seed)
    dom = np.full(4, 2, dtype=np.int32)
    pairs = [(0, 1), (0, 3), (1, 2), (1, 3), (2, 3)]
    scopes = [np.array(p, dtype=np.int32) for p in pairs]
    tables = [rng.integers(0, hi + 1, size=4, dtype=np.int64) for _ in pairs]
    return Instance("paper_example", dom, scopes, tables, "int", TOP_K)


def disjoint_union(a, b):
    """Two instances side by side (variables of b shifted by a.n)."""
    dom = np.concatenate([a.dom, b.dom]).astype(np.int32)
    scopes = [s.copy() for s in a.scopes] + [s + a.n for s in b.scopes]
    tables = [t.copy() for t in a.tables] + [t.copy() for t in b.tables]
    return Instance(f"{a.name}+{b.name}", dom, scopes, tables, a.cost_type,
                    a.top_k, meta={"parts": [a.n, b.n]})


def grid_mrf(rows, cols, d, seed, scale=1.0, unary=True, name=None):
    """Pairwise Markov random field on a rows x cols grid (variable r*cols+c):
    real costs (-log potentials) U[0, scale] on every edge (and vertex) table,
    the workload shape of the grid instances with weights instead of integer
    costs."""
    rng = np.random.default_rng(seed)
    n = rows * cols
    dom = np.full(n, d, dtype=np.int32)
    scopes, tables = [], []
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            if unary:
                scopes.append(np.array([v], dtype=np.int32))
                tables.append(rng.uniform(0.0, scale, size=d))
            for u in ((v + 1) if c + 1 < cols else None, (v + cols) if r + 1 < rows else None):
                if u is not None:
                    scopes.append(np.array([v, u], dtype=np.int32))
                    tables.append(rng.uniform(0.0, scale, size=d * d))
    return Instance(name or f"mrf{rows}x{cols}_d{d}_s{seed}", dom, scopes, tables, "real", TOP_K,
                    meta={"seed": seed, "rows": rows, "cols": cols})


def ising_ring(n, J):
    """Zero-field Ising ring of n spins s_v = 2 x_v - 1 with coupling J > 0:
    edge (v, v+1 mod n) has energy J - J s_v s_u >= 0 (0 when aligned, 2J
    when not), as a real cost table over (x_v, x_u)."""
    dom = np.full(n, 2, dtype=np.int32)
    scopes = [np.array(sorted((v, (v + 1) % n)), dtype=np.int32) for v in range(n)]
    tab = np.array([0.0, 2.0 * J, 2.0 * J, 0.0])
    return Instance(f"ising_ring{n}_J{J}", dom, scopes, [tab.copy() for _ in range(n)], "real", TOP_K,
                    meta={"J": J})


def coloring(n, edges, q, top_k=1 << 10):
    """Proper q-colouring as a WCSP: on each edge, equal colours cost the top
    cost, different colours cost 0."""
    dom = np.full(n, q, dtype=np.int32)
    eq = np.where(np.eye(q, dtype=bool).reshape(-1), top_k, 0).astype(np.int64)
    scopes = [np.array(e, dtype=np.int32) for e in edges]
    return Instance(f"color{n}_q{q}", dom, scopes, [eq.copy() for _ in edges], "int", top_k)


def with_evidence(inst, evidence, declared=None):
    """The instance with variables clamped: for each (v, value) a unary table
    that is 0 at value and infinite (the top cost for a WCSP) elsewhere.
    With ``declared`` (a list of variables), one unary table is appended per
    declared variable in that order instead: the clamp when the variable is
    in ``evidence`` (and its value is not -1 / None), all zero otherwise."""
    inf = np.inf if inst.cost_type == "real" else inst.top_k
    dt = np.float64 if inst.cost_type == "real" else np.int64
    scopes = [s.copy() for s in inst.scopes]
    tables = [t.copy() for t in inst.tables]
    for v in (declared if declared is not None else list(evidence.keys())):
        val = evidence.get(v)
        if val is None or val < 0:
            t = np.zeros(int(inst.dom[v]), dtype=dt)
        else:
            t = np.full(int(inst.dom[v]), inf, dtype=dt)
            t[val] = 0
        scopes.append(np.array([v], dtype=np.int32))
        tables.append(t)
    return Instance(inst.name + "_ev", inst.dom.copy(), scopes, tables, inst.cost_type, inst.top_k,
                    meta=dict(inst.meta, evidence=dict(evidence)))


# --------------------------------------------------------------------------- configurations
def config_instance(idx, seed=0):
    """The five benchmark workloads by index:

    0: 4x5 grid, d=4, binary + unary tables, costs U[0,100] (exact BE);
    1: 12x12 grid, d=4, binary tables U[0,1000] (exact BE, largest tables);
    2: Erdos-Renyi, 500 variables, domains U{2..8}, 1500 ternary tables
       U[0,500], 5% entries = top (mini-buckets);
    3: Bayesian network, 200 variables, domains {2,3}, <= 3 parents,
       Dirichlet(1) CPTs (MPE in the -log domain);
    4: one DCOP of the request stream (20-200 agents, domains 5-10, costs
       U[0,100], separators <= 8).
    """
    if idx == 0:
        return grid_wcsp(4, 5, 4, seed, 0, 100, unary=True)
    if idx == 1:
        return grid_wcsp(12, 12, 4, seed, 0, 1000, unary=False)
    if idx == 2:
        return er_wcsp(500, seed)
    if idx == 3:
        return bayes_net_mpe(200, seed)
    if idx == 4:
        return dcop_random(seed)
    raise ValueError(idx)
