"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare it with the oracle."""
import numpy as np

import paper_1608_05288_gb300 as gb

# Floating-point tolerance of the -log p (MPE) path: fp32 sums of fp32-rounded
# inputs against an fp64 oracle, |delta| <= 1e-4 * (1 + |value|).
FP_RTOL = 1e-4


def fp_close(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    both_inf = np.isinf(a) & np.isinf(b) & (np.sign(a) == np.sign(b))
    with np.errstate(invalid="ignore"):
        ok = both_inf | (np.abs(a - b) <= FP_RTOL * (1.0 + np.abs(b)))
    return bool(np.all(ok))


def structure(st):
    return [(int(t["var"]), [int(x) for x in t["sep"]], sorted(int(x) for x in t["inputs"]))
            for t in st.tasks()]


def orc_structure(run):
    return [(int(t.var), [int(x) for x in t.sep], sorted(int(x) for x in t.inputs)) for t in run.tasks]


def run_state(inst, kind="be", i_bound=0, parent=None, **opts):
    st = gb.UtilState(inst, kind, i_bound, parent=parent, **opts)
    st.bind()
    st.run()
    res = st.value()
    st.sync()
    return st, res


def check_tables(inst, st, run, exact=True):
    """Every bucket function and argmin table against the oracle's (a task
    that writes no argmin table reads back zeros)."""
    assert structure(st) == orc_structure(run)
    tasks = st.tasks()
    for t, T in enumerate(run.tasks):
        keeps = tasks[t]["argmin"]
        cost, arg = st.fetch(t)
        if exact:
            assert np.array_equal(cost.astype(np.int64), T.out.astype(np.int64)), f"task {t} costs"
        else:
            assert fp_close(cost, T.out), f"task {t} costs"
        if not keeps:
            assert not np.any(arg), f"task {t}: no argmin table was kept"
        elif exact:
            assert np.array_equal(arg, T.arg), f"task {t} argmin"
        else:
            assert argmin_attains_minimum(inst, run, t, arg), f"task {t} argmin"


def bucket_sums_at(dom, var, sep, rows_idx, values, inputs):
    """fp64 sum of a bucket's input tables at separator rows rows_idx (row-major
    over sep) with the eliminated variable var at values[i]; inputs = list of
    (scope, table), each table row-major over its scope as listed."""
    sep = [int(x) for x in sep]
    digits = np.unravel_index(rows_idx, [int(dom[x]) for x in sep]) if sep else ()
    val = {x: digits[i] for i, x in enumerate(sep)}
    val[int(var)] = np.asarray(values, dtype=np.int64)
    s = np.zeros(len(rows_idx))
    for scope, tab in inputs:
        flat = np.zeros(len(rows_idx), dtype=np.int64)
        stride = 1
        for x in reversed([int(y) for y in scope]):
            flat += val[x] * stride
            stride *= int(dom[x])
        s += np.asarray(tab, dtype=np.float64)[flat]
    return s


def argmin_attains_minimum(inst, run, t, arg, max_rows=1 << 16):
    """The GPU's argmin of oracle task t, checked independently of the GPU's
    cost table: the bucket's sum at the chosen value, recomputed in fp64 from
    the oracle's input tables, must equal the oracle's minimum within
    1e-4 (1 + |min|) (+inf rows: +inf).  Rows are all of them, or a seeded
    sample of max_rows for large tables."""
    T = run.tasks[t]
    rows = int(T.rows)
    arg = np.asarray(arg)
    if np.any(arg[: min(rows, 1 << 20)] >= int(inst.dom[T.var])):
        return False
    if rows <= max_rows:
        idx = np.arange(rows)
    else:
        idx = np.sort(np.random.default_rng(1000 + t).choice(rows, size=max_rows, replace=False))
    nf = inst.n_funcs
    inputs = []
    for fid in T.inputs:
        fid = int(fid)
        if fid < nf:
            inputs.append((inst.scopes[fid], inst.tables[fid]))
        else:
            U = run.tasks[fid - nf]
            inputs.append((U.sep, U.out))
    s = bucket_sums_at(inst.dom, T.var, T.sep, idx, arg[idx], inputs)
    if inst.cost_type == "int":
        s = np.minimum(s, inst.top_k)
    return fp_close(s, np.asarray(T.out)[idx])
