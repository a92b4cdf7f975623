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
    """Every bucket function and argmin table against the oracle's."""
    assert structure(st) == orc_structure(run)
    for t, T in enumerate(run.tasks):
        cost, arg = st.fetch(t)
        if exact:
            assert np.array_equal(cost.astype(np.int64), T.out.astype(np.int64)), f"task {t} costs"
            assert np.array_equal(arg, T.arg), f"task {t} argmin"
        else:
            assert fp_close(cost, T.out), f"task {t} costs"
            # argmin: the chosen value must attain the oracle's minimum within tolerance
            assert np.all(arg < inst.dom[T.var])
