"""ctypes front end of the C oracle.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use this package; the product library never
does.  The oracle is a plain, slow, sequential restatement of the paper's
Algorithms 1-2, Eq. 1 and Eq. 3 (see ``oracle.c`` for the readings it takes).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None

BE, MBE_SEP, MBE_JOINT, MBE_LOG2 = 0, 1, 2, 3
MODES = {"be": BE, "sep": MBE_SEP, "joint": MBE_JOINT, "log2": MBE_LOG2}
SEMIRINGS = {"min": 0, "sum": 1}   # min-sum (optimisation) / sum-product (-log Z)


class _Problem(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("dom", C.POINTER(C.c_int)), ("nf", C.c_int),
        ("scope_off", C.POINTER(C.c_int)), ("scope", C.POINTER(C.c_int)),
        ("tab_off", C.POINTER(C.c_longlong)), ("cost", C.POINTER(C.c_double)),
        ("saturate", C.c_int), ("top", C.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        _lib = _configure(C.CDLL(_build.build()))
    return _lib


class use_library:
    """Context manager: run the oracle functions against another build of
    oracle.c (used by the tests that plant mistakes in a copy of it)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = _configure(C.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def _configure(L):
    if True:
        P = C.POINTER(_Problem)
        ip = C.POINTER(C.c_int)
        L.orc_eval.argtypes = [P, ip]
        L.orc_eval.restype = C.c_double
        L.orc_bruteforce.argtypes = [P, ip]
        L.orc_bruteforce.restype = C.c_double
        L.orc_induced_width.argtypes = [P, ip]
        L.orc_minfill.argtypes = [P, ip]
        L.orc_dfs_pseudotree.argtypes = [P, ip]
        L.orc_pseudotree_order.argtypes = [P, ip, ip]
        L.orc_project_index.argtypes = [C.c_int, ip, C.c_int, ip, C.c_longlong]
        L.orc_project_index.restype = C.c_longlong
        L.orc_util_bucket.argtypes = [C.c_int, ip, C.c_int, C.c_int,
                                      C.POINTER(C.POINTER(C.c_double)), ip, ip, C.c_int,
                                      C.c_double, C.POINTER(C.c_double),
                                      C.POINTER(C.c_ubyte)]
        L.orc_eliminate.argtypes = [P, ip, C.c_int, C.c_int]
        L.orc_eliminate.restype = C.c_void_p
        L.orc_eliminate_sr.argtypes = [P, ip, C.c_int, C.c_int, C.c_int]
        L.orc_eliminate_sr.restype = C.c_void_p
        L.orc_sum_bruteforce.argtypes = [P]
        L.orc_sum_bruteforce.restype = C.c_double
        L.orc_run_ntasks.argtypes = [C.c_void_p]
        L.orc_run_bound.argtypes = [C.c_void_p]
        L.orc_run_bound.restype = C.c_double
        L.orc_run_cost.argtypes = [C.c_void_p]
        L.orc_run_cost.restype = C.c_double
        L.orc_run_width.argtypes = [C.c_void_p]
        L.orc_run_sigma.argtypes = [C.c_void_p, ip]
        L.orc_run_task.argtypes = [C.c_void_p, C.c_int, ip, ip, ip, ip, ip,
                                   C.POINTER(C.c_longlong)]
        L.orc_run_table.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_double),
                                    C.POINTER(C.c_ubyte)]
        L.orc_run_free.argtypes = [C.c_void_p]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_max_threads.restype = C.c_int
    return L


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


class Problem:
    """Keeps the packed arrays alive for the C structure."""

    def __init__(self, inst):
        self.inst = inst
        self.dom = np.ascontiguousarray(inst.dom, dtype=np.int32)
        so, sc, to, costs = inst.packed()
        self.scope_off = np.ascontiguousarray(so, dtype=np.int32)
        self.scope = np.ascontiguousarray(sc if sc.size else np.zeros(1, np.int32), dtype=np.int32)
        self.tab_off = np.ascontiguousarray(to, dtype=np.int64)
        self.cost = np.ascontiguousarray(costs if costs.size else np.zeros(1), dtype=np.float64)
        self.s = _Problem(inst.n, _iptr(self.dom), inst.n_funcs, _iptr(self.scope_off),
                          _iptr(self.scope), self.tab_off.ctypes.data_as(C.POINTER(C.c_longlong)),
                          self.cost.ctypes.data_as(C.POINTER(C.c_double)),
                          1 if inst.cost_type == "int" else 0, float(inst.top_k))

    @property
    def ref(self):
        return C.byref(self.s)


def set_threads(t):
    lib().orc_set_threads(int(t))


def max_threads():
    return int(lib().orc_max_threads())


def evaluate(inst, sigma):
    p = Problem(inst)
    s = np.ascontiguousarray(sigma, dtype=np.int32)
    return lib().orc_eval(p.ref, _iptr(s))


def bruteforce(inst):
    p = Problem(inst)
    s = np.zeros(max(inst.n, 1), dtype=np.int32)
    best = lib().orc_bruteforce(p.ref, _iptr(s))
    return best, s[: inst.n]


def logz_bruteforce(inst):
    """-log Z by enumeration, Z = sum over all assignments of exp(-Eq. 1 cost)
    (real costs; for a WCSP pass counting_instance(inst))."""
    p = Problem(inst)  # keeps the packed arrays alive during the call
    return lib().orc_sum_bruteforce(p.ref)


def counting_instance(inst):
    """The weights whose partition function counts a WCSP's consistent
    solutions (Section 2.1): every entry below the top cost has weight 1
    (-log weight 0), every entry at or above it weight 0 (+inf).  A real-cost
    instance is returned unchanged."""
    if inst.cost_type != "int":
        return inst
    from dataclasses import replace
    tabs = [np.where(np.asarray(t) >= inst.top_k, np.inf, 0.0).astype(np.float64) for t in inst.tables]
    return replace(inst, tables=tabs, cost_type="real", name=inst.name + "_count")


def induced_width(inst, order):
    p = Problem(inst)
    o = np.ascontiguousarray(order, dtype=np.int32)
    return int(lib().orc_induced_width(p.ref, _iptr(o)))


def minfill(inst):
    p = Problem(inst)
    o = np.zeros(max(inst.n, 1), dtype=np.int32)
    w = lib().orc_minfill(p.ref, _iptr(o))
    return o[: inst.n], int(w)


def natural_order(inst):
    return np.arange(inst.n, dtype=np.int32)


def best_order(inst):
    """Min-fill unless the natural (ascending id) order has a smaller induced
    width; ties keep min-fill."""
    mf, wm = minfill(inst)
    nat = natural_order(inst)
    wn = induced_width(inst, nat)
    return (nat, wn) if wn < wm else (mf, wm)


def dfs_pseudotree(inst):
    p = Problem(inst)
    par = np.zeros(max(inst.n, 1), dtype=np.int32)
    lib().orc_dfs_pseudotree(p.ref, _iptr(par))
    return par[: inst.n]


def pseudotree_order(inst, parent):
    p = Problem(inst)
    par = np.ascontiguousarray(parent, dtype=np.int32)
    o = np.zeros(max(inst.n, 1), dtype=np.int32)
    lib().orc_pseudotree_order(p.ref, _iptr(par), _iptr(o))
    return o[: inst.n]


def project_index(out_dom, phi, r_out):
    """Eq. 3: input-table row for output row r_out."""
    od = np.ascontiguousarray(out_dom, dtype=np.int32)
    ph = np.ascontiguousarray(phi, dtype=np.int32)
    return int(lib().orc_project_index(len(od), _iptr(od), len(ph), _iptr(ph), int(r_out)))


def util_bucket(sep_dom, d, tables, positions, saturate, top):
    """One bucket by aggregation (Eq. 3) then elimination: returns (out, arg).
    tables[i] is row-major over (sep vars at positions[i] ascending, eliminated var)."""
    sd = np.ascontiguousarray(sep_dom if len(sep_dom) else [1], dtype=np.int32)
    rows = int(np.prod([int(x) for x in sep_dom])) if len(sep_dom) else 1
    tabs = [np.ascontiguousarray(t, dtype=np.float64) for t in tables]
    arr = (C.POINTER(C.c_double) * max(len(tabs), 1))(
        *[t.ctypes.data_as(C.POINTER(C.c_double)) for t in tabs])
    ns = np.array([len(p) for p in positions] or [0], dtype=np.int32)
    pos = np.array([x for p in positions for x in p] or [0], dtype=np.int32)
    out = np.zeros(rows, dtype=np.float64)
    arg = np.zeros(rows, dtype=np.uint8)
    lib().orc_util_bucket(len(sep_dom), _iptr(sd), int(d), len(tabs), arr, _iptr(ns), _iptr(pos),
                          1 if saturate else 0, float(top),
                          out.ctypes.data_as(C.POINTER(C.c_double)),
                          arg.ctypes.data_as(C.POINTER(C.c_ubyte)))
    return out, arg


@dataclass
class Task:
    var: int
    sep: np.ndarray
    inputs: np.ndarray     # creation ids (originals 0..F-1, task t's output F+t)
    rows: int
    out: np.ndarray = None
    arg: np.ndarray = None


@dataclass
class Run:
    order: np.ndarray
    tasks: list
    bound: float
    sigma: np.ndarray
    cost: float
    width: int


def eliminate(inst, order, mode="be", z=0, tables=True, semiring="min"):
    """Algorithm 1 (mode "be") or Algorithm 2 (modes "sep", "joint", "log2"
    with bound z) along ``order``, then the value-assignment phase.  With
    semiring "sum" every bucket is eliminated by -log sum exp(-.) instead of
    min (the bound is then -log Z, or its mini-bucket lower bound, and there
    is no value phase); a WCSP is first turned into its counting instance."""
    if semiring == "sum":
        inst = counting_instance(inst)
    p = Problem(inst)
    o = np.ascontiguousarray(order, dtype=np.int32)
    L = lib()
    h = L.orc_eliminate_sr(p.ref, _iptr(o), MODES[mode], int(z), SEMIRINGS[semiring])
    try:
        nt = L.orc_run_ntasks(h)
        tasks = []
        sep = np.zeros(max(inst.n, 1), dtype=np.int32)
        ids = np.zeros(inst.n_funcs + inst.n + 8, dtype=np.int32)
        for t in range(nt):
            var, ns, ni = C.c_int(), C.c_int(), C.c_int()
            rows = C.c_longlong()
            L.orc_run_task(h, t, C.byref(var), C.byref(ns), _iptr(sep), C.byref(ni), _iptr(ids),
                           C.byref(rows))
            T = Task(var.value, sep[: ns.value].copy(), ids[: ni.value].copy(), rows.value)
            if tables:
                T.out = np.zeros(rows.value, dtype=np.float64)
                T.arg = np.zeros(rows.value, dtype=np.uint8)
                L.orc_run_table(h, t, T.out.ctypes.data_as(C.POINTER(C.c_double)),
                                T.arg.ctypes.data_as(C.POINTER(C.c_ubyte)))
            tasks.append(T)
        sig = np.zeros(max(inst.n, 1), dtype=np.int32)
        L.orc_run_sigma(h, _iptr(sig))
        return Run(o.copy(), tasks, L.orc_run_bound(h), sig[: inst.n], L.orc_run_cost(h),
                   int(L.orc_run_width(h)))
    finally:
        L.orc_run_free(h)


class Handle:
    """A finished oracle run kept in C memory, read one table at a time
    (for full-size comparisons that do not fit twice in host memory)."""

    def __init__(self, inst, order, mode="be", z=0, semiring="min"):
        if semiring == "sum":
            inst = counting_instance(inst)
        self.inst = inst
        self.p = Problem(inst)
        o = np.ascontiguousarray(order, dtype=np.int32)
        self.h = lib().orc_eliminate_sr(self.p.ref, _iptr(o), MODES[mode], int(z), SEMIRINGS[semiring])

    @property
    def ntasks(self):
        return lib().orc_run_ntasks(self.h)

    @property
    def bound(self):
        return lib().orc_run_bound(self.h)

    @property
    def cost(self):
        return lib().orc_run_cost(self.h)

    def sigma(self):
        s = np.zeros(max(self.inst.n, 1), dtype=np.int32)
        lib().orc_run_sigma(self.h, _iptr(s))
        return s[: self.inst.n]

    def task(self, t, table=True):
        var, ns, ni = C.c_int(), C.c_int(), C.c_int()
        rows = C.c_longlong()
        sep = np.zeros(max(self.inst.n, 1), dtype=np.int32)
        ids = np.zeros(self.inst.n_funcs + self.inst.n + 8, dtype=np.int32)
        lib().orc_run_task(self.h, int(t), C.byref(var), C.byref(ns), _iptr(sep), C.byref(ni),
                           _iptr(ids), C.byref(rows))
        T = Task(var.value, sep[: ns.value].copy(), ids[: ni.value].copy(), rows.value)
        if table:
            T.out = np.zeros(rows.value, dtype=np.float64)
            T.arg = np.zeros(rows.value, dtype=np.uint8)
            lib().orc_run_table(self.h, int(t), T.out.ctypes.data_as(C.POINTER(C.c_double)),
                                T.arg.ctypes.data_as(C.POINTER(C.c_ubyte)))
        return T

    def close(self):
        if self.h:
            lib().orc_run_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
