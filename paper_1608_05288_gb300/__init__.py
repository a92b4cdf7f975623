"""Python binding of the GB300 UTIL-table library (``libgpube.so``).

Thin marshalling over the C ABI of ``include/gpube.h``: every step of the
UTIL and VALUE phases runs in the library's CUDA kernels.  PyTorch is used
only for device memory (the arena) and the CUDA stream.  When the library is
missing, every call raises; nothing falls back to a CPU path.

Problems are any object with ``dom`` (int array), ``scopes`` (list of int
arrays), ``tables`` (list of arrays, row-major over the scope, first variable
slowest), ``cost_type`` ("int" for saturating WCSP costs, "real" for -log p)
and ``top_k``.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import _abi
from ._abi import (  # noqa: F401
    EAGAIN, ECUDA, EINVAL, ENODEV, ENOMEM, ETIMEDOUT, FP32_LOG, IB_JOINT_VARS, IB_LOG2_ENTRIES,
    IB_SEP_VARS, INT32_SAT, KIND_BE, KIND_DPOP, KIND_MBE, KIND_SUM, KIND_SUM_MBE, ORDER_BEST,
    ORDER_GIVEN, ORDER_MINFILL, ORDER_NATURAL, ORDER_PSEUDOTREE,
)

ORDERS = {"minfill": ORDER_MINFILL, "best": ORDER_BEST, "given": ORDER_GIVEN,
          "natural": ORDER_NATURAL, "pseudotree": ORDER_PSEUDOTREE}
IBOUND = {"sep": IB_SEP_VARS, "joint": IB_JOINT_VARS, "log2": IB_LOG2_ENTRIES}


class GpubeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gpube error {code}: {msg}")
        self.code = code


def lib():
    return _abi.load_library()


def _check(rc):
    if rc != 0:
        raise GpubeError(rc, (lib().wcsp_last_error() or b"").decode())
    return rc


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a, t=C.c_int32):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


class Packed:
    """A problem as the flat arrays of ``wcsp_desc`` (CSR scopes and tables):
    pack once, then load it any number of times without re-marshalling."""

    def __init__(self, inst):
        self.n = int(len(inst.dom))
        self.is_int = inst.cost_type == "int"
        self.dom = _i32(inst.dom)
        F = self.F = len(inst.scopes)
        self.scope_off = np.zeros(F + 1, dtype=np.int32)
        self.tab_off = np.zeros(F + 1, dtype=np.int64)
        np.cumsum(np.fromiter((len(s) for s in inst.scopes), dtype=np.int32, count=F), out=self.scope_off[1:])
        np.cumsum(np.fromiter((len(t) for t in inst.tables), dtype=np.int64, count=F), out=self.tab_off[1:])
        self.scope = _i32(np.concatenate(inst.scopes) if F and self.scope_off[-1] else np.zeros(1))
        if self.is_int:
            costs = np.concatenate(inst.tables) if F else np.zeros(1)
            self.costs = np.ascontiguousarray(np.minimum(costs, 2**31 - 1), dtype=np.int32)
        else:
            self.costs = np.ascontiguousarray(np.concatenate(inst.tables) if F else np.zeros(1), dtype=np.float32)
        self.top_k = int(min(inst.top_k, 2**31 - 1)) if self.is_int else 1


class WCSP:
    """A problem loaded into the library (``wcsp_load``), from an instance or
    from its ``Packed`` arrays."""

    def __init__(self, inst):
        L = lib()
        pk = inst if isinstance(inst, Packed) else Packed(inst)
        self.n = pk.n
        self.is_int = pk.is_int
        d = _abi.WcspDesc(pk.n, _ptr(pk.dom), pk.F, _ptr(pk.scope_off), _ptr(pk.scope),
                          pk.tab_off.ctypes.data_as(_abi.i64p), pk.costs.ctypes.data_as(C.c_void_p),
                          INT32_SAT if pk.is_int else FP32_LOG, pk.top_k)
        h = C.c_void_p()
        _check(L.wcsp_load(C.byref(d), C.byref(h)))
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _abi._lib is not None:
            _abi._lib.wcsp_free(h)
            self.h = None


LAUNCH_MODES = {"bucket": 0, "level": 1, "fused": 2}


def make_opts(order="minfill", order_array=None, parent=None, ibound_mode="sep", batched=True,
              use_graph=False, block_threads=0, rows_per_item=0, lo_target=0,
              stage_max_entries=0, arena=None, arena_bytes=0, stream=None,
              autotune_cache=None, device=0, evidence_vars=None, pipeline=True, vector_rows=False,
              argmin_tables=False):
    o = _abi.SolveOpts()
    lib().solve_opts_init(C.byref(o))
    o.order_kind = ORDERS[order] if isinstance(order, str) else int(order)
    keep = []
    if order_array is not None:
        a = _i32(order_array)
        keep.append(a)
        o.order = _ptr(a)
        if isinstance(order, str) and order == "minfill":
            o.order_kind = ORDER_GIVEN
    if parent is not None:
        p = _i32(parent)
        keep.append(p)
        o.parent = _ptr(p)
    o.ibound_mode = IBOUND[ibound_mode] if isinstance(ibound_mode, str) else int(ibound_mode)
    # launch mode: False / 0 = one launch per bucket, True / 1 = one per
    # elimination-tree level, "fused" / 2 = one launch over all levels
    o.batched = LAUNCH_MODES[batched] if isinstance(batched, str) else int(batched)
    o.use_graph = 1 if use_graph else 0
    o.block_threads = int(block_threads)
    o.rows_per_item = int(rows_per_item)
    o.lo_target = int(lo_target)
    o.stage_max_entries = int(stage_max_entries)
    o.arena = arena
    o.arena_bytes = int(arena_bytes)
    o.stream = stream
    if autotune_cache:
        b = autotune_cache.encode()
        keep.append(b)
        o.autotune_cache = b
    o.device = int(device)
    o.pipeline = 0 if pipeline else -1
    o.vector_rows = 1 if vector_rows else 0
    # argmin tables of mini-bucket plans (their value step reads none): written
    # only when asked for
    o.argmin_tables = 1 if argmin_tables else 0
    if evidence_vars is not None and len(evidence_vars):
        ev = _i32(evidence_vars)
        keep.append(ev)
        o.evidence_vars = _ptr(ev)
        o.n_evidence_vars = len(ev)
    o._keep = keep
    return o


def _torch():
    import torch  # device memory and streams only
    return torch


def current_stream(device=0):
    return _torch().cuda.current_stream(device).cuda_stream


@dataclass
class Result:
    bound: float
    cost: float
    assignment: np.ndarray
    induced_width: int = 0
    n_tasks: int = 0
    n_levels: int = 0
    n_launches: int = 0
    util_entries: int = 0
    alg_bytes: int = 0
    plan_ms: float = 0.0
    util_ms: float = 0.0
    value_ms: float = 0.0


def _result(r, sigma):
    return Result(r.bound, r.cost, sigma, r.induced_width, r.n_tasks, r.n_levels, r.n_launches,
                  r.util_entries, r.alg_bytes, r.plan_ms, r.util_ms, r.value_ms)


def _as_wcsp(p):
    return p if isinstance(p, WCSP) else WCSP(p)


def be_solve(problem, **opts):
    """Bucket Elimination (Algorithm 1) through ``be_solve``."""
    w = _as_wcsp(problem)
    o = make_opts(**opts)
    sigma = np.zeros(max(w.n, 1), dtype=np.int32)
    r = _abi.SolveResult()
    r.assignment = _ptr(sigma)
    _check(lib().be_solve(w.h, C.byref(o), C.byref(r)))
    return _result(r, sigma[: w.n])


def mbe_solve(problem, i_bound, **opts):
    """Mini-Bucket Elimination (Algorithm 2) through ``mbe_solve``."""
    w = _as_wcsp(problem)
    o = make_opts(**opts)
    sigma = np.zeros(max(w.n, 1), dtype=np.int32)
    r = _abi.SolveResult()
    r.assignment = _ptr(sigma)
    _check(lib().mbe_solve(w.h, int(i_bound), C.byref(o), C.byref(r)))
    return _result(r, sigma[: w.n])


def logz_solve(problem, i_bound=0, **opts):
    """Sum-product through ``logz_solve``: ``bound`` is -log Z (real costs:
    Z = sum of exp(-cost) over all assignments; integer WCSP: Z = number of
    assignments with no function at the top cost), or its mini-bucket lower
    bound when i_bound > 0.  No assignment; ``cost`` is NaN."""
    w = _as_wcsp(problem)
    o = make_opts(**opts)
    r = _abi.SolveResult()
    _check(lib().logz_solve(w.h, int(i_bound), C.byref(o), C.byref(r)))
    return _result(r, None)


KINDS = {"be": KIND_BE, "mbe": KIND_MBE, "dpop": KIND_DPOP, "sum": KIND_SUM, "sum_mbe": KIND_SUM_MBE}


class UtilState:
    """A planned (and, once bound, device-resident) UTIL phase."""

    def __init__(self, problem, kind="be", i_bound=0, parent=None, **opts):
        self.w = _as_wcsp(problem)
        k = KINDS[kind] if isinstance(kind, str) else kind
        self.kind = k
        if k != KIND_DPOP and parent is not None:
            opts.setdefault("parent", parent)  # the pseudo-tree of a GPUBE_ORDER_PSEUDOTREE order
            parent = None
        self.opts = make_opts(**opts)
        self.arena_tensor = None
        par = _i32(parent) if parent is not None else None
        self._par = par
        h = C.c_void_p()
        _check(lib().util_plan(self.w.h, k, int(i_bound), _ptr(par), C.byref(self.opts), C.byref(h)))
        self.h = h
        self.bound = False

    @classmethod
    def _wrap(cls, w, h):
        self = cls.__new__(cls)
        self.w, self.h, self.opts, self.arena_tensor, self.bound, self._par = w, h, None, None, True, None
        self.kind = KIND_DPOP
        return self

    def info(self):
        i = _abi.PlanInfo()
        _check(lib().util_plan_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in _abi.PlanInfo._fields_}

    def task(self, t):
        inf = self.info()
        sep = np.zeros(max(inf["n_vars"], 1), dtype=np.int32)
        ins = np.zeros(max(inf["max_inputs"], 1), dtype=np.int32)
        ti = _abi.TaskInfo()
        ti.sep = _ptr(sep)
        ti.inputs = _ptr(ins)
        _check(lib().util_task_info(self.h, int(t), C.byref(ti)))
        return {"var": ti.var, "level": ti.level, "rows": ti.rows, "sep": sep[: ti.n_sep].copy(),
                "inputs": ins[: ti.n_inputs].copy(), "lo_extent": ti.lo_extent, "groups": ti.groups,
                "r0": ti.r0, "n_lo": ti.n_lo, "n_group": ti.n_group, "n_uonly": ti.n_uonly,
                "staged_bytes": ti.staged_bytes, "argmin": bool(ti.argmin)}

    def tasks(self):
        return [self.task(t) for t in range(self.info()["n_tasks"])]

    def order(self):
        o = np.zeros(max(self.w.n, 1), dtype=np.int32)
        _check(lib().util_order(self.h, _ptr(o)))
        return o[: self.w.n]

    def bind(self, arena=None, stream=None, device=0):
        """Bind device memory: a torch uint8 tensor (allocated here when None)
        and the stream (torch's current stream when None)."""
        torch = _torch()
        need = self.info()["arena_bytes"]
        if arena is None:
            # headroom for the re-shaped layouts util_autotune tries (a smaller
            # lo extent enlarges the per-group offset tables)
            need += min(need // 8, 256 << 20) + (4 << 20)
            arena = torch.empty(max(need, 256), dtype=torch.uint8, device=f"cuda:{device}")
        self.arena_tensor = arena
        st = current_stream(device) if stream is None else stream
        self.stream = st
        _check(lib().util_bind(self.h, C.c_void_p(arena.data_ptr()), arena.numel(), C.c_void_p(st)))
        self.bound = True
        return self

    def run(self):
        _check(lib().util_run(self.h))
        return self

    def value_launch(self):
        _check(lib().util_value_launch(self.h))

    def sync(self):
        _check(lib().util_sync(self.h))

    def value(self):
        sigma = np.zeros(max(self.w.n, 1), dtype=np.int32)
        r = _abi.SolveResult()
        r.assignment = _ptr(sigma)
        _check(lib().value_propagate(self.h, _ptr(sigma), C.byref(r)))
        return _result(r, sigma[: self.w.n])

    def times(self):
        a, b = C.c_double(), C.c_double()
        _check(lib().util_last_times(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def fetch(self, t):
        rows = self.task(t)["rows"]
        # sum-product tables are fp32 -log weights whatever the problem's cost type
        fp = not self.w.is_int or self.kind in (KIND_SUM, KIND_SUM_MBE)
        cost = np.zeros(max(rows, 1), dtype=np.float32 if fp else np.int32)
        arg = np.zeros(max(rows, 1), dtype=np.uint8)
        _check(lib().util_fetch_table(self.h, int(t), cost.ctypes.data_as(C.c_void_p), _ptr(arg, C.c_uint8)))
        return cost[:rows], arg[:rows]

    def condition(self, evidence):
        """Clamp evidence variables for the next runs: {var: value}, value
        -1 (or None) frees the variable (``util_condition``)."""
        vs = _i32(list(evidence.keys()))
        xs = _i32([-1 if x is None else int(x) for x in evidence.values()])
        _check(lib().util_condition(self.h, len(vs), _ptr(vs), _ptr(xs)))

    def autotune(self):
        a, b = C.c_int32(), C.c_int32()
        _check(lib().util_autotune(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def launch_config(self):
        """The state's launch configuration (``util_launch_config``) as the
        keyword options that reproduce it in a solve."""
        c = _abi.LaunchConfig()
        _check(lib().util_launch_config(self.h, C.byref(c)))
        return {"block_threads": c.block_threads, "rows_per_item": c.rows_per_item, "lo_target": c.lo_target,
                "stage_max_entries": c.stage_max_entries if c.stage_max_entries > 0 else -1,
                "pipeline": bool(c.pipeline), "batched": c.launch_mode, "vector_rows": bool(c.vector_rows)}

    def free(self):
        if getattr(self, "h", None) and _abi._lib is not None:
            _abi._lib.util_state_free(self.h)
        self.h = None

    def __del__(self):
        self.free()


def dpop_util(problem, parent=None, **opts):
    """DPOP UTIL phase (``dpop_util``); returns a bound, run UtilState."""
    w = _as_wcsp(problem)
    o = make_opts(**opts)
    par = _i32(parent) if parent is not None else None
    h = C.c_void_p()
    _check(lib().dpop_util(w.h, _ptr(par), C.byref(o), C.byref(h)))
    return UtilState._wrap(w, h)


def util_bucket(sep_dom, d, tables, positions, out, arg, cost_type="int", top_k=(1 << 30),
                stream=None):
    """One bucket on the GPU (``util_bucket``): tables are torch CUDA tensors
    row-major over (sep positions ascending, eliminated variable)."""
    sd = _i32(sep_dom if len(sep_dom) else [1])
    ptrs = (C.c_void_p * len(tables))(*[t.data_ptr() for t in tables])
    off = np.zeros(len(positions) + 1, dtype=np.int32)
    for i, p in enumerate(positions):
        off[i + 1] = off[i] + len(p)
    pos = _i32([x for p in positions for x in p] or [0])
    st = current_stream() if stream is None else stream
    _check(lib().util_bucket(INT32_SAT if cost_type == "int" else FP32_LOG, int(top_k), len(sep_dom),
                             _ptr(sd), int(d), len(tables), ptrs, _ptr(off), _ptr(pos),
                             C.c_void_p(out.data_ptr()), C.c_void_p(arg.data_ptr()), C.c_void_p(st)))


def util_bucket_noalloc(sep_dom, d, tables, positions, out, arg, cost_type="int", top_k=(1 << 30),
                        stream=None):
    """util_bucket for callers that cannot allocate device memory: the scratch
    is a fixed array inside the library (``util_bucket_noalloc``).  tables,
    out and arg are torch CUDA tensors.  The first call on a device looks up
    the array's device address; calls that may overlap on the GPU must be
    serialised by the caller."""
    sd = _i32(sep_dom if len(sep_dom) else [1])
    ptrs = (C.c_void_p * len(tables))(*[t.data_ptr() for t in tables])
    off = np.zeros(len(positions) + 1, dtype=np.int32)
    for i, p in enumerate(positions):
        off[i + 1] = off[i] + len(p)
    pos = _i32([x for p in positions for x in p] or [0])
    st = (current_stream() if stream is None else stream)
    _check(lib().util_bucket_noalloc(INT32_SAT if cost_type == "int" else FP32_LOG, int(top_k), len(sep_dom),
                                     _ptr(sd), int(d), len(tables), ptrs, _ptr(off), _ptr(pos),
                                     C.c_void_p(out.data_ptr()), C.c_void_p(arg.data_ptr()), C.c_void_p(st)))


def util_bucket_scratch_bytes(sep_dom, d, positions):
    """Scratch bytes the single-bucket calls need for this bucket shape, and
    the size of util_bucket_noalloc's fixed scratch (``util_bucket_scratch_bytes``,
    host only: no GPU needed, nothing launched)."""
    sd = _i32(sep_dom if len(sep_dom) else [1])
    off = np.zeros(len(positions) + 1, dtype=np.int32)
    for i, p in enumerate(positions):
        off[i + 1] = off[i] + len(p)
    pos = _i32([x for p in positions for x in p] or [0])
    need, limit = C.c_size_t(), C.c_size_t()
    _check(lib().util_bucket_scratch_bytes(len(sep_dom), _ptr(sd), int(d), len(positions), _ptr(off), _ptr(pos),
                                           C.byref(need), C.byref(limit)))
    return int(need.value), int(limit.value)


class Server:
    """Continuous-batching server (``srv_*``)."""

    def __init__(self, budget_bytes, max_slots=64, arena=None, stream=None, device=0):
        torch = _torch()
        if arena is None:
            arena = torch.empty(int(budget_bytes), dtype=torch.uint8, device=f"cuda:{device}")
        self.arena = arena
        st = current_stream(device) if stream is None else stream
        h = C.c_void_p()
        _check(lib().srv_create(int(budget_bytes), int(max_slots), C.c_void_p(arena.data_ptr()),
                                arena.numel(), C.c_void_p(st), C.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, problem, kind="dpop", i_bound=0, parent=None, **opts):
        w = _as_wcsp(problem)
        o = make_opts(**opts)
        par = _i32(parent) if parent is not None else None
        k = KINDS[kind]
        rid = lib().srv_submit(self.h, w.h, k, int(i_bound), _ptr(par), C.byref(o))
        if rid < 0:
            _check(int(rid))
        self._keep[rid] = w.n  # the server copied the problem and its options
        return int(rid)

    def step(self):
        rc = lib().srv_step(self.h)
        if rc < 0:
            _check(rc)
        return rc

    def result(self, rid):
        n = self._keep[rid]
        sigma = np.zeros(max(n, 1), dtype=np.int32)
        r = _abi.SolveResult()
        rc = lib().srv_result(self.h, int(rid), _ptr(sigma), C.byref(r))
        if rc == EAGAIN:
            return None
        _check(rc)
        return _result(r, sigma[:n])

    def times(self, rid):
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        lib().srv_times(self.h, int(rid), C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    def stats(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().srv_stats(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return {"launches": a.value, "peak_bytes": b.value, "max_inflight": c.value}

    def close(self):
        if getattr(self, "h", None) and _abi._lib is not None:
            _abi._lib.srv_free(self.h)
        self.h = None

    def __del__(self):
        self.close()
