"""ctypes declarations of include/gpube.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgpube.so")

OK, EINVAL, ENOMEM, ETIMEDOUT, ECUDA, ENODEV, EAGAIN = 0, -22, -12, -110, -1000, -19, -11
INT32_SAT, FP32_LOG = 0, 1
ORDER_MINFILL, ORDER_BEST, ORDER_GIVEN, ORDER_NATURAL, ORDER_PSEUDOTREE = 0, 1, 2, 3, 4
IB_SEP_VARS, IB_JOINT_VARS, IB_LOG2_ENTRIES = 0, 1, 2
KIND_BE, KIND_MBE, KIND_DPOP, KIND_SUM, KIND_SUM_MBE = 0, 1, 2, 3, 4

i32p = C.POINTER(C.c_int32)
i64p = C.POINTER(C.c_int64)
u8p = C.POINTER(C.c_uint8)


class WcspDesc(C.Structure):
    _fields_ = [("n_vars", C.c_int32), ("dom", i32p), ("n_funcs", C.c_int32),
                ("scope_off", i32p), ("scope", i32p), ("tab_off", i64p), ("costs", C.c_void_p),
                ("cost_type", C.c_int32), ("top_k", C.c_int32)]


class SolveOpts(C.Structure):
    _fields_ = [("order_kind", C.c_int32), ("order", i32p), ("parent", i32p),
                ("ibound_mode", C.c_int32), ("batched", C.c_int32), ("use_graph", C.c_int32),
                ("block_threads", C.c_int32), ("rows_per_item", C.c_int32),
                ("lo_target", C.c_int32), ("stage_max_entries", C.c_int32),
                ("arena", C.c_void_p), ("arena_bytes", C.c_size_t), ("stream", C.c_void_p),
                ("autotune_cache", C.c_char_p), ("device", C.c_int32),
                ("evidence_vars", i32p), ("n_evidence_vars", C.c_int32), ("pipeline", C.c_int32),
                ("vector_rows", C.c_int32), ("argmin_tables", C.c_int32)]


class LaunchConfig(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("rows_per_item", C.c_int32), ("lo_target", C.c_int32),
                ("stage_max_entries", C.c_int32), ("pipeline", C.c_int32), ("launch_mode", C.c_int32),
                ("vector_rows", C.c_int32)]


class SolveResult(C.Structure):
    _fields_ = [("bound", C.c_double), ("cost", C.c_double), ("assignment", i32p),
                ("induced_width", C.c_int32), ("n_tasks", C.c_int32), ("n_levels", C.c_int32),
                ("n_launches", C.c_int32), ("util_entries", C.c_int64), ("alg_bytes", C.c_int64),
                ("plan_ms", C.c_double), ("util_ms", C.c_double), ("value_ms", C.c_double)]


class PlanInfo(C.Structure):
    _fields_ = [("n_vars", C.c_int32), ("n_tasks", C.c_int32), ("n_levels", C.c_int32),
                ("induced_width", C.c_int32), ("util_entries", C.c_int64),
                ("out_entries", C.c_int64), ("in_entries", C.c_int64), ("alg_bytes", C.c_int64),
                ("arena_bytes", C.c_size_t), ("peak_live_bytes", C.c_size_t),
                ("max_sep", C.c_int32), ("max_inputs", C.c_int32), ("n_argmin_tables", C.c_int32)]


class TaskInfo(C.Structure):
    _fields_ = [("var", C.c_int32), ("level", C.c_int32), ("n_sep", C.c_int32),
                ("n_inputs", C.c_int32), ("rows", C.c_int64), ("sep", i32p), ("inputs", i32p),
                ("lo_extent", C.c_int64), ("groups", C.c_int64), ("r0", C.c_int32), ("n_lo", C.c_int32),
                ("n_group", C.c_int32), ("n_uonly", C.c_int32), ("staged_bytes", C.c_int32),
                ("argmin", C.c_int32)]


# name -> (restype, argtypes)
SIGNATURES = {
    "wcsp_load": (C.c_int, [C.POINTER(WcspDesc), C.POINTER(C.c_void_p)]),
    "wcsp_free": (None, [C.c_void_p]),
    "wcsp_last_error": (C.c_char_p, []),
    "solve_opts_init": (None, [C.POINTER(SolveOpts)]),
    "be_solve": (C.c_int, [C.c_void_p, C.POINTER(SolveOpts), C.POINTER(SolveResult)]),
    "mbe_solve": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(SolveOpts), C.POINTER(SolveResult)]),
    "logz_solve": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(SolveOpts), C.POINTER(SolveResult)]),
    "util_condition": (C.c_int, [C.c_void_p, C.c_int32, i32p, i32p]),
    "dpop_util": (C.c_int, [C.c_void_p, i32p, C.POINTER(SolveOpts), C.POINTER(C.c_void_p)]),
    "value_propagate": (C.c_int, [C.c_void_p, i32p, C.POINTER(SolveResult)]),
    "util_state_free": (None, [C.c_void_p]),
    "util_plan": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, i32p, C.POINTER(SolveOpts),
                            C.POINTER(C.c_void_p)]),
    "util_plan_info": (C.c_int, [C.c_void_p, C.POINTER(PlanInfo)]),
    "util_task_info": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(TaskInfo)]),
    "util_order": (C.c_int, [C.c_void_p, i32p]),
    "util_bind": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "util_run": (C.c_int, [C.c_void_p]),
    "util_value_launch": (C.c_int, [C.c_void_p]),
    "util_sync": (C.c_int, [C.c_void_p]),
    "util_fetch_table": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, u8p]),
    "util_autotune": (C.c_int, [C.c_void_p, i32p, i32p]),
    "util_launch_config": (C.c_int, [C.c_void_p, C.POINTER(LaunchConfig)]),
    "util_last_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "util_bucket": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, i32p, C.c_int32, C.c_int32,
                              C.POINTER(C.c_void_p), i32p, i32p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "util_bucket_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, i32p, C.c_int32, C.c_int32,
                                      C.POINTER(C.c_void_p), i32p, i32p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "util_bucket_scratch_bytes": (C.c_int, [C.c_int32, i32p, C.c_int32, C.c_int32, i32p, i32p,
                                            C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "util_selftest_wait": (C.c_int, [C.c_uint64, C.c_void_p]),
    "util_selftest_dep_wait": (C.c_int, [C.c_uint64, C.c_void_p]),
    "srv_create": (C.c_int, [C.c_size_t, C.c_int32, C.c_void_p, C.c_size_t, C.c_void_p,
                             C.POINTER(C.c_void_p)]),
    "srv_submit": (C.c_int64, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, i32p,
                               C.POINTER(SolveOpts)]),
    "srv_step": (C.c_int, [C.c_void_p]),
    "srv_result": (C.c_int, [C.c_void_p, C.c_int64, i32p, C.POINTER(SolveResult)]),
    "srv_times": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                            C.POINTER(C.c_double)]),
    "srv_stats": (C.c_int, [C.c_void_p, i64p, i64p, i64p]),
    "srv_free": (None, [C.c_void_p]),
}

_lib = None


def load_library():
    """The CUDA library; raises when it has not been built (there is no
    fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with paper_1608_05288_gb300._build.build()")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
