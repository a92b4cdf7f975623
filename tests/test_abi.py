"""Host-side checks of the C ABI (no GPU): the library loads, exports every
declared entry point, validates problems, and plans exactly what the oracle
computes (orders, buckets, mini-bucket partitions, separators)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import synth
import paper_1608_05288_gb300 as gb
from paper_1608_05288_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1608_05288_gb300 import _build
    _build.build()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                                 src, flags=re.M):
                names.add(m.group(1))
    return names


def test_exports_every_declared_symbol():
    lib = C.CDLL(_abi.LIB_PATH)
    names = _declared()
    assert {"wcsp_load", "be_solve", "mbe_solve", "dpop_util", "value_propagate"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_abi.SIGNATURES) >= names


def test_load_rejects_malformed():
    inst = synth.paper_example()
    gb.WCSP(inst)  # fine
    bad = synth.paper_example()
    bad.scopes[0] = np.array([0, 0], dtype=np.int32)  # repeated variable
    with pytest.raises(gb.GpubeError) as e:
        gb.WCSP(bad)
    assert e.value.code == gb.EINVAL
    bad = synth.paper_example()
    bad.tables[1] = bad.tables[1][:3]  # wrong length
    with pytest.raises(gb.GpubeError):
        gb.WCSP(bad)
    bad = synth.paper_example()
    bad.tables[2] = bad.tables[2].copy()
    bad.tables[2][0] = -1  # negative cost
    with pytest.raises(gb.GpubeError):
        gb.WCSP(bad)
    bad = synth.paper_example()
    bad.dom = np.array([2, 2, 0, 2], dtype=np.int32)
    with pytest.raises(gb.GpubeError):
        gb.WCSP(bad)


def _lib_structure(st):
    return [{"var": int(t["var"]), "sep": [int(x) for x in t["sep"]],
             "inputs": sorted(int(x) for x in t["inputs"])} for t in st.tasks()]


def _orc_structure(run):
    return [{"var": int(t.var), "sep": [int(x) for x in t.sep],
             "inputs": sorted(int(x) for x in t.inputs)} for t in run.tasks]


def test_paper_example_plan(orc):
    inst = synth.paper_example()
    order = [3, 2, 1, 0]
    be = gb.UtilState(inst, "be", order="given", order_array=order)
    run = orc.eliminate(inst, np.array(order), "be")
    assert _lib_structure(be) == _orc_structure(run)
    assert be.info()["induced_width"] == 3
    mbe = gb.UtilState(inst, "mbe", 1, order="given", order_array=order, ibound_mode="sep")
    assert _lib_structure(mbe) == _orc_structure(orc.eliminate(inst, np.array(order), "sep", 1))


def test_mbe_partition_golden_plan():
    # the library's mini-bucket partition against the hand-derived partitions
    # of mixed-arity buckets (first fit by arity, unions on the bound accepted)
    import json
    with open(os.path.join(ROOT, "tests", "golden", "mbe_partition.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        dom = np.array(case["dom"], dtype=np.int32)
        scopes = [np.array(x, dtype=np.int32) for x in case["scopes"]]
        tables = [np.zeros(int(np.prod([dom[v] for v in x])), dtype=np.int64) for x in scopes]
        inst = synth.Instance(case["name"], dom, scopes, tables, "int", 1 << 30)
        st = gb.UtilState(inst, "mbe", case["z"], order="given", order_array=case["order"],
                          ibound_mode=case["mode"])
        got = [{"sep": t["sep"], "inputs": t["inputs"]} for t in _lib_structure(st) if t["var"] == 0]
        assert got == case["tasks_of_var0"], case["name"]


@pytest.mark.parametrize("seed", range(10))
def test_minfill_order_matches_oracle(orc, seed):
    inst = synth.random_small(seed, n=12, dmax=3, n_funcs=16, max_arity=3)
    st = gb.UtilState(inst, "be", order="minfill")
    o, w = orc.minfill(inst)
    assert list(st.order()) == list(o)
    assert st.info()["induced_width"] == orc.eliminate(inst, o, "be", tables=False).width


def test_config_orders_match_oracle(orc):
    for idx in (0, 1, 2, 3):
        inst = synth.config_instance(idx, 0)
        st = gb.UtilState(inst, "be" if idx < 2 else "mbe", 16, order="best" if idx == 1 else "minfill",
                          ibound_mode="log2")
        o, _ = orc.best_order(inst) if idx == 1 else orc.minfill(inst)
        assert list(st.order()) == list(o), idx


@pytest.mark.parametrize("mode", ["sep", "joint", "log2"])
@pytest.mark.parametrize("seed", range(6))
def test_mbe_partition_matches_oracle(orc, seed, mode):
    inst = synth.random_small(seed + 50, n=10, dmax=4, n_funcs=14, max_arity=3)
    o, _ = orc.minfill(inst)
    for z in (1, 2, 3, 4, 6):
        st = gb.UtilState(inst, "mbe", z, order="given", order_array=o, ibound_mode=mode)
        assert _lib_structure(st) == _orc_structure(orc.eliminate(inst, o, mode, z, tables=False))


def test_config2_partition_matches_oracle(orc):
    inst = synth.config_instance(2, 0)
    o, _ = orc.minfill(inst)
    st = gb.UtilState(inst, "mbe", 16, order="given", order_array=o, ibound_mode="log2")
    run = orc.eliminate(inst, o, "log2", 16, tables=False)
    assert _lib_structure(st) == _orc_structure(run)
    info = st.info()
    assert info["n_tasks"] == len(run.tasks)
    assert info["util_entries"] == sum(int(t.rows) * int(inst.dom[t.var]) for t in run.tasks)


@pytest.mark.parametrize("seed", range(4))
def test_dpop_plan_matches_oracle(orc, seed):
    inst = synth.dcop_random(seed, n_range=(15, 30), d_range=(2, 4))
    for parent in (None, inst.parent):
        st = gb.UtilState(inst, "dpop", parent=parent)
        par = orc.dfs_pseudotree(inst) if parent is None else parent
        o = orc.pseudotree_order(inst, par)
        assert list(st.order()) == list(o)
        assert _lib_structure(st) == _orc_structure(orc.eliminate(inst, o, "be", tables=False))


def test_dpop_rejects_invalid_pseudotree():
    inst = synth.paper_example()
    # a chain 0-1-2 with 3 hanging from 0: f(x2,x4) = (1,3) spans two branches
    parent = np.array([-1, 0, 1, 0], dtype=np.int32)
    with pytest.raises(gb.GpubeError) as e:
        gb.UtilState(inst, "dpop", parent=parent)
    assert e.value.code == gb.EINVAL
    cyc = np.array([1, 2, 0, -1], dtype=np.int32)
    with pytest.raises(gb.GpubeError):
        gb.UtilState(inst, "dpop", parent=cyc)


def test_plan_sizes_and_levels():
    inst = synth.config_instance(1, 0)
    st = gb.UtilState(inst, "be", order="best")
    info = st.info()
    assert info["induced_width"] == 12
    assert info["n_tasks"] == 144
    tasks = st.tasks()
    assert max(t["rows"] for t in tasks) == 4 ** 12
    # row-major elimination of a grid is a chain: one bucket per level
    assert info["n_levels"] == 144
    assert info["util_entries"] == sum(t["rows"] * 4 for t in tasks)
    assert info["alg_bytes"] == 4 * info["in_entries"] + 5 * info["out_entries"]
    assert info["arena_bytes"] >= 5 * info["out_entries"]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # without the built CUDA library there is no fallback: every call raises
    monkeypatch.setattr(_abi, "_lib", None)
    monkeypatch.setattr(_abi, "LIB_PATH", str(tmp_path / "libgpube.so"))
    with pytest.raises(RuntimeError):
        gb.WCSP(synth.paper_example())


@pytest.mark.parametrize("seed", range(4))
def test_sum_plans_match_oracle(orc, seed):
    # the sum-product kinds plan BE's buckets / Algorithm 2's mini-buckets
    inst = synth.random_small(seed + 70, n=10, dmax=4, n_funcs=14, max_arity=3, cost_type="real")
    o, _ = orc.minfill(inst)
    st = gb.UtilState(inst, "sum", order="given", order_array=o)
    assert _lib_structure(st) == _orc_structure(orc.eliminate(inst, o, "be", tables=False, semiring="sum"))
    for z in (1, 2, 4):
        st = gb.UtilState(inst, "sum_mbe", z, order="given", order_array=o, ibound_mode="joint")
        want = orc.eliminate(inst, o, "joint", z, tables=False, semiring="sum")
        assert _lib_structure(st) == _orc_structure(want)


def test_sum_counting_plan_of_integer_wcsp(orc):
    # counting an integer WCSP plans the same buckets and stores fp32 tables
    inst = synth.random_small(5, n=10, dmax=4, n_funcs=14, max_arity=3, p_top=0.3)
    be = gb.UtilState(inst, "be")
    sm = gb.UtilState(inst, "sum")
    assert _lib_structure(be) == _lib_structure(sm)
    # the sum-product kinds write no argmin tables: 4 bytes per output entry
    i_be, i_sm = be.info(), sm.info()
    assert i_sm["alg_bytes"] == i_be["alg_bytes"] - i_be["out_entries"]


@pytest.mark.parametrize("cost_type", ["int", "real"])
def test_argmin_tables_only_where_the_value_phase_reads_them(cost_type):
    # BE and DPOP look their assignment up in argmin tables (Algorithm 1,
    # Section 4.1); the value step of Algorithm 2 re-minimises over each
    # bucket's functions, so a mini-bucket plan leaves a task's table out
    # where the kernel has variants without it (fp32 costs, domains 2-4, at
    # most 7 inputs) unless asked for them; the sum-product writes none
    inst = synth.random_small(11, n=14, dmax=6, n_funcs=22, max_arity=3, cost_type=cost_type)
    states = {k: gb.UtilState(inst, k, 2) for k in ("be", "dpop", "sum", "mbe")}
    states["mbe_arg"] = gb.UtilState(inst, "mbe", 2, argmin_tables=True)
    info = {k: s.info() for k, s in states.items()}
    for k in ("be", "dpop", "mbe_arg"):
        assert info[k]["n_argmin_tables"] == info[k]["n_tasks"]
    assert info["sum"]["n_argmin_tables"] == 0
    tasks = states["mbe"].tasks()
    without = [t for t in tasks if cost_type == "real" and 2 <= inst.dom[t["var"]] <= 4 and len(t["inputs"]) <= 7]
    assert [not t["argmin"] for t in tasks] == [t in without for t in tasks]
    if cost_type == "real":
        assert without and len(without) < len(tasks)  # the instance has both kinds of task
    mb, mb_arg = info["mbe"], info["mbe_arg"]
    assert mb["n_argmin_tables"] == len(tasks) - len(without)
    assert mb["out_entries"] == mb_arg["out_entries"] and mb["in_entries"] == mb_arg["in_entries"]
    kept = sum(t["rows"] for t in tasks if t["argmin"])
    assert mb["alg_bytes"] == 4 * mb["in_entries"] + 4 * mb["out_entries"] + kept
    assert mb_arg["alg_bytes"] == 4 * mb_arg["in_entries"] + 5 * mb_arg["out_entries"]
    # a table left out takes no arena space
    assert mb["arena_bytes"] + sum(t["rows"] for t in without) <= mb_arg["arena_bytes"]


def test_evidence_plan_matches_oracle(orc):
    # evidence variables add one unary function each, after the problem's own
    inst = synth.random_small(11, n=10, dmax=4, n_funcs=14, max_arity=3)
    ev_vars = [7, 2, 9]
    o, _ = orc.minfill(inst)
    aug = synth.with_evidence(inst, {}, declared=ev_vars)
    for kind, mode, z in (("be", "be", 0), ("mbe", "sep", 2)):
        st = gb.UtilState(inst, kind, z, order="given", order_array=o, ibound_mode="sep", evidence_vars=ev_vars)
        assert _lib_structure(st) == _orc_structure(orc.eliminate(aug, o, mode, z, tables=False))


def test_condition_validates():
    inst = synth.random_small(12, n=6, dmax=3, n_funcs=8)
    st = gb.UtilState(inst, "be", evidence_vars=[1, 3])
    st.condition({1: 0, 3: None})            # before binding: kept for the upload
    with pytest.raises(gb.GpubeError):
        st.condition({2: 0})                 # not declared
    with pytest.raises(gb.GpubeError):
        st.condition({1: int(inst.dom[1])})  # outside the domain
    with pytest.raises(gb.GpubeError):
        gb.UtilState(inst, "be", evidence_vars=[1, 1])
    plain = gb.UtilState(inst, "be")
    with pytest.raises(gb.GpubeError):
        plain.condition({1: 0})


@pytest.mark.parametrize("seed", range(12))
def test_minfill_order_matches_oracle_larger_graphs(orc, seed):
    # the planner keeps fill counts incrementally; the order must equal the
    # oracle's plain greedy min-fill (ties: fewest neighbours, lowest id)
    kinds = [lambda s: synth.random_network_wcsp(40, 2, (0.05, 0.1, 0.25)[s % 3], seed=s),
             lambda s: synth.grid_wcsp(5 + s % 3, 6, 2, seed=s),
             lambda s: synth.scale_free_wcsp(50, 2, seed=s),
             lambda s: synth.er_wcsp(60, seed=s, n_tables=45, dmax=3)]
    inst = kinds[seed % 4](seed)
    o, w = orc.minfill(inst)
    w_lib = gb.WCSP(inst)
    try:
        st = gb.UtilState(w_lib, "be", order="minfill")
    except gb.GpubeError:
        pytest.skip("tables too large to plan")
    assert list(st.order()) == list(o)


def test_packed_arrays_load_the_same_problem():
    # WCSP from the flat wcsp_desc arrays (packed once) and from the instance
    # give the same plan, for integer and real costs
    for inst in (synth.config_instance(0, 1), synth.bayes_net_mpe(40, 2)):
        pk = gb.Packed(inst)
        a = gb.UtilState(gb.WCSP(inst), "be").info()
        for _ in range(2):  # the packed arrays are reusable
            b = gb.UtilState(gb.WCSP(pk), "be").info()
            assert a == b
