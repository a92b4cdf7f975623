"""CUDA path vs the CPU oracle, through the C ABI (needs a GPU).

Integer WCSPs: every bucket function, argmin table, the bound, the
assignment and its cost are compared bit for bit (Theorem 1: the GPU tables
are the sequential algorithm's tables).  Real (-log p) problems: within
|delta| <= 1e-4 (1 + |value|), the assignment re-evaluated in fp64 by the
oracle within the same bound.
"""
import numpy as np
import pytest

import synth
import paper_1608_05288_gb300 as gb
from gpu_util import bucket_sums_at, check_tables, fp_close, run_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1608_05288_gb300 import _build
    _build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


LAUNCH_SHAPES = [
    dict(),                                                # defaults, batched
    dict(batched=False),                                   # one launch per bucket
    dict(use_graph=True),                                  # CUDA graph of the level sequence
    dict(block_threads=32, rows_per_item=1, lo_target=8),  # many tiny items, ragged tails
    dict(block_threads=64, rows_per_item=3, lo_target=5, stage_max_entries=-1),
    dict(block_threads=512, rows_per_item=64, stage_max_entries=4),
    dict(batched="fused"),                                 # one launch over all levels
    dict(batched="fused", use_graph=True, block_threads=32, rows_per_item=1, lo_target=8),
    dict(batched="fused", block_threads=128, rows_per_item=3, lo_target=5, stage_max_entries=4),
    dict(vector_rows=True),                                # four consecutive rows per thread
    dict(vector_rows=True, block_threads=32, rows_per_item=2, lo_target=8, stage_max_entries=-1),
]


def test_paper_example(orc):
    inst = synth.paper_example()
    order = np.array([3, 2, 1, 0])
    for kind, mode, z in (("be", "be", 0), ("mbe", "sep", 1)):
        st, res = run_state(inst, kind, z, order="given", order_array=order, ibound_mode="sep", argmin_tables=True)
        run = orc.eliminate(inst, order, mode, z)
        check_tables(inst, st, run)
        assert res.bound == run.bound and res.cost == run.cost
        assert list(res.assignment) == list(run.sigma)


def test_mbe_value_golden():
    # the hand-worked MBE example: every mini-bucket's functions enter the
    # value step of their bucket (the first or last alone picks another value)
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "mbe_value_example.json")) as f:
        g = json.load(f)
    dom = np.array(g["dom"], dtype=np.int32)
    inst = synth.Instance("mbe_value", dom, [np.array(x, dtype=np.int32) for x in g["scopes"]],
                          [np.array(t, dtype=np.int64) for t in g["tables"]], "int", 1 << 30)
    for shape, keep in ((s, k) for s in LAUNCH_SHAPES[:3] for k in (True, False)):
        st, res = run_state(inst, "mbe", g["z"], order="given", order_array=g["order"], ibound_mode=g["mode"],
                            argmin_tables=keep, **shape)
        for t, T in enumerate(g["tasks"]):
            cost, arg = st.fetch(t)
            assert [int(x) for x in cost] == T["out"], t
            assert st.task(t)["argmin"]  # integer costs: every task writes its table
            assert [int(x) for x in arg] == T["arg"], t
        assert res.bound == g["bound"] and res.cost == g["cost"]
        assert list(res.assignment) == g["sigma"]
        st.free()


@pytest.mark.parametrize("shape", range(len(LAUNCH_SHAPES)))
@pytest.mark.parametrize("seed", range(6))
def test_random_be_all_launch_shapes(orc, seed, shape):
    inst = synth.random_small(seed, n=9, dmax=6, n_funcs=14, max_arity=4)
    o, _ = orc.minfill(inst)
    run = orc.eliminate(inst, o, "be")
    st, res = run_state(inst, "be", order="given", order_array=o, **LAUNCH_SHAPES[shape])
    check_tables(inst, st, run)
    assert res.bound == run.bound == orc.bruteforce(inst)[0]
    assert res.cost == run.cost and list(res.assignment) == list(run.sigma)


@pytest.mark.parametrize("dom", [(1, 3), (2, 2), (3, 3), (5, 5), (7, 8), (9, 10), (9, 12), (16, 16), (2, 8)])
@pytest.mark.parametrize("cost_type", ["int", "real"])
def test_domain_classes(orc, dom, cost_type):
    # every templated domain size (2..10, 16), the generic loop (1, 11, 12)
    inst = synth.random_small(17 + dom[0], n=7, dmin=dom[0], dmax=dom[1], n_funcs=10, max_arity=3,
                              cost_type=cost_type)
    o, _ = orc.minfill(inst)
    run = orc.eliminate(inst, o, "be")
    st, res = run_state(inst, "be", order="given", order_array=o, block_threads=64, lo_target=16)
    check_tables(inst, st, run, exact=(cost_type == "int"))
    if cost_type == "int":
        assert res.bound == run.bound and list(res.assignment) == list(run.sigma)
    else:
        assert fp_close(res.bound, run.bound)
        assert fp_close(orc.evaluate(inst, res.assignment), res.cost)


@pytest.mark.parametrize("cost_type", ["int", "real"])
@pytest.mark.parametrize("d", [2, 3, 5])
def test_hub_bucket_many_inputs(orc, cost_type, d):
    # a hub with ten binary tables to leaves that form a chain, the hub
    # eliminated first: its bucket has ten inputs, three on the lo digits,
    # six group inputs and one on the fastest hi digit (the many-input
    # variant that keeps their pointers in registers)
    rng = np.random.default_rng(d)
    n = 11
    dom = np.full(n, d, dtype=np.int32)
    scopes = [np.array([0, v], np.int32) for v in range(1, n)] + [np.array([v, v + 1], np.int32) for v in range(1, n - 1)]
    tables = []
    for sc in scopes:
        size = d * d
        tables.append(rng.integers(0, 500, size=size).astype(np.int64) if cost_type == "int"
                      else -np.log(rng.uniform(0.01, 1.0, size=size)))
    inst = synth.Instance("hub", dom, scopes, tables, cost_type, 1 << 30)
    order = np.arange(n)
    for shape in (dict(lo_target=d * d * d, block_threads=32, rows_per_item=4), dict(lo_target=d * d, batched="fused")):
        st, res = run_state(inst, "be", order="given", order_array=order, **shape)
        t0 = st.task(0)
        assert len(t0["inputs"]) == 10 and t0["n_group"] - t0["n_lo"] <= 8 and 10 - t0["n_group"] <= 2
        run = orc.eliminate(inst, order, "be")
        check_tables(inst, st, run, exact=(cost_type == "int"))
        if cost_type == "int":
            assert res.bound == run.bound and list(res.assignment) == list(run.sigma)
        else:
            assert fp_close(res.bound, run.bound)
        st.free()


@pytest.mark.parametrize("nf", [5, 9, 20])
def test_many_inputs(orc, nf):
    # buckets of more than 4 and more than 8 functions (register / generic paths)
    rng = np.random.default_rng(nf)
    n = 6
    dom = np.array([3, 4, 2, 4, 3, 4], dtype=np.int32)
    scopes, tables = [], []
    for j in range(nf):
        s = np.array(sorted(rng.choice(n, size=2, replace=False)), dtype=np.int32)
        scopes.append(s)
        tables.append(rng.integers(0, 30, size=int(dom[s[0]] * dom[s[1]])))
    inst = synth.Instance("many", dom, scopes, tables, "int", 1 << 30)
    o = np.arange(n)
    run = orc.eliminate(inst, o, "be")
    st, res = run_state(inst, "be", order="given", order_array=o)
    check_tables(inst, st, run)
    assert res.bound == run.bound


@pytest.mark.parametrize("keep", [False, True])
@pytest.mark.parametrize("mode", ["sep", "joint", "log2"])
def test_random_mbe(orc, mode, keep):
    for seed in range(4):
        inst = synth.random_small(seed + 300, n=11, dmax=4, n_funcs=18, max_arity=3)
        o, _ = orc.minfill(inst)
        for z in (1, 2, 4):
            run = orc.eliminate(inst, o, mode, z)
            st, res = run_state(inst, "mbe", z, order="given", order_array=o, ibound_mode=mode, argmin_tables=keep)
            check_tables(inst, st, run)
            assert res.bound == run.bound and res.cost == run.cost
            assert list(res.assignment) == list(run.sigma)


@pytest.mark.parametrize("cost_type", ["int", "real"])
def test_mbe_without_argmin_tables(orc, cost_type):
    # mini-bucket plans write no argmin tables by default (their value step
    # re-minimises over each bucket's functions): the same bucket functions,
    # bound and assignment as with the tables, in every launch form
    for seed in range(3):
        inst = synth.random_small(seed + 510, n=12, dmax=3, n_funcs=20, max_arity=3, cost_type=cost_type)
        o, _ = orc.minfill(inst)
        for z, mode in ((2, "sep"), (3, "joint"), (5, "log2")):
            for shape in (dict(), dict(batched=False), dict(batched="fused", use_graph=True),
                          dict(vector_rows=True), dict(block_threads=32, rows_per_item=3, lo_target=4)):
                a, ra = run_state(inst, "mbe", z, order="given", order_array=o, ibound_mode=mode, **shape)
                b, rb = run_state(inst, "mbe", z, order="given", order_array=o, ibound_mode=mode,
                                  argmin_tables=True, **shape)
                assert b.info()["n_argmin_tables"] == len(b.tasks())
                ta = a.tasks()
                for t in range(len(ta)):
                    ca, aa = a.fetch(t)
                    cb, ab = b.fetch(t)
                    assert np.array_equal(ca, cb), (seed, z, t)
                    assert np.array_equal(aa, ab) if ta[t]["argmin"] else not np.any(aa), (seed, z, t)
                if cost_type == "real":
                    assert not all(t["argmin"] for t in ta)  # some tasks leave the table out
                assert ra.bound == rb.bound and list(ra.assignment) == list(rb.assignment)
                assert ra.cost == rb.cost or (np.isnan(ra.cost) and np.isnan(rb.cost))
                a.free()
                b.free()


def test_saturation_and_infeasible(orc):
    # every joint row reaches the top cost: saturated tables, argmin 0
    inst = synth.random_small(5, n=6, dmax=3, n_funcs=10, max_arity=3, p_top=0.9, top_k=50, hi=40)
    o, _ = orc.minfill(inst)
    run = orc.eliminate(inst, o, "be")
    st, res = run_state(inst, "be", order="given", order_array=o)
    check_tables(inst, st, run)
    assert res.bound == run.bound


def test_degenerate_problems(orc):
    # no variables, only constants, an unconstrained variable, a single variable
    empty = synth.Instance("empty", np.zeros(0, np.int32), [], [], "int", 1 << 30)
    res = gb.be_solve(empty)
    assert res.bound == 0 and res.cost == 0
    consts = synth.Instance("c", np.array([3], np.int32), [np.zeros(0, np.int32)] * 2,
                            [np.array([4]), np.array([5])], "int", 1 << 30)
    res = gb.be_solve(consts)
    assert res.bound == 9 and res.cost == 9 and list(res.assignment) == [0]
    one = synth.Instance("one", np.array([5], np.int32), [np.array([0], np.int32)],
                         [np.array([7, 3, 9, 3, 4])], "int", 1 << 30)
    res = gb.be_solve(one)
    assert res.bound == 3 and list(res.assignment) == [1]


def test_components(orc):
    a = synth.random_small(41, n=6, dmax=4, n_funcs=8, with_constant=False)
    b = synth.random_small(42, n=5, dmax=4, n_funcs=7, with_constant=False)
    a.top_k = b.top_k = 10**6
    u = synth.disjoint_union(a, b)
    ra, rb, ru = gb.be_solve(a), gb.be_solve(b), gb.be_solve(u)
    assert ru.bound == ra.bound + rb.bound
    assert ru.bound == orc.eliminate(u, orc.minfill(u)[0], "be").bound


def test_config0_grid(orc):
    for seed in range(3):
        inst = synth.config_instance(0, seed)
        o, w = orc.minfill(inst)
        run = orc.eliminate(inst, o, "be")
        for shape in (dict(), dict(batched=False), dict(use_graph=True), dict(batched="fused")):
            st, res = run_state(inst, "be", **shape)
            check_tables(inst, st, run)
            assert res.bound == run.bound == res.cost
            assert list(res.assignment) == list(run.sigma)
            assert res.induced_width == w == 4


def test_config2_mbe_full(orc):
    inst = synth.config_instance(2, 0)
    o, _ = orc.minfill(inst)
    run = orc.eliminate(inst, o, "log2", 16)
    for shape in (dict(use_graph=True, argmin_tables=True), dict(batched=False), dict(batched="fused", use_graph=True),
                  dict(vector_rows=True, use_graph=True, argmin_tables=True)):
        st, res = run_state(inst, "mbe", 16, ibound_mode="log2", **shape)
        check_tables(inst, st, run)
        assert res.bound == run.bound and res.cost == run.cost
        assert list(res.assignment) == list(run.sigma)


def test_config3_mpe_mbe_and_exact_prefix(orc):
    inst = synth.config_instance(3, 0)
    o, _ = orc.minfill(inst)
    orc.set_threads(orc.max_threads())
    try:
        run = orc.eliminate(inst, o, "sep", 20)
    finally:
        orc.set_threads(1)
    for shape in (dict(use_graph=True), dict(batched="fused", use_graph=True, vector_rows=True, argmin_tables=True)):
        st, res = run_state(inst, "mbe", 20, ibound_mode="sep", **shape)
        check_tables(inst, st, run, exact=False)
        assert fp_close(res.bound, run.bound)
        # the GPU's own assignment, re-evaluated in fp64 by the oracle
        assert fp_close(res.cost, orc.evaluate(inst, res.assignment))
        assert res.bound <= orc.evaluate(inst, res.assignment) + 1e-4 * (1 + abs(res.bound))
        st.free()
    pre = synth.bn_prefix(inst, 60)
    po, _ = orc.minfill(pre)
    prun = orc.eliminate(pre, po, "be")
    st, res = run_state(pre, "be")
    check_tables(pre, st, prun, exact=False)
    assert fp_close(res.bound, prun.bound)
    assert fp_close(orc.evaluate(pre, res.assignment), prun.bound)


def test_real_small_bruteforce(orc):
    for seed in range(6):
        inst = synth.random_small(seed + 900, n=7, dmax=4, n_funcs=10, cost_type="real")
        best, _ = orc.bruteforce(inst)
        res = gb.be_solve(inst)
        assert fp_close(res.bound, best)
        assert fp_close(orc.evaluate(inst, res.assignment), best)


@pytest.mark.parametrize("seed", range(3))
def test_dpop_util_value(orc, seed):
    inst = synth.dcop_random(seed, n_range=(20, 40), d_range=(3, 5), sep_cap=4)
    st = gb.dpop_util(inst, inst.parent)
    res = st.value()
    o = orc.pseudotree_order(inst, inst.parent)
    run = orc.eliminate(inst, o, "be")
    check_tables(inst, st, run)
    assert res.bound == run.bound == res.cost
    assert list(res.assignment) == list(run.sigma)
    st.free()
    # the library's own DFS pseudo-tree
    st = gb.dpop_util(inst)
    res = st.value()
    run = orc.eliminate(inst, orc.pseudotree_order(inst, orc.dfs_pseudotree(inst)), "be")
    check_tables(inst, st, run)
    assert res.bound == run.bound
    st.free()


def test_adpop_mbe_on_pseudotree_order(orc):
    inst = synth.dcop_random(7, n_range=(25, 35), d_range=(3, 4), sep_cap=5)
    o = orc.pseudotree_order(inst, inst.parent)
    run = orc.eliminate(inst, o, "sep", 2)
    st, res = run_state(inst, "mbe", 2, order="pseudotree", parent=inst.parent, ibound_mode="sep")
    check_tables(inst, st, run)
    assert res.bound == run.bound and res.cost == run.cost


def test_rerun_is_idempotent(orc):
    inst = synth.config_instance(0, 1)
    st = gb.UtilState(inst, "be", use_graph=True)
    st.bind()
    outs = []
    for _ in range(3):
        st.run()
        res = st.value()
        outs.append((res.bound, tuple(res.assignment), tuple(st.fetch(len(st.tasks()) - 2)[0])))
    assert outs[0] == outs[1] == outs[2]


def test_autotune_keeps_parity(orc, tmp_path):
    inst = synth.config_instance(2, 1)
    o, _ = orc.minfill(inst)
    run = orc.eliminate(inst, o, "log2", 12)
    st = gb.UtilState(inst, "mbe", 12, ibound_mode="log2", use_graph=True,
                      autotune_cache=str(tmp_path / "tune.txt"))
    st.bind()
    th, rp = st.autotune()
    assert th in (128, 256, 512) and rp > 0
    cfg = st.launch_config()
    assert cfg["block_threads"] == th and cfg["rows_per_item"] == rp
    assert cfg["lo_target"] in (128, 256, 512, 1024, 2048) and cfg["batched"] in (1, 2)
    st.run()
    res = st.value()
    check_tables(inst, st, run)
    assert res.bound == run.bound


def test_autotune_cache_reshapes_bound_state(orc, tmp_path):
    # configurations read back from the tuning cache are applied to a bound
    # state: a new lo extent target and staging limit re-shape the tasks in
    # place (the staged tables change), and the tables stay exact
    inst = synth.config_instance(2, 1)
    o, _ = orc.minfill(inst)
    run = orc.eliminate(inst, o, "log2", 12)
    first = tmp_path / "first.txt"
    st = gb.UtilState(inst, "mbe", 12, ibound_mode="log2", use_graph=True, autotune_cache=str(first))
    st.bind()
    st.autotune()
    key = first.read_text().split()[0]
    st.free()
    for cfg, staged in (((256, 32, 256, 0, 0, 2, 1), False), ((512, 64, 2048, 4096, 1, 1, 0), True),
                        ((128, 16, 128, 1024, 1, 2, 1), True)):
        cache = tmp_path / f"crafted_{cfg[2]}_{cfg[3]}.txt"
        cache.write_text(key + " " + " ".join(str(x) for x in cfg) + " 1.0\n")
        st = gb.UtilState(inst, "mbe", 12, ibound_mode="log2", use_graph=True, autotune_cache=str(cache))
        st.bind()
        assert any(t["staged_bytes"] for t in st.tasks())  # the default limit stages tables
        st.autotune()
        got = st.launch_config()
        assert (got["block_threads"], got["rows_per_item"], got["lo_target"], int(got["pipeline"]),
                got["batched"], int(got["vector_rows"])) == (cfg[0], cfg[1], cfg[2], cfg[4], cfg[5], cfg[6])
        assert any(t["staged_bytes"] for t in st.tasks()) == staged
        for _ in range(2):
            st.run()
        res = st.value()
        check_tables(inst, st, run)
        assert res.bound == run.bound and res.cost == run.cost
        st.free()


@pytest.mark.parametrize("seed", range(8))
def test_util_bucket_entry(orc, seed):
    import torch
    rng = np.random.default_rng(seed)
    m = int(rng.integers(0, 6))
    sep_dom = [int(x) for x in rng.integers(1, 6, size=m)]
    d = int(rng.integers(1, 9))
    is_int = seed % 2 == 0
    tables, positions, dev = [], [], []
    for _ in range(int(rng.integers(1, 6))):
        pos = sorted(int(x) for x in rng.choice(m, size=int(rng.integers(0, m + 1)), replace=False)) if m else []
        size = int(np.prod([sep_dom[p] for p in pos])) * d if pos else d
        if is_int:
            t = rng.integers(0, 1000, size=size).astype(np.int32)
        else:
            t = (-np.log(rng.uniform(0.01, 1, size=size))).astype(np.float32)
        tables.append(t.astype(np.float64))
        positions.append(pos)
        dev.append(torch.from_numpy(t).cuda())
    rows = int(np.prod(sep_dom)) if m else 1
    out = torch.zeros(rows, dtype=torch.int32 if is_int else torch.float32, device="cuda")
    arg = torch.zeros(rows, dtype=torch.uint8, device="cuda")
    gb.util_bucket(sep_dom, d, dev, positions, out, arg, "int" if is_int else "real", 1 << 30)
    torch.cuda.synchronize()
    want, warg = orc.util_bucket(sep_dom, d, tables, positions, is_int, 1 << 30)
    if is_int:
        assert np.array_equal(out.cpu().numpy().astype(np.float64), want)
        assert np.array_equal(arg.cpu().numpy(), warg)
    else:
        assert fp_close(out.cpu().numpy(), want)
        # the chosen value attains the minimum: the bucket sum at it, in fp64
        dom = sep_dom + [d]
        a = arg.cpu().numpy()
        assert np.all(a < d)
        s = bucket_sums_at(dom, m, list(range(m)), np.arange(rows), a,
                           [(p + [m], t) for p, t in zip(positions, tables)])
        assert fp_close(s, want)


@pytest.mark.parametrize("d", [32, 40, 100, 255])
def test_wide_domains_warp_shuffle(orc, d):
    # eliminated domains of 32 values and more: a warp per row, shuffle argmin
    for cost_type in ("int", "real"):
        inst = synth.random_small(d, n=4, dmin=d, dmax=d, n_funcs=6, max_arity=2, cost_type=cost_type)
        o, _ = orc.minfill(inst)
        run = orc.eliminate(inst, o, "be")
        for shape in (dict(), dict(block_threads=64, lo_target=8, rows_per_item=1)):
            st, res = run_state(inst, "be", order="given", order_array=o, **shape)
            check_tables(inst, st, run, exact=(cost_type == "int"))
            if cost_type == "int":
                assert res.bound == run.bound and list(res.assignment) == list(run.sigma)
            else:
                assert fp_close(res.bound, run.bound)


@pytest.mark.parametrize("d", [32, 100, 200])
def test_wide_domains_ties_fp32(orc, d):
    # fp32 costs on a few integer levels (sums exact in fp32 and fp64, many
    # ties per row, some +inf): the warp-min path must give the oracle's
    # minima and first argmins exactly
    rng = np.random.default_rng(d)
    dom = np.full(4, d, np.int32)
    scopes = [np.array(s, np.int32) for s in ([0, 1], [1, 2], [2, 3], [0, 3], [1], [3, 1])]
    tables = []
    for s in scopes:
        t = rng.integers(0, 4, size=int(np.prod(dom[s]))).astype(np.float64)
        t[rng.random(t.size) < 0.05] = np.inf
        tables.append(t)
    inst = synth.Instance(f"ties{d}", dom, scopes, tables, "real", 1 << 30)
    o, _ = orc.minfill(inst)
    run = orc.eliminate(inst, o, "be")
    st, res = run_state(inst, "be", order="given", order_array=o)
    for t, T in enumerate(run.tasks):
        cost, arg = st.fetch(t)
        assert np.array_equal(cost.astype(np.float64), T.out), f"task {t} costs"
        assert np.array_equal(arg, T.arg), f"task {t} argmin"
    assert res.bound == run.bound and list(res.assignment) == list(run.sigma)


def test_paper_random_network_d100(orc):
    # the shape of the paper's random networks with d = 100 (Section 8.1, p2 = 0.5)
    inst = synth.random_network_wcsp(6, 100, 0.3, seed=3)
    o, _ = orc.minfill(inst)
    run = orc.eliminate(inst, o, "be")
    st, res = run_state(inst, "be", order="given", order_array=o)
    check_tables(inst, st, run)
    assert res.bound == run.bound == res.cost


@pytest.mark.parametrize("hi,top_k", [(1000, 1 << 30), (1000, 20000), (1000, 9000), (1 << 26, (1 << 31) - 1)])
@pytest.mark.parametrize("d", [2, 3, 4])
def test_grid_rows_below_and_at_the_top_cost(orc, d, hi, top_k):
    # the pipelined grid rows take packed (sum << 2 | l) keys when every sum
    # stays below the top cost and 2^30, and the saturating rows otherwise
    # (sums reaching k, or sums above 2^30 with k = 2^31 - 1): both against
    # the oracle, bit for bit
    inst = synth.grid_wcsp(5, 8, d, seed=d, lo=0, hi=hi, unary=False, top_k=top_k)
    o = np.arange(inst.n, dtype=np.int32)
    run = orc.eliminate(inst, o, "be")
    for kw in (dict(), dict(use_graph=True, block_threads=128, rows_per_item=16)):
        st, res = run_state(inst, "be", order="natural", **kw)
        check_tables(inst, st, run)
        assert res.bound == run.bound and list(res.assignment) == list(run.sigma)


@pytest.mark.parametrize("seed", range(8))
def test_chain_value_phase(orc, seed):
    # band-structured problems in the natural order give one variable per
    # VALUE level: the one-warp path with early candidate loads; domains
    # 1..5 (two preceding domains give at most 25 candidates)
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 60))
    dom = rng.integers(1, 6, size=n).astype(np.int32)
    scopes, tables = [], []
    for v in range(n):
        for k in range(1, int(rng.integers(1, 4)) + 1):
            if v + k < n:
                s = np.array([v, v + k], dtype=np.int32)
                scopes.append(s)
                tables.append(rng.integers(0, 50, size=int(dom[v] * dom[v + k])).astype(np.int64))
    inst = synth.Instance(f"band{seed}", dom, scopes, tables, "int", 1 << 30)
    o = np.arange(n, dtype=np.int32)
    run = orc.eliminate(inst, o, "be")
    for kw in (dict(), dict(use_graph=True)):
        st, res = run_state(inst, "be", order="natural", **kw)
        assert res.bound == run.bound and res.cost == run.cost
        assert list(res.assignment) == list(run.sigma)
