"""Sum-product elimination (-log Z, solution counting) on the GPU against the
CPU oracle and against closed forms, through the C ABI (needs a GPU).

Tolerance: fp32 sums and fp32 log-sum-exp of fp32-rounded inputs against the
fp64 oracle, |delta| <= 1e-4 (1 + |value|), per table entry and for -log Z.
"""
import itertools

import numpy as np
import pytest

import synth
import paper_1608_05288_gb300 as gb
from gpu_util import fp_close, run_state, structure, orc_structure

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1608_05288_gb300 import _build
    _build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _close(a, b):
    return fp_close(np.array([a]), np.array([b]))


def check_sum_tables(st, run):
    assert structure(st) == orc_structure(run)
    for t, T in enumerate(run.tasks):
        cost, arg = st.fetch(t)
        assert fp_close(cost, T.out), f"task {t}"


LAUNCH_SHAPES = [
    dict(),
    dict(batched=False),
    dict(use_graph=True),
    dict(block_threads=32, rows_per_item=1, lo_target=8),
    dict(block_threads=64, rows_per_item=3, lo_target=5, stage_max_entries=-1),
    dict(batched="fused", use_graph=True),
    dict(batched="fused", block_threads=32, rows_per_item=1, lo_target=8),
    dict(vector_rows=True, block_threads=64, lo_target=16),
]


@pytest.mark.parametrize("shape", range(len(LAUNCH_SHAPES)))
@pytest.mark.parametrize("seed", range(5))
def test_random_real_tables_and_logz(orc, seed, shape):
    inst = synth.random_small(seed, n=9, dmax=6, n_funcs=14, max_arity=4, cost_type="real", p_top=0.05)
    o, _ = orc.minfill(inst)
    run = orc.eliminate(inst, o, "be", semiring="sum")
    st, res = run_state(inst, "sum", order="given", order_array=o, **LAUNCH_SHAPES[shape])
    check_sum_tables(st, run)
    assert _close(res.bound, run.bound)
    assert np.isnan(res.cost)
    r2 = gb.logz_solve(inst, order="given", order_array=o, **LAUNCH_SHAPES[shape])
    assert _close(r2.bound, orc.logz_bruteforce(inst))


@pytest.mark.parametrize("seed", range(4))
def test_counting_matches_oracle(orc, seed):
    # integer WCSPs: Z counts the assignments with no function at the top cost
    inst = synth.random_small(seed + 20, n=9, dmax=4, n_funcs=12, max_arity=3, p_top=0.25)
    o, _ = orc.minfill(inst)
    run = orc.eliminate(inst, o, "be", semiring="sum")
    st, res = run_state(inst, "sum", order="given", order_array=o)
    check_sum_tables(st, run)
    assert _close(res.bound, run.bound)


def test_coloring_counts():
    q = 3
    cases = [
        (synth.coloring(9, [(v, (v + 1) % 9) for v in range(9)], q), (q - 1) ** 9 - (q - 1)),
        (synth.coloring(8, [(v, v + 1) for v in range(7)], q), q * (q - 1) ** 7),
        (synth.coloring(5, list(itertools.combinations(range(5), 2)), 6), 6 * 5 * 4 * 3 * 2),
        (synth.coloring(6, [(0, 1), (1, 2), (2, 3), (3, 4)], q), q * q * (q - 1) ** 4),
    ]
    for inst, count in cases:
        res = gb.logz_solve(inst)
        assert np.exp(-res.bound) == pytest.approx(count, rel=1e-4)
    # no proper colouring of K4 with 3 colours: Z = 0, -log Z = +inf
    k4 = synth.coloring(4, list(itertools.combinations(range(4), 2)), 3)
    assert gb.logz_solve(k4).bound == np.inf


def test_ising_ring_closed_form():
    for n, J in ((12, 0.7), (30, 1.3)):
        want = n * J - np.log((2 * np.cosh(J)) ** n + (2 * np.sinh(J)) ** n)
        assert _close(gb.logz_solve(synth.ising_ring(n, J)).bound, want)


def test_bayes_net_z_is_one_and_evidence(orc):
    inst = synth.bn_prefix(synth.bayes_net_mpe(200, 0), 60)
    res = gb.logz_solve(inst)
    assert abs(res.bound) <= 1e-4
    ev = synth.with_evidence(inst, {0: 1, 5: 0, 17: 1})
    o, _ = orc.minfill(ev)
    run = orc.eliminate(ev, o, "be", semiring="sum")
    assert _close(gb.logz_solve(ev, order="given", order_array=o).bound, run.bound)


@pytest.mark.parametrize("mode", ["sep", "joint", "log2"])
def test_minibucket_sum_bound(orc, mode):
    inst = synth.random_small(7, n=14, dmax=4, n_funcs=22, max_arity=3, cost_type="real", p_top=0.0)
    o, _ = orc.minfill(inst)
    exact = orc.eliminate(inst, o, "be", semiring="sum").bound
    for z in (2, 3, 5):
        run = orc.eliminate(inst, o, mode, z, semiring="sum")
        st, res = run_state(inst, "sum_mbe", z, order="given", order_array=o, ibound_mode=mode)
        check_sum_tables(st, run)
        assert _close(res.bound, run.bound)
        assert res.bound <= exact + 1e-4 * (1 + abs(exact))
        r2 = gb.logz_solve(inst, z, order="given", order_array=o, ibound_mode=mode)
        assert _close(r2.bound, run.bound)


@pytest.mark.parametrize("d", [2, 3, 5])
def test_hub_bucket_many_inputs(orc, d):
    # a hub eliminated first, with ten binary tables to leaves on a chain:
    # the many-input variant under the sum-product
    rng = np.random.default_rng(50 + d)
    n = 11
    dom = np.full(n, d, dtype=np.int32)
    scopes = [np.array([0, v], np.int32) for v in range(1, n)] + [np.array([v, v + 1], np.int32) for v in range(1, n - 1)]
    tables = [-np.log(rng.uniform(0.05, 1.0, size=d * d)) for _ in scopes]
    inst = synth.Instance("hub", dom, scopes, tables, "real", synth.TOP_K)
    order = np.arange(n)
    run = orc.eliminate(inst, order, "be", semiring="sum")
    for shape in (dict(lo_target=d * d * d, block_threads=32, rows_per_item=4), dict(lo_target=d * d, batched="fused")):
        st, res = run_state(inst, "sum", order="given", order_array=order, **shape)
        t0 = st.task(0)
        assert len(t0["inputs"]) == 10 and t0["n_group"] - t0["n_lo"] <= 8 and 10 - t0["n_group"] <= 2
        check_sum_tables(st, run)
        assert _close(res.bound, run.bound)
        st.free()


@pytest.mark.parametrize("d", [2, 3, 4, 5, 8, 9, 10, 12, 16, 40])
def test_domain_classes(orc, d):
    # register variants (d <= 8), the runtime-domain loop (d = 12) and the
    # warp-per-row path (d >= 32)
    inst = synth.random_network_wcsp(12 if d < 32 else 6, d, 0.5, seed=d, p2=0.0, hi=100)
    real = synth.Instance(inst.name + "_r", inst.dom, inst.scopes,
                          [np.asarray(t, np.float64) / 37.0 for t in inst.tables], "real", synth.TOP_K)
    o, _ = orc.minfill(real)
    run = orc.eliminate(real, o, "be", semiring="sum")
    st, res = run_state(real, "sum", order="given", order_array=o)
    check_sum_tables(st, run)
    assert _close(res.bound, run.bound)


def test_many_inputs_and_pipelined_grid(orc):
    # a grid MRF (the pipelined path for d = 4) and a bucket with > 7 inputs
    for inst in (synth.grid_mrf(6, 7, 4, seed=3), synth.random_small(9, n=10, dmax=3, n_funcs=40,
                                                                     max_arity=2, cost_type="real", p_top=0.0)):
        o, _ = orc.best_order(inst)
        run = orc.eliminate(inst, o, "be", semiring="sum")
        st, res = run_state(inst, "sum", order="given", order_array=o)
        check_sum_tables(st, run)
        assert _close(res.bound, run.bound)


def test_free_variables_count():
    # variables in no function multiply Z by their domain sizes
    inst = synth.coloring(6, [(0, 1), (1, 2)], 3)
    inst.dom = np.array([3, 3, 3, 4, 5, 2], dtype=np.int32)
    res = gb.logz_solve(inst)
    assert np.exp(-res.bound) == pytest.approx(3 * 2 * 2 * 4 * 5 * 2, rel=1e-5)


def test_serving_mixes_kinds_and_cost_types(orc):
    # requests of different cost types, top costs and elimination operators
    # share a server; each result equals the request's own oracle value
    import torch
    srv = gb.Server(64 << 20)
    jobs = []
    for i in range(6):
        dc = synth.dcop_random(i, n_range=(15, 25), d_range=(3, 5))
        jobs.append((dc, "dpop", 0, orc.eliminate(dc, orc.pseudotree_order(dc, orc.dfs_pseudotree(dc)), "be").bound))
        mr = synth.grid_mrf(3, 4, 3, seed=i)
        jobs.append((mr, "sum", 0, orc.eliminate(mr, orc.minfill(mr)[0], "be", semiring="sum").bound))
        bn = synth.bayes_net_mpe(14, seed=i)
        jobs.append((bn, "be", 0, orc.eliminate(bn, orc.minfill(bn)[0], "be").bound))
        sm = synth.random_small(i + 60, n=8, dmax=3, n_funcs=10, max_arity=3, p_top=0.2, top_k=50)
        jobs.append((sm, "be", 0, orc.eliminate(sm, orc.minfill(sm)[0], "be").bound))
    ids = [srv.submit(inst, kind, z) for inst, kind, z, _ in jobs]
    for _ in range(10000):
        if srv.step() == 0:
            break
    torch.cuda.synchronize()
    for rid, (inst, kind, z, want) in zip(ids, jobs):
        res = srv.result(rid)
        if inst.cost_type == "int" and kind != "sum":
            assert res.bound == want, (kind, inst.name)
        else:
            assert _close(res.bound, want), (kind, inst.name)
    srv.close()


@pytest.mark.parametrize("d", [2, 3, 4])
@pytest.mark.parametrize("scale,p_inf", [(1.0, 0.0), (60.0, 0.0), (5.0, 0.1)])
def test_grid_rows_factored_and_recomputed(orc, d, scale, p_inf):
    # the pipelined grid rows multiply exp-offsets of the partial sums and of
    # the group run; rows whose product sum is tiny (large cost scale: minima
    # at different values, far apart) or infinite (zero weights) are
    # recomputed from the raw terms.  Both against the oracle.
    inst = synth.grid_mrf(5, 8, d, seed=d, scale=scale, unary=False)
    if p_inf:
        rng = np.random.default_rng(d)
        for t in inst.tables:
            t[rng.random(t.size) < p_inf] = np.inf
    o = np.arange(inst.n, dtype=np.int32)
    run = orc.eliminate(inst, o, "be", semiring="sum")
    for kw in (dict(), dict(use_graph=True, block_threads=128, rows_per_item=16)):
        st, res = run_state(inst, "sum", order="natural", **kw)
        check_sum_tables(st, run)
        assert _close(res.bound, run.bound)
