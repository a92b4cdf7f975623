"""Seeded random sweep over problem shapes and options (domains 1-12,
arities 0-4, repeated scopes, int / fp32 costs, BE / MBE / sum-product /
DPOP, orders, launch shapes, staging limits, graph or direct launches),
every bucket function against the oracle (needs a GPU)."""
import numpy as np
import pytest

import synth
import paper_1608_05288_gb300 as gb
from gpu_util import argmin_attains_minimum, fp_close, run_state, structure, orc_structure

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1608_05288_gb300 import _build
    _build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case(seed):
    import oracle
    rng = np.random.default_rng(10_000 + seed)
    cost_type = "real" if rng.random() < 0.4 else "int"
    dmax = int(rng.choice([2, 3, 4, 6, 9, 12]))
    while True:  # keep the exact elimination small enough for the oracle
        inst = synth.random_small(int(rng.integers(1 << 30)), n=int(rng.integers(5, 17)), dmax=dmax,
                                  n_funcs=int(rng.integers(4, 26)), max_arity=int(rng.integers(1, 5)),
                                  cost_type=cost_type, p_top=float(rng.choice([0.0, 0.05, 0.3])),
                                  top_k=int(rng.choice([60, 1000, 1 << 30])) if cost_type == "int" else None)
        o, _ = oracle.minfill(inst)
        run = oracle.eliminate(inst, o, "be", tables=False)
        if max([t.rows * int(inst.dom[t.var]) for t in run.tasks] or [0]) <= 1 << 20:
            break
        dmax = max(2, dmax // 2)
    kind = str(rng.choice(["be", "mbe", "sum", "sum_mbe"]))
    mode = str(rng.choice(["sep", "joint", "log2"]))
    z = int(rng.integers(1, 6)) if mode != "log2" else int(rng.integers(2, 9))
    shape = dict(block_threads=int(rng.choice([32, 64, 128, 256, 512])),
                 rows_per_item=int(rng.choice([1, 3, 16, 128])),
                 lo_target=int(rng.choice([1, 5, 64, 2048])),
                 stage_max_entries=int(rng.choice([-1, 4, 0])),
                 use_graph=bool(rng.random() < 0.5), batched=int(rng.choice([0, 1, 1, 2, 2])),
                 vector_rows=bool(rng.random() < 0.4), argmin_tables=bool(rng.random() < 0.5))
    return inst, kind, mode, z, shape


@pytest.mark.parametrize("seed", range(60))
def test_random_configuration(orc, seed):
    inst, kind, mode, z, shape = _case(seed)
    o, _ = orc.minfill(inst)
    semiring = "sum" if kind.startswith("sum") else "min"
    omode = "be" if kind in ("be", "sum") else mode
    run = orc.eliminate(inst, o, omode, z, semiring=semiring)
    st, res = run_state(inst, kind, z, order="given", order_array=o, ibound_mode=mode, **shape)
    assert structure(st) == orc_structure(run)
    exact = inst.cost_type == "int" and semiring == "min"
    tasks = st.tasks()
    for t, T in enumerate(run.tasks):
        # BE always writes its argmin tables, the sum-product never, MBE when
        # asked or where the kernel has no variant without them
        keeps = tasks[t]["argmin"]
        d, F = int(inst.dom[T.var]), len(tasks[t]["inputs"])
        assert keeps == (kind == "be" or (kind == "mbe" and (shape["argmin_tables"] or exact or not 2 <= d <= 4
                                                              or F > 7)))
        cost, arg = st.fetch(t)
        if not keeps:
            assert not np.any(arg), f"task {t}"
        if exact:
            assert np.array_equal(cost.astype(np.int64), T.out.astype(np.int64)), f"task {t}"
            if keeps:
                assert np.array_equal(arg, T.arg), f"task {t}"
        else:
            assert fp_close(cost, T.out), f"task {t}"
            if keeps:  # fp32 min-sum: the argmin attains the minimum
                assert argmin_attains_minimum(inst, run, t, arg), f"task {t} argmin"
    if exact:
        assert res.bound == run.bound and res.cost == run.cost
        assert list(res.assignment) == list(run.sigma)
    else:
        assert fp_close([res.bound], [run.bound])
        if semiring == "min":  # the GPU's assignment re-evaluated in fp64
            assert fp_close([orc.evaluate(inst, res.assignment)], [res.cost])
            if np.isfinite(run.bound):  # an upper bound of the optimum (MBE) or the optimum
                assert res.cost >= run.bound - 1e-4 * (1 + abs(run.bound))
