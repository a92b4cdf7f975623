"""Conditioning (util_condition): repeated runs of one bound plan under
changing evidence, against the oracle on the problem with the clamps written
in as unary functions (needs a GPU).  Integer WCSPs bit for bit; fp32 within
|delta| <= 1e-4 (1 + |value|)."""
import numpy as np
import pytest

import synth
import paper_1608_05288_gb300 as gb
from gpu_util import check_tables, fp_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1608_05288_gb300 import _build
    _build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


STEPS = [{}, {2: 1}, {5: 0, 2: 2}, {2: None}, {8: 1, 5: None}, {8: None}]


def _run(st):
    st.run()
    res = st.value()
    st.sync()
    return res


@pytest.mark.parametrize("use_graph,batched", [(False, "level"), (True, "level"), (True, "fused")])
@pytest.mark.parametrize("kind,mode,z", [("be", "be", 0), ("mbe", "sep", 2)])
def test_integer_conditioning_sequence(orc, use_graph, batched, kind, mode, z):
    inst = synth.random_small(31, n=10, dmax=3, n_funcs=14, max_arity=3, p_top=0.1)
    ev_vars = [2, 5, 8]
    o, _ = orc.minfill(inst)
    st = gb.UtilState(inst, kind, z, order="given", order_array=o, ibound_mode="sep",
                      evidence_vars=ev_vars, use_graph=use_graph, batched=batched)
    st.bind()
    cur = {}
    for step in STEPS:
        step = {v: (None if a is None else a % int(inst.dom[v])) for v, a in step.items()}
        st.condition(step)
        cur.update(step)
        res = _run(st)
        aug = synth.with_evidence(inst, cur, declared=ev_vars)
        run = orc.eliminate(aug, o, mode, z)
        check_tables(aug, st, run)
        assert res.bound == run.bound and res.cost == run.cost
        assert list(res.assignment) == list(run.sigma)
        for v, a in cur.items():
            if a is not None and res.cost < inst.top_k:
                assert res.assignment[v] == a


def test_condition_before_bind(orc):
    inst = synth.random_small(32, n=9, dmax=3, n_funcs=12, max_arity=3)
    o, _ = orc.minfill(inst)
    st = gb.UtilState(inst, "be", order="given", order_array=o, evidence_vars=[0, 4])
    st.condition({4: 1})
    st.bind()
    res = _run(st)
    run = orc.eliminate(synth.with_evidence(inst, {4: 1}, declared=[0, 4]), o, "be")
    assert res.bound == run.bound and list(res.assignment) == list(run.sigma)


def test_mpe_and_probability_of_evidence(orc):
    inst = synth.bn_prefix(synth.bayes_net_mpe(200, 1), 40)
    ev_vars = [0, 3, 11, 27, 39]
    o, _ = orc.minfill(inst)
    mpe = gb.UtilState(inst, "be", order="given", order_array=o, evidence_vars=ev_vars, use_graph=True)
    pe = gb.UtilState(inst, "sum", order="given", order_array=o, evidence_vars=ev_vars, use_graph=True)
    mpe.bind()
    pe.bind()
    rng = np.random.default_rng(0)
    cur = {}
    for _ in range(5):
        v = int(rng.choice(ev_vars))
        cur[v] = int(rng.integers(0, int(inst.dom[v])))
        mpe.condition(cur)
        pe.condition(cur)
        aug = synth.with_evidence(inst, cur, declared=ev_vars)
        r1, r2 = _run(mpe), _run(pe)
        run1 = orc.eliminate(aug, o, "be")
        run2 = orc.eliminate(aug, o, "be", semiring="sum")
        assert fp_close([r1.bound], [run1.bound])
        assert fp_close([orc.evaluate(aug, r1.assignment)], [run1.bound])
        assert fp_close([r2.bound], [run2.bound])
    pe.condition({v: None for v in ev_vars})
    assert abs(_run(pe).bound) <= 1e-4  # no evidence: Z = 1
