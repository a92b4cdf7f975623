"""Continuous-batching server: every result is the same alone and in the mix
(bit for bit, integer DCOPs), admission respects the memory budget, and an
instance larger than the budget fails with ENOMEM once planned."""
import numpy as np
import pytest

import synth
import paper_1608_05288_gb300 as gb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _alone(inst):
    st = gb.dpop_util(inst, inst.parent)
    r = st.value()
    st.free()
    return r


def _drain(srv, ids, limit=100000):
    for _ in range(limit):
        if srv.step() == 0:
            break
    return {i: srv.result(r) for i, r in ids.items()}


def test_mix_equals_alone(orc):
    insts = [synth.dcop_random(s, n_range=(20, 120)) for s in range(24)]
    alone = [_alone(x) for x in insts]
    srv = gb.Server(2 << 30, max_slots=16)
    ids = {}
    # staggered arrivals: some requests join while others are mid-way
    for i, x in enumerate(insts):
        ids[i] = srv.submit(x, "dpop", parent=x.parent)
        if i % 3 == 0:
            srv.step()
    got = _drain(srv, ids)
    for i, x in enumerate(insts):
        assert got[i] is not None
        assert got[i].bound == alone[i].bound and got[i].cost == alone[i].cost
        assert list(got[i].assignment) == list(alone[i].assignment)
    st = srv.stats()
    assert st["max_inflight"] > 1  # requests really overlapped
    assert st["launches"] < sum(a.n_levels for a in alone)  # levels were merged
    srv.close()
    # and the small ones against the oracle
    for i in range(3):
        o = orc.pseudotree_order(insts[i], insts[i].parent)
        assert orc.eliminate(insts[i], o, "be", tables=False).bound == alone[i].bound


def test_budget_admission_and_refusal():
    insts = [synth.dcop_random(100 + s, n_range=(30, 60)) for s in range(10)]
    sizes = [gb.UtilState(x, "dpop", parent=x.parent).info()["arena_bytes"] for x in insts]
    budget = int(max(sizes) * 1.5) + (1 << 20)
    srv = gb.Server(budget, max_slots=8)
    ids = {i: srv.submit(x, "dpop", parent=x.parent) for i, x in enumerate(insts)}
    got = _drain(srv, ids)
    assert all(got[i] is not None for i in ids)
    st = srv.stats()
    assert st["peak_bytes"] <= budget
    for i, x in enumerate(insts):
        assert got[i].bound == _alone(x).bound
    big = synth.config_instance(1, 0)  # the 12x12 grid needs gigabytes
    assert gb.UtilState(big, "be", order="best").info()["arena_bytes"] > budget
    rid = srv.submit(big, "be", order="best")  # planned by the server's planner threads
    for _ in range(100000):
        if srv.step() == 0:
            break
    with pytest.raises(gb.GpubeError) as e:
        srv.result(rid)
    assert e.value.code == gb.ENOMEM
    srv.close()


def test_many_submissions_planned_in_parallel():
    # a burst of submissions (planned by the pool while earlier ones run);
    # the caller's problem objects are released right after submit
    insts = [synth.dcop_random(300 + s, n_range=(20, 80)) for s in range(60)]
    srv = gb.Server(2 << 30, max_slots=32)
    ids = {}
    for i, x in enumerate(insts):
        w = gb.WCSP(x)
        ids[i] = srv.submit(w, "dpop", parent=x.parent)
        del w
    got = _drain(srv, ids)
    for i, x in enumerate(insts[:12]):
        assert got[i].bound == _alone(x).bound
    srv.close()


def test_mbe_and_be_requests_in_one_server(orc):
    a = synth.config_instance(0, 3)
    b = synth.random_small(77, n=9, dmax=4, n_funcs=12)
    srv = gb.Server(1 << 28, max_slots=4)
    ia = srv.submit(a, "be")
    ib = srv.submit(b, "mbe", 2, ibound_mode="sep")
    got = _drain(srv, {0: ia, 1: ib})
    assert got[0].bound == gb.be_solve(a).bound
    assert got[1].bound == gb.mbe_solve(b, 2, ibound_mode="sep").bound
    srv.close()
