"""Failure detection without a GPU fault: a device-side wait on a barrier
that nothing completes, and the wait of a launch over all levels for a
producing bucket that never completes, give up after their time limit and
report GPUBE_ETIMEDOUT; the context stays usable (a solve right after is
correct)."""
import time

import pytest

import synth
import paper_1608_05288_gb300 as gb

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    t0 = time.perf_counter()
    rc = gb.lib().util_selftest_wait(50_000_000, None)  # 50 ms limit
    elapsed = time.perf_counter() - t0
    assert rc == gb.ETIMEDOUT
    assert 0.04 < elapsed < 10.0
    inst = synth.config_instance(0, 2)
    res = gb.be_solve(inst)
    assert res.bound == orc.eliminate(inst, orc.minfill(inst)[0], "be").bound


def test_dependency_wait_times_out_and_context_survives(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    t0 = time.perf_counter()
    rc = gb.lib().util_selftest_dep_wait(50_000_000, None)  # 50 ms limit
    elapsed = time.perf_counter() - t0
    assert rc == gb.ETIMEDOUT
    assert 0.04 < elapsed < 10.0
    inst = synth.config_instance(0, 3)
    res = gb.be_solve(inst, batched="fused")
    assert res.bound == orc.eliminate(inst, orc.minfill(inst)[0], "be").bound
