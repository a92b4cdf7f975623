"""util_bucket_noalloc: the single-bucket UTIL kernel for callers that cannot
allocate device memory (loops that forbid allocation once running, or
processes whose device memory another allocator owns).  Its scratch is a
fixed array inside the library.  The GPU test compares it with util_bucket
on the same inputs, on two calls in a row (the second call reuses the
scratch the first one left behind); this file is collected last."""
import numpy as np
import pytest

import paper_1608_05288_gb300 as gb
from gpu_util import fp_close

# (separator domains, eliminated domain, input positions, cost type)
CASES = [
    ([4] * 12, 4, [list(range(1, 12)), [0], [11]], "int"),     # the 12x12 grid's largest bucket
    ([3, 5, 2, 7, 3], 6, [[0, 2, 4], [1], [3, 4], []], "int"),  # ragged, several tiles
    ([2] * 9, 3, [list(range(9)), [0, 5]], "real"),
    ([], 5, [[], []], "int"),                                   # a root: one output row
]


def _inputs(torch, rng, sep_dom, d, positions, cost_type):
    tabs = []
    for pos in positions:
        size = int(np.prod([sep_dom[p] for p in pos])) * d if pos else d
        if cost_type == "int":
            t = rng.integers(0, 5000, size=size).astype(np.int32)
        else:
            t = (-np.log(rng.uniform(0.01, 1.0, size=size))).astype(np.float32)
        tabs.append(torch.from_numpy(t).cuda())
    return tabs


@pytest.mark.gpu
def test_noalloc_matches_util_bucket():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_05288_gb300 import _build
    _build.build()
    rng = np.random.default_rng(11)
    for sep_dom, d, positions, ct in CASES:
        tabs = _inputs(torch, rng, sep_dom, d, positions, ct)
        rows = int(np.prod(sep_dom)) if sep_dom else 1
        dt = torch.int32 if ct == "int" else torch.float32
        ref = torch.full((rows,), -1, dtype=dt, device="cuda")
        ref_arg = torch.full((rows,), 255, dtype=torch.uint8, device="cuda")
        gb.util_bucket(sep_dom, d, tabs, positions, ref, ref_arg, ct)
        for _ in range(2):  # two calls in a row share the fixed scratch
            out = torch.full((rows,), -1, dtype=dt, device="cuda")
            arg = torch.full((rows,), 255, dtype=torch.uint8, device="cuda")
            gb.util_bucket_noalloc(sep_dom, d, tabs, positions, out, arg, ct)
            torch.cuda.synchronize()
            if ct == "int":
                assert torch.equal(out, ref) and torch.equal(arg, ref_arg)
            else:
                assert fp_close(out.cpu().numpy(), ref.cpu().numpy())
                assert torch.equal(arg, ref_arg)


def test_scratch_query_flags_oversized_bucket():
    from paper_1608_05288_gb300 import _build
    _build.build()
    # host only: the size query launches nothing and needs no GPU.  2^29 rows
    # of binary variables with seven inputs need offset tables larger than the
    # fixed scratch; util_bucket_noalloc makes the same check, before any CUDA
    # call, and returns ENOMEM for such a bucket
    m = 29
    positions = [list(range(m))] + [[j] for j in range(6)]
    need, limit = gb.util_bucket_scratch_bytes([2] * m, 2, positions)
    assert limit == 4 << 20 and need > limit
    # the test cases above fit
    for sep_dom, d, pos, _ in CASES:
        need, limit = gb.util_bucket_scratch_bytes(sep_dom, d, pos)
        assert 0 < need <= limit
    with pytest.raises(gb.GpubeError) as e:
        gb.util_bucket_scratch_bytes([2, 3], 2, [[1, 0]])  # positions must ascend
    assert e.value.code == gb.EINVAL
