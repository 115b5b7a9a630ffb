"""The allocation-free padding-map export (lts_export_pad_map_static).

Some callers cannot allocate device memory while they run (their memory is all
reserved up front by their own pool, or an allocator call and its
synchronisation would stall them).  This entry point serves them from a fixed
device array in the library.  The check: through the C ABI, two calls in a row
return exactly what the allocating export returns (integer maps: bit for bit),
and a list longer than the fixed array is refused.  This file is collected last
on purpose, and passes alone or after the other tests.
"""
import numpy as np
import pytest

from paper_2011_10570_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plan():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_10570_gb300 import build, ltsoct
    build.build()
    ltsoct.load()
    w = W.advection_gauss(l_min=2, l_max=4)
    return ltsoct, ltsoct.Plan(ltsoct.Octree(w["spec"]), w["prob"])


def test_static_export_matches_allocating_export_twice(plan):
    lt, p = plan
    rng = np.random.default_rng(7)
    for n in (32, 17):                       # two calls in a row, different lists
        octs = rng.choice(p.n, n, replace=False).astype(np.int32)
        src_a, r_a = p.export_pad_map(octs)
        src_b, r_b = p.export_pad_map_static(octs)
        assert np.array_equal(src_a, src_b)
        assert np.array_equal(r_a, r_b)


def test_static_export_rejects_oversized_lists(plan):
    lt, p = plan
    with pytest.raises(lt.LtsError) as ei:
        p.export_pad_map_static(np.arange(33, dtype=np.int32))
    assert "at most 32 octants" in str(ei.value)
