"""khcore_hdegrees_static: the h-degrees of listed vertices for callers that
may not allocate device memory while they run (a plugin inside a process that
owns all device memory through its own pool, a latency-bound path that cannot
take cudaMalloc's device-wide synchronisation). Its BFS scratch is a fixed
array inside the library, shared by every call, so two calls in a row must
each start from a clean state. Compared with khcore_hdegrees_of, which
allocates its scratch in a context; integer results, bit-exact.

Collected last (file name), so that a run stopping at the first failure has
run every other test before this one."""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2006_03372_gb300 as kh
    kh.load_library()
    return kh


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def test_static_scratch_matches_context_entry_point_twice(kh):
    import torch
    g = gg.chung_lu(20000, 8.0, 2.5, 300.0, 71)
    m = int(g.row_ptr[-1])
    rp, col = _dev(g.row_ptr), _dev(g.col)
    order = np.argsort(gg.Stream(71, "static-verts").u64(g.n), kind="stable").astype(np.int32)
    # first call: 500 vertices (a ragged batch of 64); second: 1300 other
    # vertices at a larger h, over rows the first call left behind
    cases = [(2, order[:500]), (3, order[500:1800])]
    with kh.KHCore.from_graph(g) as ctx:
        want = [kh.khcore_hdegrees_of(ctx.ctx, h, v) for h, v in cases]
    for (h, v), w in zip(cases, want):
        out = torch.full((len(v),), -7, dtype=torch.int32, device="cuda")
        kh.khcore_hdegrees_static(g.n, m, rp, col, h, _dev(v), out)
        assert (out.cpu().numpy() == w).all(), h


def test_static_scratch_rejects_what_it_cannot_hold_and_recovers(kh):
    import torch
    g = gg.chung_lu(3000, 6.0, 2.5, 100.0, 72)
    m = int(g.row_ptr[-1])
    rp, col = _dev(g.row_ptr), _dev(g.col)
    v = _dev(np.arange(0, 3000, 7))
    out = torch.empty(len(v), dtype=torch.int32, device="cuda")
    # sizes beyond the fixed array: refused before any device work
    with pytest.raises(kh.KHCoreError, match="too large"):
        kh.khcore_hdegrees_static(2_000_000, 40_000_000, rp, col, 2, v, out)
    # a repeated listed id is found on the device
    rep = _dev(np.array([5, 9, 5], dtype=np.int32))
    with pytest.raises(kh.KHCoreError, match="twice"):
        kh.khcore_hdegrees_static(g.n, m, rp, col, 2, rep, torch.empty(3, dtype=torch.int32, device="cuda"))
    # the next call starts clean
    kh.khcore_hdegrees_static(g.n, m, rp, col, 2, v, out)
    with kh.KHCore.from_graph(g) as ctx:
        want = kh.khcore_hdegrees_of(ctx.ctx, 2, v.cpu().numpy())
    assert (out.cpu().numpy() == want).all()
