"""khcore_hdegrees_static: the h-degrees of listed vertices for callers that
may not allocate device memory while they run (a plugin inside a process that
owns all device memory through its own pool, a latency-bound path that cannot
take cudaMalloc's device-wide synchronisation). Its BFS scratch is a fixed
array inside the library, shared by every call, so two calls in a row must
each start from a clean state. Checked against the CPU oracle (one BFS per
listed vertex, Sec. II) and against khcore_hdegrees_of, which allocates its
scratch in a context; integer results, bit-exact.

Collected last (file name), so that a run stopping at the first failure has
run every other test before this one."""
import numpy as np
import pytest

import graphgen as gg
import oracle

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


def test_static_scratch_matches_oracle_and_context_entry_point_twice(kh):
    import torch
    g = gg.chung_lu(20000, 8.0, 2.5, 300.0, 71)
    m = int(g.row_ptr[-1])
    rp, col = _dev(g.row_ptr), _dev(g.col)
    order = np.argsort(gg.Stream(71, "static-verts").u64(g.n), kind="stable").astype(np.int32)
    # first call: 500 vertices (a ragged batch of 64); second: 1300 other
    # vertices at a larger h, over rows the first call left behind
    cases = [(2, order[:500]), (3, order[500:1800])]
    with kh.KHCore.from_graph(g) as ctx:
        via_ctx = [kh.khcore_hdegrees_of(ctx.ctx, h, v) for h, v in cases]
    for (h, v), w in zip(cases, via_ctx):
        out = torch.full((len(v),), -7, dtype=torch.int32, device="cuda")
        kh.khcore_hdegrees_static(g.n, m, rp, col, h, _dev(v), out)
        got = out.cpu().numpy()
        assert np.array_equal(got, oracle.hdegree_list(g, h, v)), h
        assert np.array_equal(got, w), h


def test_static_scratch_allocates_nothing_on_a_caller_stream(kh):
    import torch
    g = gg.erdos_renyi_gnm(30000, 120000, 73)
    m = int(g.row_ptr[-1])
    rp, col = _dev(g.row_ptr), _dev(g.col)
    v = np.arange(3, g.n, 37, dtype=np.int32)
    vd = _dev(v)
    out = torch.full((len(v),), -1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()  # inputs were written on the default stream
    # the first call on the device loads the library's device code (and with
    # it the fixed array) and caches the array's address: the caller's set-up
    kh.khcore_hdegrees_static(g.n, m, rp, col, 2, vd, out, stream=s.cuda_stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    out.fill_(-1)
    torch.cuda.synchronize()
    kh.khcore_hdegrees_static(g.n, m, rp, col, 3, vd, out, stream=s.cuda_stream)
    got = out.cpu().numpy()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == reserved0
    assert np.array_equal(got, oracle.hdegree_list(g, 3, v))


def test_static_scratch_rejects_what_it_cannot_hold_and_recovers(kh):
    import torch
    g = gg.chung_lu(3000, 6.0, 2.5, 100.0, 72)
    m = int(g.row_ptr[-1])
    rp, col = _dev(g.row_ptr), _dev(g.col)
    vh = np.arange(0, 3000, 7, dtype=np.int32)
    v = _dev(vh)
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
    assert np.array_equal(out.cpu().numpy(), oracle.hdegree_list(g, 2, vh))
