"""Failure paths made on the host, with no GPU fault, trap or hang: the
allocation-failure injector (KHCORE_FAIL_ALLOC_AT) makes the N-th device
allocation fail as if the device were full. Every such failure must return
KHCORE_ENOMEM, release everything the call had allocated, and leave a context
that survived it usable with exact results."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

ENOMEM = 2


@pytest.fixture(scope="module")
def kh():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2006_03372_gb300 as kh
    kh.load_library()
    return kh


def test_injected_allocation_failure_is_enomem_and_leaks_nothing(kh, monkeypatch):
    import torch
    # buffers of >= 2 MiB each (n = 6e5 int32), so a leaked one shows in the
    # device's free memory
    g = gg.erdos_renyi_gnm(600_000, 1_200_000, 81)
    small = gg.erdos_renyi_gnm(400, 1600, 82)
    monkeypatch.delenv("KHCORE_FAIL_ALLOC_AT", raising=False)
    for _ in range(2):  # module loading, first allocations of the process
        ctx = kh.khcore_create(g.n, g.row_ptr, g.col, kh.FLAG_TRUST_INPUT)
        kh.khcore_decompose(ctx, 1)
        kh.khcore_destroy(ctx)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    create_fails = decompose_fails = 0
    for nth in range(1, 90):
        monkeypatch.setenv("KHCORE_FAIL_ALLOC_AT", str(nth))
        try:
            ctx = kh.khcore_create(g.n, g.row_ptr, g.col, kh.FLAG_TRUST_INPUT)
        except kh.KHCoreError as e:
            assert e.status == ENOMEM, str(e)
            create_fails += 1
            continue
        try:
            kh.khcore_decompose(ctx, 1)
        except kh.KHCoreError as e:
            # the BFS rows are allocated on first use: the same context
            # retries with the injection spent
            assert e.status == ENOMEM, str(e)
            decompose_fails += 1
            kh.khcore_decompose(ctx, 1)
        kh.khcore_destroy(ctx)
    monkeypatch.delenv("KHCORE_FAIL_ALLOC_AT")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert create_fails >= 40 and decompose_fails >= 1, (create_fails, decompose_fails)
    assert free1 == free0, f"{(free0 - free1) / 2**20:.1f} MiB not returned"
    # a context created after the failures gives exact results
    with kh.KHCore.from_graph(small) as c2:
        assert np.array_equal(c2.decompose(2), oracle.peel(small, 2))
