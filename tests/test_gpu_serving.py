"""Serving: requests admitted by memory budget into concurrent batches give
exactly the core indices each graph gets alone (tolerance 0: integers)."""
import time

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


def _requests(count, seed):
    rng = gg.Stream(seed, "serve-test")
    out = []
    for i in range(count):
        n = int(20 + rng.below(400, 1)[0])
        d = 2.0 + 4.0 * float(rng.uniform(1)[0])
        g = gg.chung_lu(n, d, 2.5, max(np.sqrt(d * n), 2 * d), 900 + i)
        h = int(1 + rng.below(4, 1)[0])
        out.append((g, h))
    return out


def test_served_equals_alone(kh):
    reqs = _requests(40, 5)
    alone = [oracle.peel(g, h) for g, h in reqs]
    budget = sum(kh.request_bytes(g.n, g.m_directed) for g, _ in reqs[:6])  # ~6 at a time
    with kh.Server(budget, slots=3, max_batch=8) as srv:
        tickets = []
        for i, (g, h) in enumerate(reqs):
            tickets.append(srv.submit(g.n, g.row_ptr, g.col, h))
            if i % 7 == 3:
                time.sleep(0.002)  # later requests arrive while earlier ones run
        lat = []
        for t, (g, h), want in zip(tickets, reqs, alone):
            core, ms = srv.wait(t, timeout_s=120)
            assert (core == want).all(), (g.name, h)
            lat.append(ms)
        st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["batches"] >= 2  # admission split the stream into several batches
    assert min(lat) >= 0


def test_request_larger_than_budget_is_rejected(kh):
    g = gg.cycle(1000)
    with kh.Server(kh.request_bytes(10, 20), slots=1) as srv:
        with pytest.raises(kh.KHCoreError) as ei:
            srv.submit(g.n, g.row_ptr, g.col, 2)
        assert ei.value.status == 2


def test_batch_of_one_equals_context(kh):
    g = gg.erdos_renyi_gnm(300, 900, 8)
    with kh.Server(1 << 30, slots=1) as srv:
        t = srv.submit(g.n, g.row_ptr, g.col, 3)
        core, _ = srv.wait(t)
    with kh.KHCore.from_graph(g) as ctx:
        assert (ctx.decompose(3) == core).all()
