"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (persistent round loop, automatic W), on outputs the oracle can check
one by one: h-degrees of seeded vertex samples by plain BFS, and the whole
decomposition of the 2000-vertex configuration by Algorithm 1. The core
indices of the large configurations are certified on every vertex in
test_gpu_zlarge.py."""
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


def _sample(g, k, tag):
    return np.argsort(gg.Stream(17, tag).u64(g.n), kind="stable")[:k].astype(np.int32)


@pytest.mark.parametrize("name,h,k", [("cl1m", 2, 400), ("cl1m", 3, 60), ("rmat18", 4, 100), ("rmat18", 5, 60)])
def test_hdegrees_sampled(kh, name, h, k):
    g = gg.config_graph(name)
    with kh.KHCore.from_graph(g, flags=kh.FLAG_TRUST_INPUT) as ctx:
        d = ctx.hdegrees(h)
    v = _sample(g, k, f"hdeg-{name}-{h}")
    assert (d[v] == oracle.hdegree_list(g, h, v)).all()


def test_config1_full_parity_bench_configuration(kh):
    g = gg.config1_er()
    with kh.KHCore.from_graph(g, flags=kh.FLAG_TRUST_INPUT) as ctx:
        kh.khcore_set_profiling(ctx.ctx, 1)
        core, rnd, st = ctx.decompose_ex(2)
    assert (core == oracle.peel(g, 2)).all()
    assert oracle.certificate(g, 2, core, rnd)[0] == 0
