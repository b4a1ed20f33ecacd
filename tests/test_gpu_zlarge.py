"""Full-size parity for the 1e6-vertex Chung-Lu graph at h = 3 (about three
minutes on a GB300: 301,205 peel rounds): the exactness certificate
(oracle.certificate: property (0) on every vertex, the two BFS inequalities on
a seeded sample of low, middle and top core values). In a file of its own,
collected after the other GPU parity tests, because it is the slowest."""
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


def test_chung_lu_1e6_h3_certificate(kh):
    g = gg.config_graph("cl1m")
    h, k = 3, 18
    with kh.KHCore.from_graph(g, flags=kh.FLAG_TRUST_INPUT) as ctx:
        core, rnd, st = ctx.decompose_ex(h)
    assert st["deleted_total"] == g.n and (core >= 0).all()
    order = np.argsort(core, kind="stable")
    sample = np.argsort(gg.Stream(17, "cert-cl1m-3").u64(g.n), kind="stable")[:k // 3]
    picks = np.unique(np.concatenate([order[:k // 3], order[len(order) // 2:][:k // 3], order[-(k // 3):],
                                      sample])).astype(np.int32)
    fails, bad = oracle.certificate(g, h, core, rnd, picks)
    assert fails == 0, picks[bad != 0][:10]
