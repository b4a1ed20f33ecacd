"""The paper's sampling variant on the GPU (Sec. IV-C, Algorithms 5 and 6):
estimated core indices on a caller-drawn sample, bit-exact against the
oracle's restatement (oracle.peel_sampled) on the same sample; exact with the
full sample and with the empty one (no vertex has a rate); and the paper's
precision metric (Sec. V, Exp-4) against the exact cores."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from conftest import small_graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2006_03372_gb300 as kh
    kh.load_library()
    return kh


def sample(n, rate, seed):
    """r|V| vertices drawn uniformly (Algorithm 5): the rate's share of a
    seeded permutation."""
    perm = np.argsort(gg.Stream(seed, "sample").u64(n), kind="stable")
    s = np.zeros(n, np.uint8)
    s[perm[: int(round(rate * n))]] = 1
    return s


def precision(exact, est):
    """Sec. V, Exp-4: 1 - (sum over v of |core - est| / core) / |V|, over the
    vertices with core > 0 (the term is undefined at core 0)."""
    m = exact > 0
    return 1.0 - float(np.mean(np.abs(exact[m] - est[m]) / exact[m]))


@pytest.mark.parametrize("h", [1, 2, 3])
def test_sampled_cores_match_the_oracle(kh, h):
    for i, g in enumerate(small_graphs(800 + h, 7, (2, 260)) + [gg.chung_lu(700, 6.0, 2.3, 80.0, 81 + h)]):
        for rate in (0.1, 0.35, 0.8):
            in_s = sample(g.n, rate, 10 * i + h)
            want, _ = oracle.peel_sampled(g, h, in_s)
            with kh.KHCore.from_graph(g) as ctx:
                got, rnd, st = kh.khcore_decompose_sampled(ctx.ctx, h, in_s)
            assert np.array_equal(got, want), (g.name, h, rate)
            assert st["deleted_total"] == g.n


def test_full_and_empty_samples_are_exact(kh):
    g = gg.chung_lu(900, 7.0, 2.4, 90.0, 85)
    for h in (1, 2, 3):
        exact = oracle.peel(g, h)
        with kh.KHCore.from_graph(g) as ctx:
            full, _, _ = kh.khcore_decompose_sampled(ctx.ctx, h, np.ones(g.n, np.uint8))
            empty, _, _ = kh.khcore_decompose_sampled(ctx.ctx, h, np.zeros(g.n, np.uint8))
            plain = ctx.decompose(h)  # the context is reusable afterwards
        assert np.array_equal(full, exact) and np.array_equal(empty, exact) and np.array_equal(plain, exact), h


def test_precision_grows_with_the_sample(kh):
    g = gg.chung_lu(2500, 8.0, 2.5, 150.0, 86)
    exact = oracle.peel(g, 2)
    prec = {}
    with kh.KHCore.from_graph(g) as ctx:
        for rate in (0.1, 0.4, 1.0):
            in_s = sample(g.n, rate, 87)
            est, _, _ = kh.khcore_decompose_sampled(ctx.ctx, 2, in_s)
            assert np.array_equal(est, oracle.peel_sampled(g, 2, in_s)[0]), rate
            prec[rate] = precision(exact, est)
    assert prec[1.0] == 1.0 and prec[0.4] >= prec[0.1] and prec[0.1] > 0.8, prec
