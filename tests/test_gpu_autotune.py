"""The autotuner and the knobs it sets (W, block size, pull degree classes,
push alpha, the per-block cut of batches): no knob changes a result, the
tuner's choice is applied and cached, and a cached choice is reused without
measuring."""
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


def test_knobs_do_not_change_results(kh):
    graphs = small_graphs(950, 5, (40, 400)) + [gg.disjoint_union(gg.star(1100), gg.chung_lu(900, 6.0, 2.2,
                                                                                              300.0, 95))]
    for g in graphs:
        for h in (2, 3):
            want_d, want_c = oracle.hdegrees(g, h), oracle.peel(g, h)
            for light, medium, block, alpha in [(0, 0, 128, 4), (16, 256, 256, 16), (64, 4096, 512, 64),
                                                (10 ** 6, 10 ** 6, 256, 0)]:
                with kh.KHCore.from_graph(g, alpha=alpha) as ctx:
                    kh.khcore_set_degree_classes(ctx.ctx, light, medium)
                    kh.khcore_set_block_size(ctx.ctx, block)
                    assert np.array_equal(ctx.hdegrees(h), want_d), (g.name, h, light, medium, block)
                    assert np.array_equal(ctx.decompose(h), want_c), (g.name, h, light, medium, block)


def test_round_kernel_residency_does_not_change_results(kh):
    g = gg.chung_lu(1500, 7.0, 2.4, 150.0, 94)
    for h in (2, 3):
        want = oracle.peel(g, h)
        rounds = None
        for blocks, sms in ((1, 0), (2, 0), (1, 7), (2, 1), (1, 76)):
            with kh.KHCore.from_graph(g) as ctx:
                kh.khcore_set_round_blocks(ctx.ctx, blocks)
                kh.khcore_set_round_sms(ctx.ctx, sms)
                c, r, _ = ctx.decompose_ex(h)
            assert np.array_equal(c, want), (h, blocks, sms)
            if rounds is None:
                rounds = r
            assert np.array_equal(r, rounds), (h, blocks, sms)


def test_knob_arguments_are_checked(kh):
    g = gg.cycle(20)
    with kh.KHCore.from_graph(g) as ctx:
        for bad in [lambda: kh.khcore_set_degree_classes(ctx.ctx, 10, 5),
                    lambda: kh.khcore_set_degree_classes(ctx.ctx, -1, 5),
                    lambda: kh.khcore_set_block_size(ctx.ctx, 300),
                    lambda: kh.khcore_set_block_graph_max(ctx.ctx, -2),
                    lambda: kh.khcore_set_round_blocks(ctx.ctx, 3),
                    lambda: kh.khcore_set_round_sms(ctx.ctx, -1),
                    lambda: kh.khcore_set_round_sms(ctx.ctx, 100000)]:
            with pytest.raises(kh.KHCoreError):
                bad()


def test_autotune_one_graph_applies_and_caches(kh, tmp_path):
    g = gg.chung_lu(20000, 10.0, 2.4, 400.0, 96)
    cache = str(tmp_path / "tune.jsonl")
    want = oracle.hdegrees(g, 2)
    with kh.KHCore.from_graph(g) as ctx:
        t = kh.khcore_autotune(ctx.ctx, 2, cache)
        assert t["from_cache"] == 0 and t["trials"] >= 10
        assert t["words"] in (4, 8, 16) and t["block"] in (128, 256, 512)
        assert np.array_equal(ctx.hdegrees(2), want)
        core = ctx.decompose(2)
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and '"words": %d' % t["words"] in lines[0]
    with kh.KHCore.from_graph(g) as ctx2:
        t2 = kh.khcore_autotune(ctx2.ctx, 2, cache)
        assert t2["from_cache"] == 1 and t2["trials"] == 0
        for k in ("words", "block", "light_max", "medium_max", "push_alpha"):
            assert t2[k] == t[k], k
        assert np.array_equal(ctx2.decompose(2), core)
    # a different h is another key: measured again, a second line
    with kh.KHCore.from_graph(g) as ctx3:
        assert kh.khcore_autotune(ctx3.ctx, 3, cache)["from_cache"] == 0
    assert len(open(cache).read().strip().splitlines()) == 2


def test_autotune_batch_cut(kh):
    sizes = [600, 1500, 3000, 6000, 9000, 14000]
    graphs = [gg.erdos_renyi_gnm(n, 3 * n, 97 + i) for i, n in enumerate(sizes)]
    v_off, e_off, rp, col = kh.pack_graphs(graphs)
    ctx = kh.khcore_batch_create(v_off, e_off, rp, col)
    try:
        t = kh.khcore_autotune(ctx, 2)
        assert t["block_graph_max"] in [0] + sizes and t["trials"] == 2 * len(sizes)
        core, _, _ = kh.khcore_batch_decompose(ctx, np.full(len(graphs), 2, np.int32))
    finally:
        kh.khcore_destroy(ctx)
    for g, a, b in zip(graphs, v_off[:-1], v_off[1:]):
        assert np.array_equal(core[a:b], oracle.peel(g, 2))
