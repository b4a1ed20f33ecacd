"""The paper's exact h-degree update on the GPU (Sec. IV-A, Observation 2,
Theorem 1 and Algorithm 3, with the bitmaps of Sec. IV-B, Algorithm 4):
per deletion against the oracle's restatement of the same algorithm
(oracle.bitmap_update) and a fresh BFS (oracle.hdegrees), and whole
decompositions driven by it (Algorithm 2, khcore_set_update(ctx, 1)) against
Algorithm 1, bit-exact, rounds included."""
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


def _alive_subset(g, frac, seed):
    u = gg.Stream(seed, "alive").u64(g.n)
    return ((u % 1000) < int(1000 * frac)).astype(np.uint8)


def test_table1_ball_of_v5(kh, fig1):
    # Table 1: v5 deleted from G - {v1, v2, v3} at h = 2
    g, vals = fig1
    alive = np.ones(g.n, np.uint8)
    alive[[0, 1, 2]] = 0
    deg = oracle.hdegrees(g, 2, alive)
    with kh.KHCore.from_graph(g) as ctx:
        got, ball = kh.khcore_bitmap_update(ctx.ctx, 2, alive, 4, deg)
    want, _, _ = oracle.bitmap_update(g, 2, 4, deg, alive, trace_cap=g.n)
    assert ball == len(vals["ball2_v5_after_v123"])
    assert np.array_equal(got, want)
    a2 = alive.copy()
    a2[4] = 0
    fresh = oracle.hdegrees(g, 2, a2)
    assert np.array_equal(got[a2 == 1], fresh[a2 == 1])


@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_per_deletion_matches_oracle_and_fresh_bfs(kh, h):
    graphs = small_graphs(700 + h, 6, (10, 220)) + [gg.chung_lu(900, 6.0, 2.3, 120.0, 33 + h)]
    for gi, g in enumerate(graphs):
        if g.n < 2:
            continue
        alive = _alive_subset(g, 0.85, 10 * gi + h)
        deg = oracle.hdegrees(g, h, alive)
        # within the bitmap limit: |N_v^{h-1}| <= 256 (h = 1: no bits at all)
        inner = oracle.hdegrees(g, h - 1, alive) if h > 1 else np.zeros(g.n, np.int32)
        live = np.flatnonzero((alive == 1) & (inner <= 256))
        rng = gg.Stream(gi, f"upd-{h}")
        picks = live[np.argsort(rng.u64(len(live)), kind="stable")[:6]]
        with kh.KHCore.from_graph(g) as ctx:
            for v in picks:
                got, ball = kh.khcore_bitmap_update(ctx.ctx, h, alive, int(v), deg)
                want, labels, _ = oracle.bitmap_update(g, h, int(v), deg, alive, trace_cap=g.n)
                assert ball == len(labels), (g.name, h, v)
                assert np.array_equal(got, want), (g.name, h, v)
                a2 = alive.copy()
                a2[v] = 0
                fresh = oracle.hdegrees(g, h, a2)
                assert np.array_equal(got[a2 == 1], fresh[a2 == 1]), (g.name, h, v)


def test_multi_word_bitmaps_and_large_balls(kh):
    # |N_v^{h-1}| > 64 (several bitmap words) and balls of thousands of members
    g = gg.disjoint_union(gg.star(200), gg.chung_lu(3000, 10.0, 2.2, 400.0, 61))
    alive = np.ones(g.n, np.uint8)
    with kh.KHCore.from_graph(g) as ctx:
        for h in (2, 3):
            d = oracle.hdegrees(g, h, alive)
            inner = oracle.hdegrees(g, h - 1, alive)  # |N_v^{h-1}|: bitmap bits
            ok = np.flatnonzero(inner <= 256)
            big_ball = ok[np.argsort(-d[ok], kind="stable")[:3]]
            wide = ok[inner[ok] > 64][:3]
            picks = np.unique(np.concatenate([big_ball, wide, [0]]))
            assert (inner[picks] > 64).any() and d[picks].max() > 1000
            for v in picks:
                got, ball = kh.khcore_bitmap_update(ctx.ctx, h, alive, int(v), d)
                want, labels, _ = oracle.bitmap_update(g, h, int(v), d, alive, trace_cap=g.n)
                assert ball == len(labels) and np.array_equal(got, want), (v, h)
    # over the limits (|N_v^{h-1}| = 299 > 256): refused, nothing changed
    big = gg.star(300)
    with kh.KHCore.from_graph(big) as ctx:
        d0 = oracle.hdegrees(big, 2)
        with pytest.raises(kh.KHCoreError, match="limits"):
            kh.khcore_bitmap_update(ctx.ctx, 3, np.ones(big.n, np.uint8), 1, d0)


@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_decomposition_with_the_paper_update(kh, h):
    for g in small_graphs(760 + h, 8, (2, 260)) + [gg.config1_er()]:
        want = oracle.peel(g, h)
        with kh.KHCore.from_graph(g, update=1) as ctx:
            c, r, st = ctx.decompose_ex(h)
        with kh.KHCore.from_graph(g) as ref:
            _, r0, _ = ref.decompose_ex(h)
        assert np.array_equal(c, want), (g.name, h)
        assert np.array_equal(r, r0), (g.name, h)  # the same level-synchronous rounds
        assert oracle.certificate(g, h, c, r)[0] == 0


def test_paper_update_falls_back_over_the_limits(kh):
    # a hub with 300 neighbours (|N_v^{h-1}| > 256 at h = 3) and rounds that
    # delete more than 64 vertices: those rounds use the BFS recompute
    g = gg.disjoint_union(gg.star(301), gg.cycle(500), gg.erdos_renyi_gnm(700, 2100, 5))
    for h in (2, 3):
        with kh.KHCore.from_graph(g, update=1) as ctx:
            c = ctx.decompose(h)
        assert np.array_equal(c, oracle.peel(g, h)), h
