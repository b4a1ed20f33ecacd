"""GPU parity: the CUDA path through the C ABI against the CPU oracle,
element by element, bit-exact (integer results)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from conftest import small_graphs

pytestmark = pytest.mark.gpu

WORDS = [1, 2, 4, 8, 16]


@pytest.fixture(scope="module")
def kh():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2006_03372_gb300 as kh
    kh.load_library()
    return kh


def _run(kh, g, h, words=0, loop=None):
    with kh.KHCore.from_graph(g, words=words, loop=loop) as ctx:
        d = ctx.hdegrees(h)
        c, r, st = ctx.decompose_ex(h)
    return d, c, r, st


def test_fig1_example(kh, fig1):
    g, vals = fig1
    for h in [1, 2, 3, 4]:
        d, c, r, st = _run(kh, g, h)
        assert (d == oracle.hdegrees(g, h)).all()
        assert (c == oracle.peel(g, h)).all()
    d, c, r, st = _run(kh, g, 2)
    assert (c == np.array([int(x) for x in vals["core_h2"]])).all()
    # level-synchronous rounds of the example at h=2 (each round one level step)
    want_r = oracle.level_rounds(g, 2, c)
    assert st["rounds"] == want_r.max() + 1 and st["k_max"] == 6
    assert (r == want_r).all()


@pytest.mark.parametrize("h", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("loop", [0, 1])
def test_small_graphs_all_words(kh, h, loop):
    for g in small_graphs(40 + h, 9, (2, 300)):
        want_d = oracle.hdegrees(g, h)
        want_c = oracle.peel(g, h)
        for w in WORDS:
            for alpha in [0, 16, 1 << 20]:
                with kh.KHCore.from_graph(g, words=w, alpha=alpha, loop=loop) as ctx:
                    d = ctx.hdegrees(h)
                    c, r, st = ctx.decompose_ex(h)
                assert (d == want_d).all(), (g.name, h, w, alpha)
                assert (c == want_c).all(), (g.name, h, w, alpha)
                if alpha == 16:
                    fails, _ = oracle.certificate(g, h, c, r)
                    assert fails == 0


@pytest.mark.parametrize("loop", [0, 1])
def test_config1_er_h2_exact(kh, loop):
    g = gg.config1_er()
    want = oracle.peel(g, 2)
    for w in [0, 1, 4, 16]:
        d, c, r, st = _run(kh, g, 2, words=w, loop=loop)
        assert (d == oracle.hdegrees(g, 2)).all()
        assert (c == want).all()
        assert oracle.certificate(g, 2, c, r)[0] == 0


def test_ragged_batches_and_degree_classes(kh):
    # a hub above the block threshold, medium-degree vertices, a ragged tail
    parts = [gg.star(1100), gg.chung_lu(1501, 6.0, 2.2, 700.0, 17), gg.cycle(77), gg.empty(5)]
    g = gg.disjoint_union(*parts)
    deg = g.degrees()
    assert deg.max() > 1024 and ((deg > 32) & (deg <= 1024)).any()
    for h in [1, 2, 3]:
        want_d = oracle.hdegrees(g, h)
        want_c = oracle.peel(g, h) if h < 3 else None
        for w in [1, 8, 16]:
            for alpha in [0, 16, 1 << 20]:  # pull only, automatic, push wherever possible
                with kh.KHCore.from_graph(g, words=w, alpha=alpha, loop=(w // 8) % 2) as ctx:
                    assert (ctx.hdegrees(h) == want_d).all(), (h, w, alpha)
                    if want_c is not None:
                        assert (ctx.decompose(h) == want_c).all(), (h, w, alpha)


def test_closed_forms(kh):
    for n in [1, 2, 7, 40]:
        d, c, _, _ = _run(kh, gg.complete(n), 2)
        assert (d == n - 1).all() and (c == n - 1).all()
    for n in [9, 70]:
        _, c, _, _ = _run(kh, gg.star(n), 2)
        assert (c == n - 1).all()
        _, c, _, _ = _run(kh, gg.star(n), 1)
        assert (c == 1).all()
    for n in [11, 200]:
        for h in [1, 2, 3, 5]:
            d, c, _, _ = _run(kh, gg.cycle(n), h)
            assert (d == min(2 * h, n - 1)).all()
            assert (c == (2 * h if 2 * h < n else n - 1)).all()
            _, c, _, _ = _run(kh, gg.path(n), h)
            assert (c == min(h, n - 1)).all()


def test_edge_cases(kh):
    # empty graph, single vertex, isolated vertices, h >= n
    with kh.KHCore(0, np.zeros(1, np.int32), np.zeros(0, np.int32)) as ctx:
        assert len(ctx.decompose(2)) == 0
        assert len(ctx.hdegrees(2)) == 0
    d, c, _, _ = _run(kh, gg.empty(1), 3)
    assert d[0] == 0 and c[0] == 0
    d, c, _, _ = _run(kh, gg.empty(100), 2)
    assert (d == 0).all() and (c == 0).all()
    g = gg.erdos_renyi_gnm(50, 80, 5)
    _, c_big, _, _ = _run(kh, g, 10_000)
    assert (c_big == oracle.peel(g, 49)).all()
    with kh.KHCore.from_graph(g) as ctx:
        with pytest.raises(kh.KHCoreError) as ei:
            ctx.decompose(0)
        assert ei.value.status == 1
        with pytest.raises(kh.KHCoreError):
            ctx.set_words(3)


def test_device_pointers_in_and_out(kh):
    import torch
    g = gg.chung_lu(4000, 8.0, 2.5, 300.0, 21)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    ctx = kh.khcore_create(g.n, rp, col, stream=torch.cuda.current_stream())
    try:
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        kh.khcore_decompose(ctx, 2, out)
        assert (out.cpu().numpy() == oracle.peel(g, 2)).all()
        kh.khcore_hdegrees(ctx, 3, out)
        assert (out.cpu().numpy() == oracle.hdegrees(g, 3)).all()
    finally:
        kh.khcore_destroy(ctx)


def test_repeatable_and_order_independent(kh):
    g = gg.rmat(11, 8, 0.57, 0.19, 0.19, 0.05, 33)
    perm = np.argsort(gg.Stream(3, "perm").u64(g.n), kind="stable")
    gp = gg.relabel(g, perm)
    _, c1, _, _ = _run(kh, g, 2)
    _, c2, _, _ = _run(kh, g, 2)
    _, c3, _, _ = _run(kh, gp, 2)
    assert (c1 == c2).all()
    assert (c3[perm] == c1).all()
    assert (c1 == oracle.peel(g, 2)).all()


def test_batch_matches_solo_oracle(kh):
    """Many graphs of uneven size in one context, each with its own h: every
    graph's core indices equal the oracle's on that graph alone."""
    rng = gg.Stream(77, "batch-test")
    graphs, hs = [], []
    for i in range(24):
        n = int(5 + rng.below(200, 1)[0])
        if i % 3 == 0:
            graphs.append(gg.erdos_renyi_gnm(n, min(3 * n, n * (n - 1) // 2), 500 + i))
        elif i % 3 == 1:
            graphs.append(gg.chung_lu(n, min(4.0, n / 4), 2.3, max(n / 2, 8.0), 600 + i))
        else:
            graphs.append(gg.cycle(n))
        hs.append(int(1 + rng.below(4, 1)[0]))
    graphs.append(gg.empty(3))
    hs.append(2)
    v_off, e_off, rp, col = kh.pack_graphs(graphs)
    ctx = kh.khcore_batch_create(v_off, e_off, rp, col)
    try:
        kh.khcore_set_graph_blocks(ctx, -1)  # the lock-step union path
        for w, loop in [(1, 0), (4, 1), (16, 0)]:
            kh.khcore_set_words(ctx, w)
            kh.khcore_set_round_loop(ctx, loop)
            core, rnd, st = kh.khcore_batch_decompose(ctx, np.array(hs, dtype=np.int32))
            for g, h, a, b in zip(graphs, hs, v_off[:-1], v_off[1:]):
                assert (core[a:b] == oracle.peel(g, h)).all(), (g.name, h, w)
                assert oracle.certificate(g, h, core[a:b], rnd[a:b])[0] == 0
        # one h for the whole batch through the single-h entry point
        core = kh.khcore_decompose(ctx, 2)
        for g, a, b in zip(graphs, v_off[:-1], v_off[1:]):
            assert (core[a:b] == oracle.peel(g, 2)).all()
        d = kh.khcore_hdegrees(ctx, 3)
        for g, a, b in zip(graphs, v_off[:-1], v_off[1:]):
            assert (d[a:b] == oracle.hdegrees(g, 3)).all()
    finally:
        kh.khcore_destroy(ctx)


def test_barrier_wait_limit_returns_etimeout_and_recovers(kh):
    """A grid-barrier wait that runs out ends the persistent launch with
    KHCORE_ETIMEOUT (no hang, no fault); the next call is exact again."""
    g = gg.erdos_renyi_gnm(3000, 12000, 12)
    want = oracle.peel(g, 2)
    with kh.KHCore.from_graph(g) as ctx:
        kh.khcore_set_wait_limit(ctx.ctx, 0)
        with pytest.raises(kh.KHCoreError) as ei:
            ctx.decompose(2)
        assert ei.value.status == 4
        kh.khcore_set_wait_limit(ctx.ctx, 10 ** 10)
        assert (ctx.decompose(2) == want).all()


def test_hdegrees_of_listed_vertices(kh):
    g = gg.chung_lu(5000, 10.0, 2.5, 400.0, 31)
    rng = gg.Stream(4, "listed")
    verts = np.argsort(rng.u64(g.n), kind="stable")[:777].astype(np.int32)
    with kh.KHCore.from_graph(g) as ctx:
        for h in (1, 2, 3):
            got = kh.khcore_hdegrees_of(ctx.ctx, h, verts)
            assert (got == oracle.hdegree_list(g, h, verts)).all()
        with pytest.raises(kh.KHCoreError):
            kh.khcore_hdegrees_of(ctx.ctx, 2, np.array([3, 3], dtype=np.int32))


def test_round_words_and_loops_agree(kh):
    g = gg.chung_lu(4000, 8.0, 2.5, 300.0, 41)
    want = oracle.peel(g, 2)
    for wr in (1, 2, 4, 8, 16):
        for loop in (0, 1):
            with kh.KHCore.from_graph(g, loop=loop) as ctx:
                kh.khcore_set_round_words(ctx.ctx, wr)
                c, r, st = ctx.decompose_ex(2)
                assert (c == want).all(), (wr, loop)
                assert st["recomputed_total"] <= st["affected_total"]


@pytest.mark.parametrize("loop", [0, 1])
def test_lazy_bounds_and_eager_recompute_agree(kh, loop):
    """The bound-based mode (default) and the eager mode peel the same sets at
    the same levels: core indices and rounds equal, and equal the oracle."""
    graphs = [gg.chung_lu(600, 6.0, 2.5, 60.0, 43), gg.chung_lu(500, 5.0, 2.1, 80.0, 44)] \
        + list(small_graphs(60, 4, (2, 200)))
    for g in graphs:
        for h in (2, 3, 4):
            want = oracle.peel(g, h)
            out = {}
            for lazy in (0, 1):
                with kh.KHCore.from_graph(g, loop=loop, lazy=lazy) as ctx:
                    out[lazy] = ctx.decompose_ex(h)
            (c0, r0, s0), (c1, r1, s1) = out[0], out[1]
            assert (c0 == want).all() and (c1 == want).all(), (g.name, h)
            assert (r0 == r1).all() and s0["rounds"] == s1["rounds"], (g.name, h)
            assert s1["recomputed_total"] <= s0["recomputed_total"] + g.n, (g.name, h)


def _batch_graphs(seed, count, nmax):
    rng = gg.Stream(seed, "block-batch")
    graphs, hs = [], []
    for i in range(count):
        n = int(2 + rng.below(nmax, 1)[0])
        if i % 4 == 0:
            graphs.append(gg.erdos_renyi_gnm(n, min(3 * n, n * (n - 1) // 2), 900 + i))
        elif i % 4 == 1 and n >= 8:
            graphs.append(gg.chung_lu(n, min(4.0, n / 4), 2.3, max(n / 2, 8.0), 950 + i))
        elif i % 4 == 2:
            graphs.append(gg.cycle(n))
        else:
            graphs.append(gg.star(n))
        hs.append(int(1 + rng.below(5, 1)[0]))
    graphs.append(gg.empty(1))
    hs.append(3)
    return graphs, np.array(hs, dtype=np.int32)


def test_graph_blocks_batch_matches_solo_oracle_and_grid_path(kh):
    """A batch of 81 small graphs takes the one-block-per-graph path by
    default: each graph's core indices equal the oracle's on that graph alone,
    and cores and rounds equal the lock-step union path's."""
    graphs, hs = _batch_graphs(81, 80, 150)
    v_off, e_off, rp, col = kh.pack_graphs(graphs)
    ctx = kh.khcore_batch_create(v_off, e_off, rp, col)
    try:
        out = {}
        for mode in (0, -1, 1):
            kh.khcore_set_graph_blocks(ctx, mode)
            out[mode] = kh.khcore_batch_decompose(ctx, hs)
        core, rnd, st = out[0]
        assert st["words_per_vertex"] == 1  # the per-block path ran
        for g, h, a, b in zip(graphs, hs, v_off[:-1], v_off[1:]):
            assert (core[a:b] == oracle.peel(g, int(h))).all(), (g.name, h)
            assert oracle.certificate(g, int(h), core[a:b], rnd[a:b])[0] == 0
        for mode in (-1, 1):
            assert (out[mode][0] == core).all() and (out[mode][1] == rnd).all(), mode
        assert out[-1][2]["rounds"] == st["rounds"]
    finally:
        kh.khcore_destroy(ctx)


@pytest.mark.parametrize("h", [1, 2, 3, 4, 5])
def test_graph_blocks_single_graphs(kh, h):
    """One block decomposing one graph, forced: equal to the oracle, rounds
    equal to the grid path's; graphs span many 64-source batches."""
    for g in list(small_graphs(70 + h, 6, (2, 300))) + [gg.chung_lu(700, 6.0, 2.3, 60.0, 71 + h)]:
        want = oracle.peel(g, h)
        with kh.KHCore.from_graph(g, blocks=1) as ctx:
            c, r, st = ctx.decompose_ex(h)
        with kh.KHCore.from_graph(g, blocks=-1) as ctx:
            c2, r2, st2 = ctx.decompose_ex(h)
        assert (c == want).all(), (g.name, h)
        assert (r == r2).all() and st["rounds"] == st2["rounds"], (g.name, h)


def test_hdegrees_ex_statistics(kh):
    """khcore_hdegrees_ex returns the same h-degrees as the oracle and counts
    the traversed edges of a plain single-source BFS from every vertex (at
    h = 1: the sum of the degrees; at h = 2: sum of deg(v) + sum over
    neighbours of deg(u), i.e. sum deg + sum deg^2)."""
    g = gg.chung_lu(3000, 8.0, 2.5, 200.0, 88)
    deg = np.diff(g.row_ptr).astype(np.int64)
    with kh.KHCore.from_graph(g) as ctx:
        d1, st1 = kh.khcore_hdegrees_ex(ctx.ctx, 1)
        d2, st2 = kh.khcore_hdegrees_ex(ctx.ctx, 2)
    assert (d1 == oracle.hdegrees(g, 1)).all() and (d2 == oracle.hdegrees(g, 2)).all()
    assert st1["edges_traversed"] == int(deg.sum())
    assert st2["edges_traversed"] == int(deg.sum() + (deg * deg).sum())
    assert st2["device_ms"] > 0 and st2["source_batches"] >= 1 and st2["level_bytes"] > 0


def test_batch_mixed_small_and_large_graphs(kh):
    """Default batch mode: small graphs on one block each, the larger ones
    (above 4,096 vertices) alone on the grid-wide path; every graph equals the
    oracle (a cycle: 2h) and the lock-step union path."""
    small, _ = _batch_graphs(91, 12, 200)
    big = [gg.chung_lu(5000, 6.0, 2.5, 80.0, 92), gg.cycle(4300)]
    graphs = small[:6] + big[:1] + small[6:] + big[1:]
    hs = np.array([2, 3, 1, 4, 2, 3, 2, 2, 3, 1, 2, 4, 3, 3, 3], dtype=np.int32)[:len(graphs)]
    v_off, e_off, rp, col = kh.pack_graphs(graphs)
    ctx = kh.khcore_batch_create(v_off, e_off, rp, col)
    try:
        core, rnd, st = kh.khcore_batch_decompose(ctx, hs)
        kh.khcore_set_graph_blocks(ctx, -1)
        core2, rnd2, st2 = kh.khcore_batch_decompose(ctx, hs)
    finally:
        kh.khcore_destroy(ctx)
    assert (core == core2).all() and (rnd == rnd2).all()
    for g, h, a, b in zip(graphs, hs, v_off[:-1], v_off[1:]):
        if g is big[1]:
            assert (core[a:b] == 2 * int(h)).all()
        else:
            assert (core[a:b] == oracle.peel(g, int(h))).all(), (g.name, h)
        assert oracle.certificate(g, int(h), core[a:b], rnd[a:b])[0] == 0
    assert st["k_max"] == st2["k_max"]
