"""Pins for the CPU oracle, independent of the oracle itself.

Each test checks the oracle against something the paper or plain mathematics
fixes: the paper's running example (Sec. II Example 1, Sec. IV Example 2 and
Table 1), SciPy's all-pairs shortest paths (a library routine, for d_v^h),
closed forms on structured graphs, Definition 2 by exhaustion, the classic
k-core at h = 1 (Sec. II: the (k,1)-core is the k-core) via networkx and the
Batagelj-Zaversnik bin sort, and invariants of the model.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import graphgen as gg
import oracle
from conftest import small_graphs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def scipy_hdeg(g, h, alive=None):
    """d_v^h by SciPy's unweighted all-pairs shortest paths on G[alive]."""
    n = g.n
    alive = np.ones(n, bool) if alive is None else np.asarray(alive, bool)
    src = np.repeat(np.arange(n), g.degrees())
    A = sp.csr_matrix((np.ones(len(g.col)), (src, g.col)), shape=(n, n))
    idx = np.flatnonzero(alive)
    out = np.full(n, -1, dtype=np.int64)
    if len(idx) == 0:
        return out
    D = shortest_path(A[idx][:, idx], unweighted=True, directed=False)
    out[idx] = (D <= h).sum(axis=1) - 1
    return out


# ---------------------------------------------------------------- paper pins

def test_fig1_core_h2_matches_example1(fig1):
    g, vals = fig1
    want = np.array([int(x) for x in vals["core_h2"]])
    assert (oracle.peel(g, 2) == want).all()
    assert (oracle.bruteforce(g, 2) == want).all()


def test_fig1_level_rounds_match_example2_order(fig1):
    # the level-synchronous round sequence (4:{v1}) (4:{v2,v3}) (5:{v5})
    # (5:{v4,v6}) (5:{v7}) (6:{v8..v14}), derived by hand in the golden file
    g, vals = fig1
    want = np.array([int(x) for x in vals["rounds_h2"]])
    core = np.array([int(x) for x in vals["core_h2"]])
    rnd = oracle.level_rounds(g, 2, core)
    assert np.array_equal(rnd, want)
    # and the certificate accepts exactly this pair
    assert oracle.certificate(g, 2, core, rnd)[0] == 0


def test_fig1_core_h1_is_2_everywhere(fig1):
    g, vals = fig1
    want = np.array([int(x) for x in vals["core_h1"]])
    assert (oracle.peel(g, 1) == want).all()
    assert (oracle.kcore_bz(g) == want).all()


def test_fig1_example2_hdegrees(fig1):
    g, vals = fig1
    d = oracle.hdegrees(g, 2)
    v1 = 0
    assert d[v1] == int(vals["hdeg2_v1"][0])
    assert (d[1:] > d[v1]).all(), "v1 is the unique minimum"
    alive = np.ones(g.n, np.uint8)
    alive[v1] = 0
    d1 = oracle.hdegrees(g, 2, alive)
    for item in vals["after_v1_hdeg2"]:
        v, want = item.split(":")
        assert d1[int(v) - 1] == int(want)
    # the ball of v1 is exactly {v2,v3,v4,v6}: deleting a ball vertex lowers
    # d^2(v1), deleting anything else leaves it at 4
    ball = {int(x) - 1 for x in vals["ball2_v1"]}
    for u in range(1, g.n):
        a = np.ones(g.n, np.uint8)
        a[u] = 0
        assert (oracle.hdegrees(g, 2, a)[v1] < 4) == (u in ball)


def test_fig1_table1_ball_of_v5(fig1):
    g, vals = fig1
    alive = np.ones(g.n, np.uint8)
    alive[[0, 1, 2]] = 0
    ball = sorted(int(x) - 1 for x in vals["ball2_v5_after_v123"])
    far = sorted(int(x) - 1 for x in vals["dist2_v5_after_v123"])
    v5 = 4
    assert oracle.hdegrees(g, 2, alive)[v5] == len(ball)
    assert oracle.hdegrees(g, 1, alive)[v5] == len(ball) - len(far)
    # exact membership: removing a ball vertex lowers d^2(v5) by at least one
    for u in range(3, g.n):
        if u == v5:
            continue
        a = alive.copy()
        a[u] = 0
        dropped = oracle.hdegrees(g, 2, a)[v5] < len(ball)
        assert dropped == (u in ball)


# ---------------------------------------------------------------- h-degrees

@pytest.mark.parametrize("h", [1, 2, 3, 4, 6])
def test_hdegrees_match_scipy_shortest_path(h):
    for g in small_graphs(7, 9, (5, 60)):
        assert (oracle.hdegrees(g, h) == scipy_hdeg(g, h)).all(), g.name


@pytest.mark.parametrize("h", [1, 2, 3])
def test_hdegrees_induced_subgraph_match_scipy(h):
    rng = gg.Stream(11, "alive")
    for g in small_graphs(8, 9, (5, 60)):
        alive = (rng.uniform(g.n) < 0.7).astype(np.uint8)
        got = oracle.hdegrees(g, h, alive)
        want = scipy_hdeg(g, h, alive)
        assert (got == want).all(), g.name


def test_hdegrees_closed_forms():
    for n in [1, 2, 5, 9]:
        assert (oracle.hdegrees(gg.complete(n), 1) == n - 1).all()
    for n in [3, 7]:
        s = gg.star(n)
        d1, d2 = oracle.hdegrees(s, 1), oracle.hdegrees(s, 2)
        assert d1[0] == n - 1 and (d1[1:] == 1).all()
        assert (d2 == n - 1).all()
    for n in [5, 8, 11]:
        for h in [1, 2, 3, 4, 6]:
            assert (oracle.hdegrees(gg.cycle(n), h) == min(2 * h, n - 1)).all()
            i = np.arange(n)
            want = np.minimum(i, h) + np.minimum(n - 1 - i, h)
            assert (oracle.hdegrees(gg.path(n), h) == want).all()
    assert (oracle.hdegrees(gg.empty(6), 3) == 0).all()


def test_hdegree_list_matches_full():
    g = gg.chung_lu(3000, 8.0, 2.5, 200.0, 9)
    v = np.array([0, 5, 17, 2999, 1234], dtype=np.int32)
    for h in [1, 2, 3]:
        assert (oracle.hdegree_list(g, h, v) == oracle.hdegrees(g, h)[v]).all()


# ---------------------------------------------------------------- core index

def test_core_closed_forms():
    for n in [2, 4, 7]:
        for h in [1, 2, 3]:
            assert (oracle.peel(gg.complete(n), h) == n - 1).all()
    for n in [4, 9]:
        assert (oracle.peel(gg.star(n), 1) == 1).all()
        for h in [2, 3]:
            assert (oracle.peel(gg.star(n), h) == n - 1).all()
    for n in [7, 10, 13]:
        for h in [1, 2, 3]:
            want = 2 * h if 2 * h < n else n - 1
            assert (oracle.peel(gg.cycle(n), h) == want).all(), (n, h)
    for n in [2, 6, 9]:
        for h in [1, 2, 3]:
            assert (oracle.peel(gg.path(n), h) == min(h, n - 1)).all(), (n, h)
    for a, b in [(2, 3), (3, 5)]:
        assert (oracle.peel(gg.complete_bipartite(a, b), 1) == min(a, b)).all()
        assert (oracle.peel(gg.complete_bipartite(a, b), 2) == a + b - 1).all()
    assert (oracle.peel(gg.empty(5), 2) == 0).all()


def test_core_disjoint_union_is_per_component():
    parts = [gg.cycle(9), gg.complete(4), gg.star(5), gg.erdos_renyi_gnm(30, 60, 3)]
    u = gg.disjoint_union(*parts)
    for h in [1, 2, 3]:
        want = np.concatenate([oracle.peel(p, h) for p in parts])
        assert (oracle.peel(u, h) == want).all()


@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_peel_matches_bruteforce_random(h):
    for g in small_graphs(100 + h, 15, (3, 13)):
        assert (oracle.peel(g, h) == oracle.bruteforce(g, h)).all(), g.name


def test_peel_matches_bruteforce_all_graphs_n5():
    n = 5
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        e = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        g = gg.from_edge_list(n, e) if e else gg.empty(n)
        for h in (1, 2, 3):
            assert (oracle.peel(g, h) == oracle.bruteforce(g, h)).all(), (mask, h)


def test_h1_equals_classic_kcore():
    nx = pytest.importorskip("networkx")
    for g in small_graphs(200, 9, (20, 400)) + [gg.chung_lu(2000, 10, 2.5, 300, 4)]:
        c1 = oracle.peel(g, 1)
        assert (c1 == oracle.kcore_bz(g)).all()
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        G.add_edges_from(g.edges().tolist())
        cn = nx.core_number(G)
        assert all(cn[v] == c1[v] for v in range(g.n)), g.name


def test_invariants_monotone_bounded_equivariant():
    for g in small_graphs(300, 9, (10, 120)):
        prev = None
        for h in [1, 2, 3, 4]:
            c = oracle.peel(g, h)
            d = oracle.hdegrees(g, h)
            assert (c <= d).all()
            if prev is not None:
                assert (c >= prev).all(), "core_h <= core_{h+1}"
            prev = c
        perm = np.argsort(gg.Stream(5, g.name).u64(g.n), kind="stable")
        gp = gg.relabel(g, perm)
        c2 = oracle.peel(g, 2)
        assert (oracle.peel(gp, 2)[perm] == c2).all()


def test_h_at_least_diameter_gives_component_size_minus_one():
    from scipy.sparse.csgraph import connected_components
    for g in small_graphs(400, 6, (5, 40)):
        src = np.repeat(np.arange(g.n), g.degrees())
        A = sp.csr_matrix((np.ones(len(g.col)), (src, g.col)), shape=(g.n, g.n))
        _, lab = connected_components(A, directed=False)
        size = np.bincount(lab)[lab]
        assert (oracle.peel(g, g.n) == size - 1).all()


# ---------------------------------------------------------------- certificate

def test_certificate_accepts_true_and_rejects_mutations():
    for g in small_graphs(500, 6, (10, 80)):
        for h in [1, 2, 3]:
            c = oracle.peel(g, h)
            r = oracle.level_rounds(g, h, c)
            fails, _ = oracle.certificate(g, h, c, r)
            assert fails == 0, (g.name, h)
            if g.n < 2:
                continue
            v = int(np.argmax(c))
            for delta in (+1, -1):
                c2 = c.copy()
                c2[v] += delta
                if c2[v] < 0:
                    continue
                assert oracle.certificate(g, h, c2, r)[0] > 0
            # shifting the latest round earlier breaks it too
            late = int(np.argmax(r))
            if r[late] > 0 and (r == r[late]).sum() == 1 and (c == c[late]).sum() < g.n:
                r2 = r.copy()
                r2[late] = 0
                c2 = c.copy()
                assert oracle.certificate(g, h, c2, r2)[0] > 0


def _mutations(c, r, seed):
    """Claimed (core, round) pairs that are wrong in the ways a kernel could
    be: one value off by one, a uniform shift, a random vertex's round moved,
    two vertices' cores swapped."""
    rng = np.random.default_rng(seed)
    out = []
    v = int(rng.integers(len(c)))
    for delta in (+1, -1):
        c2 = c.copy()
        c2[v] = max(0, c2[v] + delta)
        out.append((c2, r))
    out.append((c + 1, r))
    out.append((np.maximum(c - 1, 0), r))
    r2 = r.copy()
    r2[v] = int(rng.integers(r.max() + 1))
    out.append((c, r2))
    a, b = rng.integers(len(c), size=2)
    c3 = c.copy()
    c3[a], c3[b] = c3[b], c3[a]
    out.append((c3, r))
    return out


# both paths of certificate_all: every vertex by its own early-stopped BFS
# (small_cap large), every vertex bit-parallel (small_cap -1) with one-word
# and two-word batches (several batches, a ragged last one), and a mix
PATHS = [(10 ** 9, 8), (-1, 1), (-1, 2), (3, 1)]


def test_certificate_all_agrees_with_per_vertex_certificate():
    # the all-vertex check makes the same per-vertex decisions as the plain
    # per-vertex one, on true results and on every mutation, on every path
    for i, g in enumerate(small_graphs(510, 9, (8, 150))):
        for h in [1, 2, 3, 4]:
            c = oracle.peel(g, h)
            r = oracle.level_rounds(g, h, c)
            for cap, w in PATHS:
                assert oracle.certificate_all(g, h, c, r, cap, w)[0] == 0, (g.name, h, cap, w)
            for c2, r2 in _mutations(c, r, 100 * i + h):
                fp, bp = oracle.certificate(g, h, c2, r2)
                for cap, w in PATHS:
                    fa, ba = oracle.certificate_all(g, h, c2, r2, cap, w)
                    assert fa == fp and np.array_equal(ba, bp), (g.name, h, cap, w)
                if not (np.array_equal(c2, c)):
                    assert fp > 0, (g.name, h)


def test_certificate_all_on_a_chung_lu_graph_with_hubs():
    # hubs make long rows and large balls: the early stop must not change a
    # decision
    g = gg.chung_lu(1500, 8.0, 2.3, 200.0, 91)
    for h in (2, 3):
        c = oracle.peel(g, h)
        r = oracle.level_rounds(g, h, c)
        c2 = c.copy()
        top = np.flatnonzero(c == c.max())
        c2[top[0]] += 1
        fp, bp = oracle.certificate(g, h, c2, r)
        assert fp > 0
        for cap, w in PATHS + [(int(np.median(c)), 4)]:
            assert oracle.certificate_all(g, h, c, r, cap, w)[0] == 0
            fa, ba = oracle.certificate_all(g, h, c2, r, cap, w)
            assert fa == fp and np.array_equal(ba, bp)


def test_certificate_rejects_uniform_shift():
    g = gg.erdos_renyi_gnm(60, 150, 12)
    c = oracle.peel(g, 2)
    r = oracle.level_rounds(g, 2, c)
    assert oracle.certificate(g, 2, c + 1, r)[0] > 0
    assert oracle.certificate(g, 2, np.maximum(c - 1, 0), r)[0] > 0


def test_hdegree_list_scanned_edges_closed_form():
    # a BFS to radius h scans the rows of every vertex at distance < h
    g = gg.path(10)
    d, sc = oracle.hdegree_list(g, 2, [0, 5], return_scanned=True)
    assert list(d) == [2, 4]
    assert list(sc) == [1 + 2, 2 + 2 + 2]
    s = gg.star(8)
    d, sc = oracle.hdegree_list(s, 2, [0, 3], return_scanned=True)
    assert list(d) == [7, 7] and list(sc) == [7 + 7 * 1, 1 + 7]


def test_peel_bounded_is_a_prefix_of_the_full_peel():
    g = gg.erdos_renyi_gnm(300, 900, 21)
    core, order = oracle.peel(g, 2, return_order=True)
    r, c2, o2 = oracle.peel_bounded(g, 2, 57)
    assert r == 57 and (o2[:57] == order[:57]).all() and (c2[o2[:57]] == core[order[:57]]).all()
    r, c3, o3 = oracle.peel_bounded(g, 2, -1, deg_init=oracle.hdegrees(g, 2))
    assert r == g.n and (c3 == core).all()


# ------------------------------------------- the paper's update (Alg. 2-4)

def test_bitmap_update_reproduces_table1(fig1):
    """Sec. IV-B, Table 1 and Example 3: labels, and every bitmap after the
    initialisation and after each of the two DP iterations, for v5 in
    G - {v1, v2, v3} at h = 2; then the update equals a fresh BFS."""
    g, vals = fig1
    alive = np.ones(g.n, np.uint8)
    alive[[0, 1, 2]] = 0
    deg = oracle.hdegrees(g, 2, alive)
    new, labels, trace = oracle.bitmap_update(g, 2, 4, deg, alive, trace_cap=64)
    assert list(labels + 1) == [int(x) for x in vals["table1_labels"]]
    for t, key in enumerate(["table1_init", "table1_iter1", "table1_iter2"]):
        assert list(trace[t]) == [int(x) for x in vals[key]], key
    after = alive.copy()
    after[4] = 0
    fresh = oracle.hdegrees(g, 2, after)
    assert (new[labels] == fresh[labels]).all()


def test_bitmap_update_reproduces_example2(fig1):
    """Sec. IV-A, Example 2: deleting v1 at h = 2 leaves d^2 = 3, 3, 7, 7 for
    v2, v3, v4, v6."""
    g, vals = fig1
    deg = oracle.hdegrees(g, 2)
    new, _, _ = oracle.bitmap_update(g, 2, 0, deg)
    for item in vals["after_v1_hdeg2"]:
        v, want = item.split(":")
        assert new[int(v) - 1] == int(want)


@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_bitmap_update_equals_bfs_after_one_deletion(h):
    """Observation 2 / Theorem 1: the DP on the ball's induced subgraph gives
    exactly the h-degrees of G[alive] - v, on random alive subsets, including
    balls of more than 64 members (several bitmap words)."""
    rng = gg.Stream(500 + h, "bitmap")
    graphs = small_graphs(600 + h, 8, (2, 60)) + [gg.chung_lu(400, 6.0, 2.3, 80.0, 31 + h), gg.star(150)]
    for g in graphs:
        for _ in range(4):
            alive = (rng.uniform(g.n) < 0.85).astype(np.uint8)
            cand = np.nonzero(alive)[0]
            if len(cand) == 0:
                continue
            v = int(cand[rng.below(len(cand), 1)[0]])
            deg = oracle.hdegrees(g, h, alive)
            new, _, _ = oracle.bitmap_update(g, h, v, deg, alive)
            after = alive.copy()
            after[v] = 0
            fresh = oracle.hdegrees(g, h, after)
            keep = after.astype(bool)
            assert (new[keep] == fresh[keep]).all(), (g.name, h, v)


@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_peel_bitmap_equals_algorithm1_and_bruteforce(h):
    """Algorithm 2 with the bitmap update gives Algorithm 1's core indices,
    and the definition's on tiny graphs."""
    for g in small_graphs(700 + h, 10, (2, 80)):
        assert (oracle.peel_bitmap(g, h) == oracle.peel(g, h)).all(), (g.name, h)
    for g in small_graphs(800 + h, 6, (2, 11)):
        assert (oracle.peel_bitmap(g, h) == oracle.bruteforce(g, h)).all(), (g.name, h)


# ------------------------------------------------ sampling variant (Alg. 5-6)

def _sampling_example():
    import os
    from conftest import GOLDEN
    rows = []
    with open(os.path.join(GOLDEN, "sampling_example.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, rate, sel, want = line.split()
            num, den = (int(x) for x in rate.split("/"))
            rows.append((key, num, den, int(sel), int(want)))
    return rows


def test_sampled_estimator_matches_the_papers_example():
    """Sec. IV-C example: select / rate, rounded down (rate = num/den, so the
    estimate of a vertex with select0 = num sampled among d0 = den is
    floor(select * den / num))."""
    for key, num, den, sel, want in _sampling_example():
        assert oracle.sampled_estimate(sel, num, den) == want, key


@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_sampling_with_every_vertex_sampled_is_exact(h):
    """With S = V every rate is 1 and Algorithm 6 reduces to Algorithm 4
    (which needs the <= h - s reading): the estimates are the exact h-degrees
    and the cores are Algorithm 1's."""
    for g in small_graphs(900 + h, 8, (2, 70)) + [gg.chung_lu(300, 6.0, 2.3, 60.0, 41 + h)]:
        core, est = oracle.peel_sampled(g, h, np.ones(g.n, np.uint8))
        assert (est == oracle.hdegrees(g, h)).all(), (g.name, h)
        assert (core == oracle.peel(g, h)).all(), (g.name, h)


def test_sampling_estimates_track_the_exact_cores():
    """On a 2,000-vertex Chung-Lu graph at h = 2 the estimated cores stay
    within 10 % of the exact ones on average, the error shrinks as the sample
    grows (20 % against 95 % of the vertices), and the full sample is exact."""
    g = gg.chung_lu(2000, 8.0, 2.5, 150.0, 51)
    exact = oracle.peel(g, 2)
    u = gg.Stream(52, "sample").uniform(g.n)
    err = {}
    for r in (0.2, 0.95, 1.0):
        core, _ = oracle.peel_sampled(g, 2, (u < r).astype(np.uint8))
        err[r] = np.abs(core - exact).mean() / exact.mean()
    assert err[0.2] < 0.1 and err[0.95] < err[0.2] and err[1.0] == 0.0


@pytest.mark.parametrize("h", [1, 2, 3])
def test_sampling_vertices_without_a_sampled_neighbour_stay_exact(h):
    """A component with no sampled vertex has no rate anywhere: its vertices
    keep their exact h-degrees, so its estimated cores are Algorithm 1's; a
    fully sampled component beside it is exact too (rate 1)."""
    a, b = gg.chung_lu(150, 5.0, 2.3, 40.0, 61 + h), gg.erdos_renyi_gnm(120, 400, 62 + h)
    g = gg.disjoint_union(a, b)
    in_s = np.concatenate([np.zeros(a.n, np.uint8), np.ones(b.n, np.uint8)])
    core, est = oracle.peel_sampled(g, h, in_s)
    assert (core[: a.n] == oracle.peel(a, h)).all()
    assert (core[a.n:] == oracle.peel(b, h)).all()
    assert (est == oracle.hdegrees(g, h)).all()


def test_sampled_cores_are_order_free():
    """Each estimate is a monotone function of the surviving vertex set, so
    the level-by-level peel gives the same estimated cores whatever the order
    of deletions inside a level: relabelling the vertices (which changes the
    order Algorithm 2 takes them in) permutes the result and nothing else."""
    g = gg.chung_lu(400, 6.0, 2.4, 60.0, 63)
    in_s = (gg.Stream(64, "sample").uniform(g.n) < 0.3).astype(np.uint8)
    core, _ = oracle.peel_sampled(g, 2, in_s)
    perm = np.argsort(gg.Stream(65, "perm").u64(g.n), kind="stable")
    g2 = gg.relabel(g, perm)
    s2 = np.zeros(g.n, np.uint8)
    s2[perm] = in_s
    core2, _ = oracle.peel_sampled(g2, 2, s2)
    assert (core2[perm] == core).all()
