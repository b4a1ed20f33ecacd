"""The seeded input generators: determinism and simple-graph structure."""
import numpy as np

import graphgen as gg


def _check_simple(g):
    rp, col = g.row_ptr.astype(np.int64), g.col.astype(np.int64)
    assert rp[0] == 0 and (np.diff(rp) >= 0).all() and rp[-1] == len(col)
    src = np.repeat(np.arange(g.n), np.diff(rp))
    assert ((col >= 0) & (col < g.n)).all()
    assert (src != col).all(), "self-loop"
    key = src * g.n + col
    assert (np.diff(key) > 0).all(), "rows sorted, no duplicates"
    rev = np.sort(col * g.n + src)
    assert (rev == key).all(), "symmetric"


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the published first outputs of the sequence
    s = gg.Stream.__new__(gg.Stream)
    s.state = np.uint64(0)
    s.counter = 0
    got = [int(x) for x in s.u64(3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_streams_are_deterministic_and_keyed():
    a = gg.Stream(7, "x").u64(5)
    b = gg.Stream(7, "x").u64(5)
    c = gg.Stream(7, "y").u64(5)
    assert (a == b).all() and not (a == c).all()
    u = gg.Stream(3).uniform(10000)
    assert 0 <= u.min() and u.max() < 1 and abs(u.mean() - 0.5) < 0.02


def test_er_exact_m_and_simple():
    g = gg.erdos_renyi_gnm(500, 2000, 1)
    assert g.m == 2000
    _check_simple(g)
    g2 = gg.erdos_renyi_gnm(500, 2000, 1)
    assert (g.col == g2.col).all()


def test_chung_lu_and_rmat_simple():
    g = gg.chung_lu(5000, 10.0, 2.5, 300.0, 2)
    _check_simple(g)
    assert 0.8 * 25000 < g.m <= 25000
    w = gg.chung_lu_weights(5000, 10.0, 2.5, 300.0)
    assert abs(w.mean() - 10.0) < 1e-6 and abs(w.max() - 300.0) < 1e-6
    r = gg.rmat(10, 8, 0.57, 0.19, 0.19, 0.05, 3)
    _check_simple(r)
    assert r.n == 1024


def test_structured():
    for g in [gg.complete(5), gg.star(6), gg.cycle(7), gg.path(4), gg.complete_bipartite(2, 3),
              gg.disjoint_union(gg.cycle(4), gg.path(3))]:
        _check_simple(g)
    assert gg.complete(5).m == 10 and gg.cycle(7).m == 7


def test_config_specs():
    spec = gg.config4_spec()
    assert len(spec.ns) == 1024 and spec.ns.min() >= 500 and spec.ns.max() <= 100000
    assert spec.kinds.count("er") == 512
    assert set(np.unique(spec.hs)) <= {2, 3, 4}
    reqs = gg.config5_requests(duration_s=5.0)
    assert 700 < len(reqs) < 1300
    assert all(1000 <= r.n <= 500000 and r.h in (2, 3, 4) for r in reqs)
