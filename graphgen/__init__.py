"""Seeded synthetic graph generators shared by the oracle tests and the CUDA path.

This module holds input recipes only: random numbers, graph shapes and CSR
assembly. It computes nothing of the (k,h)-core method itself (no distances,
no h-hop degrees, no peeling), so both sides of every parity test can take
their inputs from here without sharing any of the method's arithmetic.

Random numbers come from one counter-based generator, SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): output i of a stream with state s0 is mix(s0 + (i+1)*GOLDEN).
It is written out here in numpy so the streams are identical on every machine
and every numpy version.

All graphs are simple and undirected (Sec. II): the CSR holds both directions
of every edge, no self-loops and no duplicates, rows sorted by neighbour id.
Isolated vertices are kept.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _mix_scalar(x: int) -> int:
    x &= _MASK64
    x ^= x >> 30
    x = (x * 0xBF58476D1CE4E5B9) & _MASK64
    x ^= x >> 27
    x = (x * 0x94D049BB133111EB) & _MASK64
    x ^= x >> 31
    return x


class Stream:
    """A SplitMix64 stream keyed by (seed, tag); draws are taken in order."""

    def __init__(self, seed: int, tag: str = ""):
        key = seed & _MASK64
        for ch in tag.encode():
            key = _mix_scalar(key ^ ch)
        self.state = np.uint64(_mix_scalar(key))
        self.counter = 0

    def u64(self, count: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + 1 + count, dtype=np.uint64)
        self.counter += count
        with np.errstate(over="ignore"):
            return _mix(self.state + idx * _GOLDEN)

    def uniform(self, count: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def below(self, bound: int, count: int) -> np.ndarray:
        """Integers in [0, bound) (modulo reduction; bias < bound / 2**64)."""
        return (self.u64(count) % np.uint64(bound)).astype(np.int64)


@dataclass
class Graph:
    """An undirected simple graph as an int32 CSR holding both edge directions."""

    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col: np.ndarray      # int32[row_ptr[n]]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m_directed(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        return self.m_directed // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def edges(self) -> np.ndarray:
        """Each undirected edge once, as an (m, 2) int64 array with u < v."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        dst = self.col.astype(np.int64)
        keep = src < dst
        return np.stack([src[keep], dst[keep]], axis=1)


def csr_from_pairs(n: int, a: np.ndarray, b: np.ndarray, name: str = "", meta=None) -> Graph:
    """Symmetrise, drop self-loops and duplicates, and build a sorted int32 CSR."""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    keep = a != b
    a, b = a[keep], b[keep]
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    und = np.unique(lo * n + hi)
    lo, hi = und // n, und % n
    src = np.concatenate([lo, hi])
    dst = np.concatenate([hi, lo])
    key = np.sort(src * n + dst)
    src, dst = key // n, key % n
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("graph too large for an int32 CSR")
    return Graph(n, row_ptr.astype(np.int32), dst.astype(np.int32), name, dict(meta or {}))


def from_edge_list(n: int, edges, name: str = "") -> Graph:
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    return csr_from_pairs(n, e[:, 0], e[:, 1], name)


# ---------------------------------------------------------------------------
# Generators
# ---------------------------------------------------------------------------

def erdos_renyi_gnm(n: int, m: int, seed: int) -> Graph:
    """G(n, m): exactly m distinct edges drawn uniformly, no loops."""
    if m > n * (n - 1) // 2:
        raise ValueError("m exceeds the number of vertex pairs")
    rng = Stream(seed, "gnm")
    keys = np.empty(0, dtype=np.int64)
    order = np.empty(0, dtype=np.int64)
    drawn = 0
    while True:
        need = m - len(keys)
        if need <= 0:
            break
        c = int(need * 1.2) + 64
        u = rng.below(n, c)
        v = rng.below(n, c)
        ok = u != v
        lo = np.minimum(u, v)[ok]
        hi = np.maximum(u, v)[ok]
        k = lo * n + hi
        allk = np.concatenate([keys, k])
        allo = np.concatenate([order, drawn + np.arange(len(k), dtype=np.int64)])
        drawn += len(k)
        uk, first = np.unique(allk, return_index=True)
        sel = np.argsort(allo[first], kind="stable")
        keys, order = uk[sel], allo[first][sel]
    keys = keys[:m]
    return csr_from_pairs(n, keys // n, keys % n, f"er_n{n}_m{m}_s{seed}",
                          dict(kind="er", n=n, m_target=m, seed=seed))


def chung_lu_weights(n: int, mean_deg: float, gamma: float, max_deg: float) -> np.ndarray:
    """Expected degrees w_i = c * (i + i0)^(-1/(gamma-1)), with c and i0 chosen so
    that the mean is mean_deg and the largest weight is max_deg."""
    beta = 1.0 / (gamma - 1.0)
    i = np.arange(n, dtype=np.float64)

    def mean_for(i0):
        w = (i + i0) ** (-beta)
        return max_deg * w.mean() / w[0]

    lo, hi = 1e-9, float(n) * 1e3
    if mean_for(hi) < mean_deg:
        hi_mean = mean_for(hi)
        raise ValueError(f"mean degree {mean_deg} unreachable (max {hi_mean:.3f})")
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if mean_for(mid) < mean_deg:
            lo = mid
        else:
            hi = mid
    i0 = math.sqrt(lo * hi)
    w = (i + i0) ** (-beta)
    return w * (max_deg / w[0])


def chung_lu(n: int, mean_deg: float, gamma: float, max_deg: float, seed: int,
             tag: str = "cl") -> Graph:
    """Chung-Lu power-law graph: n*mean_deg/2 endpoint pairs, each endpoint drawn
    with probability proportional to its expected degree; loops and duplicate
    edges are dropped, so m comes out slightly below the target."""
    w = chung_lu_weights(n, mean_deg, gamma, max_deg)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    m_target = int(round(n * mean_deg / 2))
    rng = Stream(seed, tag)
    a = np.searchsorted(cdf, rng.uniform(m_target), side="right")
    b = np.searchsorted(cdf, rng.uniform(m_target), side="right")
    a = np.minimum(a, n - 1)
    b = np.minimum(b, n - 1)
    # vertex ids are shuffled so that the hubs are not all at the low ids
    perm = np.argsort(rng.u64(n), kind="stable")
    return csr_from_pairs(n, perm[a], perm[b], f"cl_n{n}_d{mean_deg}_g{gamma}_s{seed}",
                          dict(kind="chung_lu", n=n, mean_deg=mean_deg, gamma=gamma,
                               max_deg=max_deg, seed=seed, m_target=m_target))


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, d: float,
         seed: int) -> Graph:
    """R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): each of
    edge_factor * 2^scale edges picks one quadrant per level with probabilities
    (a, b, c, d); the result is symmetrised and deduplicated."""
    n = 1 << scale
    e = edge_factor * n
    rng = Stream(seed, "rmat")
    src = np.zeros(e, dtype=np.int64)
    dst = np.zeros(e, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for lvl in range(scale):
        u = rng.uniform(e)
        bit = np.int64(1) << np.int64(scale - 1 - lvl)
        right = ((u >= a) & (u < ab)) | (u >= abc)   # quadrants b and d
        down = u >= ab                                # quadrants c and d
        src += np.where(down, bit, 0)
        dst += np.where(right, bit, 0)
    return csr_from_pairs(n, src, dst, f"rmat_s{scale}_ef{edge_factor}_s{seed}",
                          dict(kind="rmat", scale=scale, edge_factor=edge_factor,
                               abcd=(a, b, c, d), seed=seed))


# ---------------------------------------------------------------------------
# Named workloads (the five configurations) and small families used by tests
# ---------------------------------------------------------------------------

def config1_er() -> Graph:
    """Erdos-Renyi G(n=2000, m=8000), seed 1 (decomposed at h=2)."""
    return erdos_renyi_gnm(2000, 8000, 1)


def config2_chung_lu(n: int = 1_000_000, mean_deg: float = 20.0) -> Graph:
    """Chung-Lu n=1e6, m~1e7 (mean degree 20), exponent 2.5, max expected degree
    1e4, seed 2 (decomposed at h=2 and h=3). Smaller n gives the same recipe."""
    return chung_lu(n, mean_deg, 2.5, min(10_000.0, n - 1.0), 2)


def config3_rmat(scale: int = 18) -> Graph:
    """R-MAT scale 18, edge factor 16, (0.57, 0.19, 0.19, 0.05), seed 3
    (decomposed at h=4 and h=5)."""
    return rmat(scale, 16, 0.57, 0.19, 0.19, 0.05, 3)


@dataclass
class BatchSpec:
    ns: np.ndarray        # vertex counts
    kinds: list           # "er" or "cl"
    hs: np.ndarray        # h per graph
    seeds: np.ndarray     # per-graph generator seeds


def config4_spec(count: int = 1024, n_lo: int = 500, n_hi: int = 100_000, seed: int = 4) -> BatchSpec:
    """1024 graphs, n log-uniform in [500, 1e5], exactly half ER (mean degree 6)
    and half Chung-Lu (exponent 2.3, mean degree 6, max expected degree
    sqrt(6 n)), order shuffled, h uniform in {2,3,4}."""
    rng = Stream(seed, "batch")
    u = rng.uniform(count)
    ns = np.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo))).round().astype(np.int64)
    kinds = np.array(["er"] * (count // 2) + ["cl"] * (count - count // 2))
    kinds = kinds[np.argsort(rng.u64(count), kind="stable")]
    hs = 2 + rng.below(3, count)
    seeds = (rng.u64(count) >> np.uint64(1)).astype(np.int64)
    return BatchSpec(ns, list(kinds), hs, seeds)


def batch_graph(spec: BatchSpec, i: int) -> Graph:
    n = int(spec.ns[i])
    if spec.kinds[i] == "er":
        m = min(3 * n, n * (n - 1) // 2)
        return erdos_renyi_gnm(n, m, int(spec.seeds[i]))
    return chung_lu(n, 6.0, 2.3, math.sqrt(6.0 * n), int(spec.seeds[i]))


@dataclass
class Request:
    arrival_s: float
    n: int
    mean_deg: float
    h: int
    seed: int


def config5_requests(rate: float = 200.0, duration_s: float = 60.0, seed: int = 5,
                     n_lo: int = 1000, n_hi: int = 500_000) -> list:
    """Open-loop Poisson arrivals; each request a Chung-Lu graph (exponent 2.5)
    with n log-uniform in [1e3, 5e5], mean degree uniform in [4, 20], h uniform
    in {2,3,4}."""
    rng = Stream(seed, "serve")
    reqs = []
    t = 0.0
    while True:
        t += -math.log(1.0 - float(rng.uniform(1)[0])) / rate
        if t >= duration_s:
            break
        u = rng.uniform(2)
        n = int(round(math.exp(math.log(n_lo) + u[0] * (math.log(n_hi) - math.log(n_lo)))))
        d = 4.0 + 16.0 * float(u[1])
        h = 2 + int(rng.below(3, 1)[0])
        s = int(rng.u64(1)[0] >> np.uint64(1))
        reqs.append(Request(t, n, d, h, s))
    return reqs


def request_graph(r: Request) -> Graph:
    return chung_lu(r.n, r.mean_deg, 2.5, math.sqrt(r.mean_deg * r.n), r.seed)


# Small deterministic families with known structure (test inputs)

def complete(n: int) -> Graph:
    i, j = np.triu_indices(n, 1)
    return csr_from_pairs(n, i, j, f"K{n}")


def star(n: int) -> Graph:
    return csr_from_pairs(n, np.zeros(n - 1, dtype=np.int64), np.arange(1, n), f"star{n}")


def cycle(n: int) -> Graph:
    i = np.arange(n)
    return csr_from_pairs(n, i, (i + 1) % n, f"C{n}")


def path(n: int) -> Graph:
    i = np.arange(n - 1)
    return csr_from_pairs(n, i, i + 1, f"P{n}")


def complete_bipartite(a: int, b: int) -> Graph:
    i, j = np.meshgrid(np.arange(a), a + np.arange(b), indexing="ij")
    return csr_from_pairs(a + b, i.ravel(), j.ravel(), f"K{a},{b}")


def disjoint_union(*gs: Graph) -> Graph:
    off = 0
    aa, bb = [], []
    for g in gs:
        e = g.edges()
        aa.append(e[:, 0] + off)
        bb.append(e[:, 1] + off)
        off += g.n
    return csr_from_pairs(off, np.concatenate(aa) if aa else np.zeros(0),
                          np.concatenate(bb) if bb else np.zeros(0), "union")


def relabel(g: Graph, perm: np.ndarray) -> Graph:
    """Vertex v of g becomes perm[v]."""
    e = g.edges()
    return csr_from_pairs(g.n, perm[e[:, 0]], perm[e[:, 1]], g.name + "_relabelled")


def empty(n: int) -> Graph:
    return Graph(n, np.zeros(n + 1, dtype=np.int32), np.zeros(0, dtype=np.int32), f"empty{n}")


# ---------------------------------------------------------------------------
# On-disk cache of generated graphs (generation of the 1e6-vertex graph takes
# tens of seconds); keyed by the generator call, stored as .npz.
# ---------------------------------------------------------------------------

def cache_dir() -> str:
    import os
    d = os.environ.get("KHCORE_GRAPH_CACHE", os.path.join("/tmp", "khcore_graphs"))
    os.makedirs(d, exist_ok=True)
    return d


def cached(key: str, make) -> Graph:
    import os
    path = os.path.join(cache_dir(), key + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        return Graph(int(z["n"]), z["row_ptr"], z["col"], key)
    g = make()
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, n=g.n, row_ptr=g.row_ptr, col=g.col)
    os.replace(tmp, path)
    g.name = key
    return g


def profile_chung_lu() -> Graph:
    """The 1M Chung-Lu recipe at n=2e5 (same mean degree, exponent, cap and
    seed): a smaller case of the same kernels for counter captures."""
    return config2_chung_lu(200_000)


CONFIGS = {
    "er2000": (config1_er, (2,)),
    "cl1m": (config2_chung_lu, (2, 3)),
    "rmat18": (config3_rmat, (4, 5)),
    "cl200k": (profile_chung_lu, (2,)),
}


def config_graph(name: str) -> Graph:
    make, _ = CONFIGS[name]
    return cached(name, make)


def config4_packed(count: int = 1024, first: int = None):
    """The batching workload packed for khcore_batch_create: (graphs spec,
    v_off, e_off, row_ptr_local, col_local, h). first=k keeps graphs 0..k-1.
    Cached on disk (generation of all 1024 graphs takes a minute)."""
    import os
    spec = config4_spec(count)
    k = count if first is None else min(first, count)
    path = os.path.join(cache_dir(), f"batch{count}_first{k}.npz")
    if os.path.exists(path):
        z = np.load(path)
        return spec, z["v_off"], z["e_off"], z["rp"], z["col"], z["h"]
    gs = [batch_graph(spec, i) for i in range(k)]
    ns = np.array([g.n for g in gs], dtype=np.int64)
    ms = np.array([len(g.col) for g in gs], dtype=np.int64)
    v_off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    e_off = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
    rp = np.concatenate([g.row_ptr for g in gs]).astype(np.int32)
    col = np.concatenate([g.col for g in gs]).astype(np.int32)
    h = spec.hs[:k].astype(np.int32)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, v_off=v_off, e_off=e_off, rp=rp, col=col, h=h)
    os.replace(tmp, path)
    return spec, v_off, e_off, rp, col, h


def unpack(v_off, e_off, rp, col, i) -> Graph:
    """Graph i of a packed batch."""
    a, b = int(v_off[i]), int(v_off[i + 1])
    ea, eb = int(e_off[i]), int(e_off[i + 1])
    return Graph(b - a, rp[a + i:b + i + 1].copy(), col[ea:eb].copy(), f"batch{i}")
