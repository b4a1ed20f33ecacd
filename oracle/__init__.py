"""CPU oracle for (k,h)-core decomposition — TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this
package. It wraps oracle.c (plain C, compiled here with gcc) through ctypes and
shares nothing with the CUDA library in paper_2006_03372_gb300.

Functions (each follows the passage named in oracle.c):
  hdegrees(g, h, alive=None)          d_v^h(G[alive]) for every v   (Sec. II)
  hdegree_list(g, h, verts, alive)    the same for a list of vertices
  peel(g, h)                          Algorithm 1, plain peeling     (Sec. III)
  bruteforce(g, h)                    Definition 2 by exhaustion, n <= 20
  kcore_bz(g)                         h = 1: Batagelj-Zaversnik k-core (Sec. II)
  certificate(g, h, core, rnd, verts) exactness certificate for a claimed
                                      core index and peel round
  certificate_all(g, h, core, rnd)    the same on every vertex, early-stopped
                                      BFS (full-size graphs)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        lib.orc_hdegrees.argtypes = [i32, P, P, P, i32, P]
        lib.orc_hdegrees.restype = ctypes.c_int
        lib.orc_hdegree_list.argtypes = [i32, P, P, P, i32, i64, P, P, P]
        lib.orc_hdegree_list.restype = ctypes.c_int
        lib.orc_peel.argtypes = [i32, P, P, i32, P, P]
        lib.orc_peel.restype = ctypes.c_int
        lib.orc_peel_bounded.argtypes = [i32, P, P, i32, P, i64, P, P]
        lib.orc_peel_bounded.restype = ctypes.c_int64
        lib.orc_bruteforce.argtypes = [i32, P, i32, P]
        lib.orc_bruteforce.restype = ctypes.c_int
        lib.orc_kcore_bz.argtypes = [i32, P, P, P]
        lib.orc_kcore_bz.restype = ctypes.c_int
        lib.orc_certificate.argtypes = [i32, P, P, i32, P, P, i64, P, P]
        lib.orc_certificate.restype = ctypes.c_int64
        lib.orc_certificate_all.argtypes = [i32, P, P, i32, P, P, i32, i32, P]
        lib.orc_certificate_all.restype = ctypes.c_int64
        lib.orc_bitmap_update.argtypes = [i32, P, P, P, i32, i32, P, P, i64, P]
        lib.orc_bitmap_update.restype = ctypes.c_int64
        lib.orc_peel_bitmap.argtypes = [i32, P, P, i32, P, P]
        lib.orc_peel_bitmap.restype = ctypes.c_int
        lib.orc_peel_sampled.argtypes = [i32, P, P, i32, P, P, P]
        lib.orc_peel_sampled.restype = ctypes.c_int
        lib.orc_sampled_estimate.argtypes = [i64, i64, i64]
        lib.orc_sampled_estimate.restype = i32
        lib.orc_has_openmp.argtypes = []
        lib.orc_has_openmp.restype = ctypes.c_int
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    return rp, col


def _alive(alive, n):
    if alive is None:
        return None
    a = np.ascontiguousarray(alive, dtype=np.uint8)
    assert a.shape == (n,)
    return a


def threads() -> int:
    """OpenMP threads the oracle uses (0 when built without OpenMP)."""
    return _load().orc_has_openmp()


def hdegrees(g, h: int, alive=None) -> np.ndarray:
    lib = _load()
    rp, col = _csr(g)
    out = np.zeros(max(g.n, 1), dtype=np.int32)
    al = _alive(alive, g.n)
    if lib.orc_hdegrees(g.n, _p(rp), _p(col), _p(al), int(h), _p(out)) != 0:
        raise MemoryError("oracle: out of memory")
    return out[: g.n]


def hdegree_list(g, h: int, verts, alive=None, return_scanned: bool = False):
    """d_v^h for the listed vertices; with return_scanned also the number of
    CSR entries each BFS scanned (sum of deg(x) over x at distance < h)."""
    lib = _load()
    rp, col = _csr(g)
    v = np.ascontiguousarray(verts, dtype=np.int32)
    out = np.zeros(max(len(v), 1), dtype=np.int32)
    sc = np.zeros(max(len(v), 1), dtype=np.int64)
    al = _alive(alive, g.n)
    if lib.orc_hdegree_list(g.n, _p(rp), _p(col), _p(al), int(h), len(v), _p(v), _p(out), _p(sc)) != 0:
        raise MemoryError("oracle: out of memory")
    if return_scanned:
        return out[: len(v)], sc[: len(v)]
    return out[: len(v)]


def peel(g, h: int, return_order: bool = False):
    lib = _load()
    rp, col = _csr(g)
    core = np.zeros(max(g.n, 1), dtype=np.int32)
    order = np.zeros(max(g.n, 1), dtype=np.int32)
    rc = lib.orc_peel(g.n, _p(rp), _p(col), int(h), _p(core), _p(order))
    if rc != 0:
        raise RuntimeError(f"oracle peel failed ({rc})")
    if return_order:
        return core[: g.n], order[: g.n]
    return core[: g.n]


def bitmap_update(g, h: int, v: int, deg, alive=None, trace_cap: int = 0):
    """The paper's update after deleting v from G[alive] (Sec. IV-A/IV-B,
    Algorithms 3 and 4). deg: current h-degrees (copied). Returns (new_deg,
    labels, trace): labels[i] = vertex of u_i (distance from v, then id);
    trace[t][i] = first bitmap word of u_i after the initialisation (t = 0)
    and after hop t, when the ball has at most trace_cap members."""
    lib = _load()
    rp, col = _csr(g)
    d = np.ascontiguousarray(deg, dtype=np.int32).copy()
    a = _alive(alive, g.n)
    cap = max(int(trace_cap), 0)
    tr = np.zeros(max((h + 1) * cap, 1), dtype=np.uint64)
    lab = np.zeros(max(cap, 1), dtype=np.int32)
    nr = lib.orc_bitmap_update(g.n, _p(rp), _p(col), _p(a), int(h), int(v), _p(d), _p(tr) if cap else None,
                               cap, _p(lab) if cap else None)
    if nr < 0:
        raise RuntimeError("oracle bitmap update failed")
    if cap and nr <= cap:
        return d, lab[:nr].copy(), tr[: (h + 1) * nr].reshape(h + 1, nr).copy()
    return d, None, None


def peel_bitmap(g, h: int, return_order: bool = False):
    """The paper's decomposition with the bitmap update (Algorithm 2)."""
    lib = _load()
    rp, col = _csr(g)
    core = np.zeros(max(g.n, 1), dtype=np.int32)
    order = np.zeros(max(g.n, 1), dtype=np.int32)
    if lib.orc_peel_bitmap(g.n, _p(rp), _p(col), int(h), _p(core), _p(order)) != 0:
        raise RuntimeError("oracle bitmap peel failed")
    if return_order:
        return core[: g.n], order[: g.n]
    return core[: g.n]


def peel_sampled(g, h: int, in_s):
    """The sampling variant (Algorithms 5 and 6) with the sample given as a
    0/1 mask: (core estimates, initial h-degree estimates)."""
    lib = _load()
    rp, col = _csr(g)
    s = np.ascontiguousarray(in_s, dtype=np.uint8)
    assert s.shape == (g.n,)
    core = np.zeros(max(g.n, 1), dtype=np.int32)
    est = np.zeros(max(g.n, 1), dtype=np.int32)
    if lib.orc_peel_sampled(g.n, _p(rp), _p(col), int(h), _p(s), _p(core), _p(est)) != 0:
        raise RuntimeError("oracle sampled peel failed")
    return core[: g.n], est[: g.n]


def sampled_estimate(sel: int, sel0: int, d0: int) -> int:
    """select / rate with rate = sel0 / d0, rounded down, in integers."""
    return int(_load().orc_sampled_estimate(int(sel), int(sel0), int(d0)))


def peel_bounded(g, h: int, max_removed: int, deg_init=None):
    """Algorithm 1 stopped after max_removed removals (optionally from given
    initial h-degrees). Returns (removed, core, order); core/order are valid
    for the first `removed` vertices of order."""
    lib = _load()
    rp, col = _csr(g)
    core = np.full(max(g.n, 1), -1, dtype=np.int32)
    order = np.full(max(g.n, 1), -1, dtype=np.int32)
    d = None if deg_init is None else np.ascontiguousarray(deg_init, dtype=np.int32)
    r = lib.orc_peel_bounded(g.n, _p(rp), _p(col), int(h), _p(d), int(max_removed), _p(core), _p(order))
    if r < 0:
        raise MemoryError("oracle: out of memory")
    return int(r), core[: g.n], order[: g.n]


def adjacency_masks(g) -> np.ndarray:
    adj = np.zeros(max(g.n, 1), dtype=np.uint32)
    for v in range(g.n):
        for u in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]:
            adj[v] |= np.uint32(1) << np.uint32(int(u))
    return adj


def bruteforce(g, h: int) -> np.ndarray:
    if g.n > 20:
        raise ValueError("bruteforce is for n <= 20")
    lib = _load()
    adj = adjacency_masks(g)
    core = np.zeros(max(g.n, 1), dtype=np.int32)
    if lib.orc_bruteforce(g.n, _p(adj), int(h), _p(core)) != 0:
        raise RuntimeError("oracle bruteforce failed")
    return core[: g.n]


def kcore_bz(g) -> np.ndarray:
    lib = _load()
    rp, col = _csr(g)
    core = np.zeros(max(g.n, 1), dtype=np.int32)
    if lib.orc_kcore_bz(g.n, _p(rp), _p(col), _p(core)) != 0:
        raise MemoryError("oracle: out of memory")
    return core[: g.n]


def certificate(g, h: int, core, rnd, verts=None):
    """Returns (failures, per-vertex bad mask). verts=None checks every vertex."""
    lib = _load()
    rp, col = _csr(g)
    c = np.ascontiguousarray(core, dtype=np.int32)
    r = np.ascontiguousarray(rnd, dtype=np.int32)
    v = np.arange(g.n, dtype=np.int32) if verts is None else np.ascontiguousarray(verts, dtype=np.int32)
    bad = np.zeros(max(len(v), 1), dtype=np.int32)
    rc = lib.orc_certificate(g.n, _p(rp), _p(col), int(h), _p(c), _p(r), len(v), _p(v), _p(bad))
    if rc == -1:
        raise MemoryError("oracle: out of memory")
    if rc == -2:
        raise ValueError("negative core or round value")
    return int(rc), bad[: len(v)]


def certificate_all(g, h: int, core, rnd, small_cap: int = 1024, words: int = 8):
    """The certificate of `certificate` on every vertex (full-size graphs):
    vertices with core <= small_cap by one early-stopped BFS each, the others
    by a bit-parallel BFS of 64*words sources. Returns (failures, per-vertex
    bad mask: 1 = (i) failed, 2 = (ii) failed)."""
    lib = _load()
    rp, col = _csr(g)
    c = np.ascontiguousarray(core, dtype=np.int32)
    r = np.ascontiguousarray(rnd, dtype=np.int32)
    bad = np.zeros(max(g.n, 1), dtype=np.int32)
    rc = lib.orc_certificate_all(g.n, _p(rp), _p(col), int(h), _p(c), _p(r), int(small_cap), int(words),
                                  _p(bad))
    if rc == -1:
        raise MemoryError("oracle: out of memory")
    if rc == -2:
        raise ValueError("negative core or round value")
    return int(rc), bad[: g.n]


def level_rounds(g, h: int, core):
    """Peel rounds implied by level-synchronous deletion of a known core index:
    replays 'delete every alive vertex with d^h <= k' with this oracle's own
    BFS. Used only to build certificate inputs in oracle self-tests."""
    n = g.n
    alive = np.ones(n, dtype=np.uint8)
    rnd = np.full(n, -1, dtype=np.int32)
    k = 0
    r = 0
    while alive.any():
        d = hdegrees(g, h, alive)
        k = max(k, int(d[alive.astype(bool)].min()))
        D = np.flatnonzero(alive.astype(bool) & (d <= k))
        rnd[D] = r
        alive[D] = 0
        r += 1
    return rnd
