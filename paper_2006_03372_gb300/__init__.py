"""GB300 (sm_103a) library for distance-generalized (k,h)-core decomposition.

A thin ctypes binding over the C ABI in include/khcore.h. The binding only
marshals arguments: every step of the computation runs in the library's CUDA
kernels (libkhcore.so, built by paper_2006_03372_gb300._build). There is no
CPU fallback: if the library is missing or no GPU is present the calls raise.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); the C library tells host and device pointers apart itself.

    ctx = khcore_create(n, row_ptr, col)          # int32 CSR, both directions
    deg = khcore_hdegrees(ctx, h)                 # d_v^h(G) for all v   (Sec. II)
    core = khcore_decompose(ctx, h)               # core_h(v) for all v  (Sec. II)
    core, rnd, stats = khcore_decompose_ex(ctx, h)
    khcore_destroy(ctx)
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from ._build import LIB as _LIB_PATH
from ._build import build as _build_lib

__all__ = [
    "KHCoreError", "khcore_create", "khcore_hdegrees", "khcore_decompose", "khcore_decompose_ex",
    "khcore_destroy", "khcore_last_error", "khcore_set_words", "khcore_set_profiling",
    "khcore_set_push_alpha", "khcore_set_round_loop", "khcore_set_wait_limit", "khcore_set_round_words", "khcore_set_lazy", "khcore_set_graph_blocks",
    "khcore_status_string", "Stats",
    "KHCore", "library_path", "load_library", "khcore_batch_create", "khcore_batch_decompose", "pack_graphs",
    "khcore_hdegrees_of", "khcore_hdegrees_ex", "khcore_hdegrees_static", "Server", "request_bytes",
    "khcore_set_update", "khcore_bitmap_update", "khcore_decompose_sampled", "khcore_set_degree_classes",
    "khcore_set_block_size", "khcore_set_block_graph_max", "khcore_autotune", "Tuning", "khcore_set_round_blocks",
    "khcore_set_concurrent_graphs", "khcore_set_round_sms",
]

STATUS = {0: "KHCORE_OK", 1: "KHCORE_EINVAL", 2: "KHCORE_ENOMEM", 3: "KHCORE_ECUDA",
          4: "KHCORE_ETIMEOUT", 5: "KHCORE_EBUSY", 6: "KHCORE_EINTERNAL"}
FLAG_TRUST_INPUT = 0x1


class Tuning(ctypes.Structure):
    _fields_ = [("words", ctypes.c_int32), ("block", ctypes.c_int32), ("light_max", ctypes.c_int32),
                ("medium_max", ctypes.c_int32), ("push_alpha", ctypes.c_int32),
                ("block_graph_max", ctypes.c_int32), ("from_cache", ctypes.c_int32), ("trials", ctypes.c_int32),
                ("trial_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KHCoreError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Stats(ctypes.Structure):
    _fields_ = [("h", ctypes.c_int32), ("rounds", ctypes.c_int32), ("k_max", ctypes.c_int32),
                ("words_per_vertex", ctypes.c_int32), ("deleted_total", ctypes.c_int64),
                ("affected_total", ctypes.c_int64), ("source_batches", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("device_ms", ctypes.c_double),
                ("edges_traversed", ctypes.c_int64), ("level_launches", ctypes.c_int64),
                ("level_ms", ctypes.c_double), ("level_bytes", ctypes.c_double),
                ("recomputed_total", ctypes.c_int64), ("init_ms", ctypes.c_double),
                ("round_ms", ctypes.c_double), ("round_bytes", ctypes.c_double),
                ("phase_ms", ctypes.c_double * 5), ("grid_barriers", ctypes.c_int64),
                ("round_words", ctypes.c_int32), ("round_blocks", ctypes.c_int32)]

    def as_dict(self):
        out = {k: getattr(self, k) for k, _ in self._fields_}
        out["phase_ms"] = list(out["phase_ms"])
        return out


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _LIB_PATH


def load_library(build_if_missing: bool = False):
    """Load libkhcore.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            if not build_if_missing:
                raise ImportError(
                    f"libkhcore.so is not built ({_LIB_PATH}); run __graft_entry__.build() or "
                    "python -m paper_2006_03372_gb300._build")
            _build_lib()
        lib = ctypes.CDLL(_LIB_PATH)
        P, i32, u32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64
        lib.khcore_create.argtypes = [i32, P, P, u32, P, ctypes.POINTER(P)]
        lib.khcore_create.restype = ctypes.c_int
        lib.khcore_hdegrees.argtypes = [P, i32, P]
        lib.khcore_hdegrees.restype = ctypes.c_int
        lib.khcore_decompose.argtypes = [P, i32, P]
        lib.khcore_decompose.restype = ctypes.c_int
        lib.khcore_decompose_ex.argtypes = [P, i32, P, P, ctypes.POINTER(Stats)]
        lib.khcore_decompose_ex.restype = ctypes.c_int
        lib.khcore_destroy.argtypes = [P]
        lib.khcore_destroy.restype = None
        lib.khcore_last_error.argtypes = [P]
        lib.khcore_last_error.restype = ctypes.c_char_p
        lib.khcore_status_string.argtypes = [ctypes.c_int]
        lib.khcore_status_string.restype = ctypes.c_char_p
        lib.khcore_set_words.argtypes = [P, i32]
        lib.khcore_set_words.restype = ctypes.c_int
        lib.khcore_set_round_words.argtypes = [P, i32]
        lib.khcore_set_round_words.restype = ctypes.c_int
        lib.khcore_set_push_alpha.argtypes = [P, i32]
        lib.khcore_set_push_alpha.restype = ctypes.c_int
        lib.khcore_set_lazy.argtypes = [P, i32]
        lib.khcore_set_lazy.restype = ctypes.c_int
        lib.khcore_set_graph_blocks.argtypes = [P, i32]
        lib.khcore_set_graph_blocks.restype = ctypes.c_int
        lib.khcore_decompose_sampled.argtypes = [P, i32, P, P, P, ctypes.POINTER(Stats)]
        lib.khcore_decompose_sampled.restype = ctypes.c_int
        lib.khcore_set_degree_classes.argtypes = [P, i32, i32]
        lib.khcore_set_degree_classes.restype = ctypes.c_int
        lib.khcore_set_block_size.argtypes = [P, i32]
        lib.khcore_set_block_size.restype = ctypes.c_int
        lib.khcore_set_concurrent_graphs.argtypes = [P, i32]
        lib.khcore_set_concurrent_graphs.restype = ctypes.c_int
        lib.khcore_set_round_blocks.argtypes = [P, i32]
        lib.khcore_set_round_blocks.restype = ctypes.c_int
        lib.khcore_set_round_sms.argtypes = [P, i32]
        lib.khcore_set_round_sms.restype = ctypes.c_int
        lib.khcore_set_block_graph_max.argtypes = [P, i32]
        lib.khcore_set_block_graph_max.restype = ctypes.c_int
        lib.khcore_autotune.argtypes = [P, i32, ctypes.c_char_p, ctypes.POINTER(Tuning)]
        lib.khcore_autotune.restype = ctypes.c_int
        lib.khcore_set_update.argtypes = [P, i32]
        lib.khcore_set_update.restype = ctypes.c_int
        lib.khcore_bitmap_update.argtypes = [P, i32, P, i32, P, ctypes.POINTER(i64)]
        lib.khcore_bitmap_update.restype = ctypes.c_int
        lib.khcore_set_round_loop.argtypes = [P, i32]
        lib.khcore_set_round_loop.restype = ctypes.c_int
        lib.khcore_set_wait_limit.argtypes = [P, ctypes.c_uint64]
        lib.khcore_set_wait_limit.restype = ctypes.c_int
        lib.khcore_set_profiling.argtypes = [P, i32]
        lib.khcore_set_profiling.restype = ctypes.c_int
        lib.khcore_num_vertices.argtypes = [P]
        lib.khcore_num_vertices.restype = i32
        lib.khcore_num_entries.argtypes = [P]
        lib.khcore_num_entries.restype = i64
        lib.khcore_hdegrees_ex.argtypes = [P, i32, P, P]
        lib.khcore_hdegrees_ex.restype = ctypes.c_int
        lib.khcore_hdegrees_of.argtypes = [P, i32, i32, P, P]
        lib.khcore_hdegrees_of.restype = ctypes.c_int
        lib.khcore_hdegrees_static.argtypes = [i32, i64, P, P, i32, i32, P, P, P]
        lib.khcore_hdegrees_static.restype = ctypes.c_int
        sz = ctypes.c_size_t
        lib.khcore_request_bytes.argtypes = [i32, i64]
        lib.khcore_request_bytes.restype = sz
        lib.khcore_server_create.argtypes = [sz, i32, i32, ctypes.POINTER(P)]
        lib.khcore_server_create.restype = ctypes.c_int
        lib.khcore_server_submit.argtypes = [P, i32, P, P, i32, ctypes.POINTER(ctypes.c_uint64)]
        lib.khcore_server_submit.restype = ctypes.c_int
        lib.khcore_server_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(i32)]
        lib.khcore_server_poll.restype = ctypes.c_int
        lib.khcore_server_wait.argtypes = [P, ctypes.c_uint64, P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
        lib.khcore_server_wait.restype = ctypes.c_int
        lib.khcore_server_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                            ctypes.POINTER(sz)]
        lib.khcore_server_stats.restype = ctypes.c_int
        lib.khcore_server_last_error.argtypes = [P]
        lib.khcore_server_last_error.restype = ctypes.c_char_p
        lib.khcore_server_destroy.argtypes = [P]
        lib.khcore_server_destroy.restype = None
        lib.khcore_num_graphs.argtypes = [P]
        lib.khcore_num_graphs.restype = i32
        lib.khcore_batch_create.argtypes = [i32, P, P, P, P, u32, P, ctypes.POINTER(P)]
        lib.khcore_batch_create.restype = ctypes.c_int
        lib.khcore_batch_decompose.argtypes = [P, P, P, P, ctypes.POINTER(Stats)]
        lib.khcore_batch_decompose.restype = ctypes.c_int
        _lib = lib
        return lib


# ---------------------------------------------------------------- marshalling

def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype=np.int32):
    """(pointer, keepalive) for a numpy array or torch tensor of int32."""
    if a is None:
        return None, None
    if _is_torch(a):
        import torch
        want = torch.uint8 if dtype == np.uint8 else torch.int32
        if a.dtype != want:
            raise TypeError(f"expected a {want} tensor")
        if not a.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return ctypes.c_void_p(a.data_ptr() if a.numel() else 0), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), arr


def _check(lib, ctx, status):
    if status != 0:
        msg = lib.khcore_last_error(ctx)
        raise KHCoreError(status, msg.decode() if msg else "")


class _Ctx(ctypes.c_void_p):
    pass


def khcore_create(n: int, row_ptr, col, flags: int = 0, stream=None):
    """Copy an undirected int32 CSR to the device; returns an opaque context.
    stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
    lib = load_library()
    rp, k1 = _ptr(row_ptr)
    cl, k2 = _ptr(col)
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    out = ctypes.c_void_p()
    st = lib.khcore_create(int(n), rp, cl, int(flags), ctypes.c_void_p(stream) if stream else None,
                           ctypes.byref(out))
    _check(lib, None, st)
    del k1, k2
    return _Ctx(out.value)


def khcore_destroy(ctx) -> None:
    if ctx is not None and ctx.value:
        load_library().khcore_destroy(ctx)
        ctx.value = None


def khcore_last_error(ctx=None) -> str:
    m = load_library().khcore_last_error(ctx)
    return m.decode() if m else ""


def khcore_status_string(status: int) -> str:
    return load_library().khcore_status_string(int(status)).decode()


def khcore_set_words(ctx, words: int) -> None:
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_words(ctx, int(words)))


def khcore_set_round_words(ctx, words: int) -> None:
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_round_words(ctx, int(words)))


def khcore_set_push_alpha(ctx, alpha: int) -> None:
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_push_alpha(ctx, int(alpha)))


def khcore_set_lazy(ctx, on: int) -> None:
    """1 (default): bound-based exact peeling; 0: recompute every inner affected vertex."""
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_lazy(ctx, int(on)))


def khcore_set_graph_blocks(ctx, mode: int) -> None:
    """0: automatic; 1: one thread block per whole graph; -1: grid-wide rounds only."""
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_graph_blocks(ctx, int(mode)))


def khcore_decompose_sampled(ctx, h: int, in_s, core_out=None, round_out=None, want_rounds: bool = True):
    """(estimated core, round, stats) of the sampling variant (Algorithms 5
    and 6) on the caller's sample in_s (uint8[n], 1 = sampled)."""
    lib = load_library()
    core = _out(ctx, core_out)
    rnd = _out(ctx, round_out) if (want_rounds or round_out is not None) else None
    a = np.ascontiguousarray(in_s, dtype=np.uint8) if not _is_torch(in_s) else in_s
    pa, _ = _ptr(a, np.uint8)
    pc, _ = _ptr(core)
    pr, _ = _ptr(rnd)
    stats = Stats()
    _check(lib, ctx, lib.khcore_decompose_sampled(ctx, int(h), pa, pc, pr, ctypes.byref(stats)))
    return core, rnd, stats.as_dict()


def khcore_set_degree_classes(ctx, light_max: int, medium_max: int) -> None:
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_degree_classes(ctx, int(light_max), int(medium_max)))


def khcore_set_block_size(ctx, threads: int) -> None:
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_block_size(ctx, int(threads)))


def khcore_set_concurrent_graphs(ctx, k: int) -> None:
    """Batch contexts: larger graphs decomposed k at a time (own stream each)."""
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_concurrent_graphs(ctx, int(k)))


def khcore_set_round_blocks(ctx, blocks: int) -> None:
    """Resident blocks per SM of the round kernel (0: by h, 1 or 2)."""
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_round_blocks(ctx, int(blocks)))


def khcore_set_round_sms(ctx, sms: int) -> None:
    """SMs the round kernel's grid covers (0: all)."""
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_round_sms(ctx, int(sms)))


def khcore_set_block_graph_max(ctx, nmax: int) -> None:
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_block_graph_max(ctx, int(nmax)))


def khcore_autotune(ctx, h: int, cache_path=None) -> dict:
    """Measure and apply the tuning knobs for this graph, GPU and h (see
    include/khcore.h); returns the chosen values."""
    lib = load_library()
    t = Tuning()
    p = None if cache_path is None else os.fsencode(cache_path)
    _check(lib, ctx, lib.khcore_autotune(ctx, int(h), p, ctypes.byref(t)))
    return t.as_dict()


def khcore_set_update(ctx, mode: int) -> None:
    """0: BFS recompute (default); 1: the paper's per-deletion update (Algorithms 3/4)."""
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_update(ctx, int(mode)))


def khcore_bitmap_update(ctx, h: int, alive, v: int, deg):
    """The paper's update after deleting v from G[alive] (Algorithm 3 with
    Algorithm 4's bitmaps): returns (updated h-degrees, |N_v^h|). alive:
    uint8[n]; deg: int32[n] h-degrees in G[alive] (not modified; a copy is
    returned unless deg is a device tensor, which is updated in place)."""
    lib = load_library()
    a = np.ascontiguousarray(alive, dtype=np.uint8) if not _is_torch(alive) else alive
    d = deg if _is_torch(deg) else np.array(deg, dtype=np.int32, copy=True)
    pa, _ = _ptr(a, np.uint8)
    pd, _ = _ptr(d)
    ball = ctypes.c_int64(0)
    _check(lib, ctx, lib.khcore_bitmap_update(ctx, int(h), pa, int(v), pd, ctypes.byref(ball)))
    return d, int(ball.value)


def khcore_set_round_loop(ctx, mode: int) -> None:
    """0: one persistent kernel per decomposition (default); 1: host-driven rounds."""
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_round_loop(ctx, int(mode)))


def khcore_set_wait_limit(ctx, ns: int) -> None:
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_wait_limit(ctx, int(ns)))


def khcore_set_profiling(ctx, on: int) -> None:
    lib = load_library()
    _check(lib, ctx, lib.khcore_set_profiling(ctx, int(on)))


def _out(ctx, out):
    n = load_library().khcore_num_vertices(ctx)
    if out is None:
        out = np.empty(n, dtype=np.int32)
    elif len(out) != n:
        raise ValueError(f"output has {len(out)} entries, graph has {n} vertices")
    if isinstance(out, np.ndarray) and (out.dtype != np.int32 or not out.flags["C_CONTIGUOUS"]):
        raise TypeError("output must be a contiguous int32 array")
    return out


def khcore_hdegrees(ctx, h: int, deg_out=None):
    """d_v^h(G) for all v; writes deg_out (host or device) if given."""
    lib = load_library()
    out = _out(ctx, deg_out)
    p, _ = _ptr(out)
    _check(lib, ctx, lib.khcore_hdegrees(ctx, int(h), p))
    return out


def khcore_hdegrees_ex(ctx, h: int, deg_out=None):
    """(deg, stats) of the all-vertex h-degree pass."""
    lib = load_library()
    out = _out(ctx, deg_out)
    p, _ = _ptr(out)
    stats = Stats()
    _check(lib, ctx, lib.khcore_hdegrees_ex(ctx, int(h), p, ctypes.byref(stats)))
    return out, stats.as_dict()


def khcore_hdegrees_of(ctx, h: int, verts, deg_out=None):
    """d_v^h(G) for the listed (distinct) vertices."""
    lib = load_library()
    pv, k = _ptr(verts)
    count = len(verts)
    out = np.empty(count, dtype=np.int32) if deg_out is None else deg_out
    po, _ = _ptr(out)
    _check(lib, ctx, lib.khcore_hdegrees_of(ctx, int(h), int(count), pv, po))
    del k
    return out


def khcore_hdegrees_static(n: int, m: int, row_ptr, col, h: int, verts, deg_out, stream=None):
    """d_v^h(G) of the listed vertices with no device allocation.

    For callers that may not allocate device memory while they run (a plugin
    whose host process owns all device memory, a latency-bound path). Every
    array is a CUDA int32 tensor the caller already holds: row_ptr [n+1],
    col [m], verts [count] (distinct ids), deg_out [count]. The scratch is a
    fixed array inside the library, shared by every call on a device: calls
    whose device work overlaps race, so order them on one stream."""
    lib = load_library()
    for a in (row_ptr, col, verts, deg_out):
        if not (_is_torch(a) and a.is_cuda):
            raise TypeError("khcore_hdegrees_static takes CUDA int32 tensors only")
    if len(deg_out) != len(verts):
        raise ValueError("deg_out and verts differ in length")
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    prp, _ = _ptr(row_ptr)
    pcl, _ = _ptr(col)
    pv, _ = _ptr(verts)
    po, _ = _ptr(deg_out)
    _check(lib, None, lib.khcore_hdegrees_static(int(n), int(m), prp, pcl, int(h), int(len(verts)), pv, po,
                                                 ctypes.c_void_p(stream) if stream else None))
    return deg_out


def khcore_decompose(ctx, h: int, core_out=None):
    """core_h(v) for all v."""
    lib = load_library()
    out = _out(ctx, core_out)
    p, _ = _ptr(out)
    _check(lib, ctx, lib.khcore_decompose(ctx, int(h), p))
    return out


def khcore_decompose_ex(ctx, h: int, core_out=None, round_out=None, want_rounds: bool = True):
    """(core, round, stats): core index, peel round of every vertex, statistics."""
    lib = load_library()
    core = _out(ctx, core_out)
    rnd = _out(ctx, round_out) if (want_rounds or round_out is not None) else None
    pc, _ = _ptr(core)
    pr, _ = _ptr(rnd)
    stats = Stats()
    _check(lib, ctx, lib.khcore_decompose_ex(ctx, int(h), pc, pr, ctypes.byref(stats)))
    return core, rnd, stats.as_dict()


def khcore_batch_create(v_off, e_off, row_ptr_local, col_local, flags: int = 0, stream=None):
    """One context over G packed graphs (see include/khcore.h)."""
    lib = load_library()
    vo = np.ascontiguousarray(v_off, dtype=np.int64)
    eo = np.ascontiguousarray(e_off, dtype=np.int64)
    G = len(vo) - 1
    rp, k1 = _ptr(row_ptr_local)
    cl, k2 = _ptr(col_local)
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    out = ctypes.c_void_p()
    st = lib.khcore_batch_create(G, vo.ctypes.data_as(ctypes.c_void_p), eo.ctypes.data_as(ctypes.c_void_p), rp, cl,
                                 int(flags), ctypes.c_void_p(stream) if stream else None, ctypes.byref(out))
    _check(lib, None, st)
    del k1, k2
    return _Ctx(out.value)


def khcore_batch_decompose(ctx, h, core_out=None, round_out=None, want_rounds: bool = True):
    """(core, round, stats) of a batch context; h[g] is graph g's hop bound."""
    lib = load_library()
    hv, k = _ptr(h)
    core = _out(ctx, core_out)
    rnd = _out(ctx, round_out) if (want_rounds or round_out is not None) else None
    pc, _ = _ptr(core)
    pr, _ = _ptr(rnd)
    stats = Stats()
    _check(lib, ctx, lib.khcore_batch_decompose(ctx, hv, pc, pr, ctypes.byref(stats)))
    del k
    return core, rnd, stats.as_dict()


def pack_graphs(graphs):
    """(v_off, e_off, row_ptr_local, col_local) for a list of graphs with
    .n, .row_ptr, .col (the packed layout of khcore_batch_create)."""
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    ms = np.array([len(g.col) for g in graphs], dtype=np.int64)
    v_off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    e_off = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
    rp = np.concatenate([np.asarray(g.row_ptr, dtype=np.int32) for g in graphs]) if graphs else np.zeros(0, np.int32)
    col = np.concatenate([np.asarray(g.col, dtype=np.int32) for g in graphs]) if graphs else np.zeros(0, np.int32)
    return v_off, e_off, rp, col


class Server:
    """Request server with continuous batching (khcore_server_* in the C ABI)."""

    def __init__(self, budget_bytes: int, slots: int = 2, max_batch: int = 256):
        self.lib = load_library()
        self.h = ctypes.c_void_p()
        st = self.lib.khcore_server_create(int(budget_bytes), int(slots), int(max_batch), ctypes.byref(self.h))
        if st != 0:
            raise KHCoreError(st, "khcore_server_create failed")
        self._n = {}

    def submit(self, n, row_ptr, col, h) -> int:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        t = ctypes.c_uint64()
        st = self.lib.khcore_server_submit(self.h, int(n), rp.ctypes.data_as(ctypes.c_void_p),
                                           cl.ctypes.data_as(ctypes.c_void_p) if cl.size else None, int(h),
                                           ctypes.byref(t))
        if st != 0:
            raise KHCoreError(st, "khcore_server_submit failed")
        self._n[t.value] = int(n)
        return t.value

    def done(self, ticket) -> bool:
        d = ctypes.c_int32()
        st = self.lib.khcore_server_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(d))
        if st != 0:
            raise KHCoreError(st, "khcore_server_poll failed")
        return bool(d.value)

    def wait(self, ticket, timeout_s: float = 600.0):
        """(core, latency_ms) of a request."""
        n = self._n.pop(ticket)
        out = np.empty(max(n, 1), dtype=np.int32)
        lat = ctypes.c_double()
        st = self.lib.khcore_server_wait(self.h, ctypes.c_uint64(ticket), out.ctypes.data_as(ctypes.c_void_p),
                                         float(timeout_s), ctypes.byref(lat))
        if st != 0:
            if st == 4:
                self._n[ticket] = n
            msg = self.lib.khcore_server_last_error(self.h)
            raise KHCoreError(st, "khcore_server_wait: " + (msg.decode() if msg else ""))
        return out[:n], lat.value

    def stats(self):
        q, c, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        u = ctypes.c_size_t()
        self.lib.khcore_server_stats(self.h, ctypes.byref(q), ctypes.byref(c), ctypes.byref(b), ctypes.byref(u))
        return dict(queued=q.value, completed=c.value, batches=b.value, bytes_in_use=u.value)

    def close(self):
        if self.h:
            self.lib.khcore_server_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def request_bytes(n: int, m: int) -> int:
    return int(load_library().khcore_request_bytes(int(n), int(m)))


class KHCore:
    """Context manager around one device-resident graph."""

    def __init__(self, n, row_ptr, col, flags: int = 0, stream=None, words: int = 0, alpha=None, loop=None,
                 lazy=None, blocks=None, update=None):
        self.ctx = khcore_create(n, row_ptr, col, flags, stream)
        self.n = int(n)
        if update is not None:
            khcore_set_update(self.ctx, update)
        if lazy is not None:
            khcore_set_lazy(self.ctx, lazy)
        if blocks is not None:
            khcore_set_graph_blocks(self.ctx, blocks)
        if loop is not None:
            khcore_set_round_loop(self.ctx, loop)
        if words:
            khcore_set_words(self.ctx, words)
        if alpha is not None:
            khcore_set_push_alpha(self.ctx, alpha)

    @classmethod
    def from_graph(cls, g, **kw):
        return cls(g.n, g.row_ptr, g.col, **kw)

    def hdegrees(self, h, out=None):
        return khcore_hdegrees(self.ctx, h, out)

    def decompose(self, h, out=None):
        return khcore_decompose(self.ctx, h, out)

    def decompose_ex(self, h, core_out=None, round_out=None):
        return khcore_decompose_ex(self.ctx, h, core_out, round_out)

    def set_words(self, w):
        khcore_set_words(self.ctx, w)

    def close(self):
        khcore_destroy(self.ctx)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
