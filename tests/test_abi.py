"""The C-ABI boundary on the CPU: the library builds for sm_103a, loads, and
exports every entry point include/khcore.h declares; host-side argument and
CSR validation returns KHCORE_EINVAL before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(khcore_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import paper_2006_03372_gb300 as kh
    from paper_2006_03372_gb300 import _build
    _build.build()
    return kh.load_library()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["khcore_create", "khcore_hdegrees", "khcore_decompose", "khcore_decompose_ex",
              "khcore_destroy", "khcore_last_error"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), f"{s} declared in include/ but not exported"


def test_status_strings(lib):
    import paper_2006_03372_gb300 as kh
    for code, name in kh.STATUS.items():
        assert kh.khcore_status_string(code) == name


def _create_status(n, rp, col):
    import paper_2006_03372_gb300 as kh
    try:
        ctx = kh.khcore_create(n, rp, col)
    except kh.KHCoreError as e:
        return e.status, str(e)
    kh.khcore_destroy(ctx)
    return 0, ""


@pytest.mark.parametrize("case", ["selfloop", "dup", "asym", "range", "rowptr", "neg_n", "rowptr_wrap"])
def test_malformed_csr_is_einval(lib, case):
    g = gg.cycle(6)
    rp, col, n = g.row_ptr.copy(), g.col.copy(), g.n
    if case == "selfloop":
        col[0] = 0
    elif case == "dup":
        col[1] = col[0]
    elif case == "asym":
        # drop one direction of edge 0-1 by rewiring 0's entry to 3
        col[np.flatnonzero(col[rp[0]:rp[1]] == 1)[0]] = 3
    elif case == "range":
        col[2] = 99
    elif case == "rowptr":
        rp[3] = rp[2] - 1
    elif case == "neg_n":
        n = -1
    elif case == "rowptr_wrap":
        # offsets whose int32 differences wrap to non-negative row lengths:
        # 2^31 - 1 followed by -2 (csr_row_ok takes them in 64 bits)
        n = 3
        rp = np.array([0, 2 ** 31 - 1, -2, 4], dtype=np.int32)
        col = np.array([1, 0, 2, 1], dtype=np.int32)
    st, msg = _create_status(n, rp, col)
    assert st == 1, msg


def test_compiled_for_sm_103a_only():
    from paper_2006_03372_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_batch_create_rejects_bad_graph(lib):
    import paper_2006_03372_gb300 as kh
    good, bad = gg.cycle(5), gg.cycle(6)
    col = bad.col.copy()
    col[0] = 0  # self-loop in graph 1
    bad = gg.Graph(bad.n, bad.row_ptr, col)
    v_off, e_off, rp, cl = kh.pack_graphs([good, bad])
    with pytest.raises(kh.KHCoreError) as ei:
        kh.khcore_batch_create(v_off, e_off, rp, cl)
    assert ei.value.status == 1 and "graph 1" in str(ei.value)
