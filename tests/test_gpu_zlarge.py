"""Full-size exactness: every vertex of the benchmark-scale decompositions
(the 1e6-vertex Chung-Lu graph at h = 2 and 3, the R-MAT scale-18 graph at
h = 4 and 5), in the launch configuration bench.py times (persistent round
loop, automatic W), checked by the oracle's certificate on ALL vertices
(oracle.certificate_all: Definition 2 and the containment after it; property
(0) plus the two BFS inequalities for every vertex, which together imply the
claimed core index is exact). The CPU checks run in a worker thread while the
GPU decomposes the next configuration (the oracle's C code releases the
interpreter lock and uses every host core). In a file of its own, collected
after the other GPU parity tests, because it is the slowest."""
import concurrent.futures as cf
import time

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

# (graph, h, certificate small_cap, certificate words): vertices with a claimed
# core <= small_cap run one early-stopped BFS each, the others a bit-parallel
# BFS of 64*words sources
CASES = [("cl1m", 2, 10 ** 9, 8), ("rmat18", 4, 1024, 8), ("rmat18", 5, 1024, 8), ("cl1m", 3, 1024, 16)]


@pytest.fixture(scope="module")
def kh():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2006_03372_gb300 as kh
    kh.load_library()
    return kh


def _check(g, h, core, rnd, cap, words):
    t0 = time.perf_counter()
    fails, bad = oracle.certificate_all(g, h, core, rnd, cap, words)
    return fails, np.flatnonzero(bad)[:10], time.perf_counter() - t0


def test_every_vertex_certified_at_full_size(kh):
    graphs = {}
    pending = []
    with cf.ThreadPoolExecutor(max_workers=1) as pool:
        for name, h, cap, words in CASES:
            g = graphs.setdefault(name, gg.config_graph(name))
            with kh.KHCore.from_graph(g, flags=kh.FLAG_TRUST_INPUT) as ctx:
                core, rnd, st = ctx.decompose_ex(h)
            assert st["deleted_total"] == g.n and (core >= 0).all() and (rnd >= 0).all(), (name, h)
            pending.append(((name, h), st["device_ms"], pool.submit(_check, g, h, core, rnd, cap, words)))
        report = []
        for key, gpu_ms, fut in pending:
            fails, first_bad, cpu_s = fut.result()
            report.append((key, gpu_ms, cpu_s))
            assert fails == 0, (key, first_bad)
    print("\nfull-size certificate (all vertices), %d host threads:" % oracle.threads())
    for (name, h), gpu_ms, cpu_s in report:
        print(f"  {name} h={h}: GPU decomposition {gpu_ms / 1e3:.1f} s, CPU certificate {cpu_s:.1f} s")
