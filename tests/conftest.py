import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size configuration (minutes)")


def load_fig1():
    """The paper's running example (tests/golden/fig1_example.txt), 0-based."""
    import graphgen as gg
    edges, vals = [], {}
    with open(os.path.join(GOLDEN, "fig1_example.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            if key == "edge":
                edges.append((int(rest[0]) - 1, int(rest[1]) - 1))
            else:
                vals[key] = rest
    return gg.from_edge_list(14, edges, "fig1"), vals


@pytest.fixture(scope="session")
def fig1():
    return load_fig1()


def small_graphs(seed_base=0, count=12, n_range=(2, 40)):
    """A seeded mix of tiny ER, Chung-Lu, R-MAT and structured graphs."""
    import graphgen as gg
    out = []
    rng = gg.Stream(seed_base, "small")
    for i in range(count):
        n = int(n_range[0] + rng.below(n_range[1] - n_range[0] + 1, 1)[0])
        kind = i % 3
        if kind == 0:
            m = int(rng.below(max(1, min(3 * n, n * (n - 1) // 2)) + 1, 1)[0])
            out.append(gg.erdos_renyi_gnm(n, m, 1000 + i))
        elif kind == 1 and n >= 4:
            mean = min(4.0, n / 4)
            out.append(gg.chung_lu(n, mean, 2.5, max(n / 2, 2 * mean), 2000 + i))
        else:
            s = max(2, int(np.ceil(np.log2(max(n, 4)))))
            out.append(gg.rmat(s, 4, 0.57, 0.19, 0.19, 0.05, 3000 + i))
    return out
