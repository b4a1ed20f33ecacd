"""bench.py reports the round kernel's stored DRAM traffic only while the
kernel's code matches the capture it came from: the digest ignores comments
and whitespace and changes with any code edit."""
import importlib.util
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = ("khcore_persist.cuh", "khcore_device.cuh", "khcore_internal.cuh")


@pytest.fixture()
def bench(tmp_path):
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    csrc = tmp_path / "paper_2006_03372_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in FILES:
        shutil.copy(os.path.join(ROOT, "paper_2006_03372_gb300", "csrc", name), csrc / name)
    mod.ROOT = str(tmp_path)
    return mod, csrc


def test_digest_ignores_comments_and_whitespace(bench):
    mod, csrc = bench
    d0 = mod.kernel_source_digest()
    p = csrc / "khcore_persist.cuh"
    text = p.read_text()
    p.write_text("// a new comment line\n" + text.replace("\n", "\n\n", 3) + "\n/* block\n comment */\n")
    assert mod.kernel_source_digest() == d0


def test_digest_changes_with_code(bench):
    mod, csrc = bench
    d0 = mod.kernel_source_digest()
    p = csrc / "khcore_device.cuh"
    p.write_text(p.read_text() + "\nconstexpr int kUnusedProbe = 1;\n")
    assert mod.kernel_source_digest() != d0

