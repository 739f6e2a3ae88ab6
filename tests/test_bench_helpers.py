"""Host-side bookkeeping of bench.py (no GPU): the DRAM traffic of an ncu summary is reported only
while the summary's source digest matches the kernel sources, and the algorithmic byte and flop
counts follow their stated definitions."""
import hashlib
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _tree(tmp_path, sources, sha):
    csrc = tmp_path / "paper_2509_10226_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name, text in sources.items():
        (csrc / name).write_text(text)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k.md").write_text(
        "# title\n\n- kernel: `k<1>`\n"
        f"- source_sha1: `{sha}`  (sha1 of the concatenated sources below)\n"
        "- dram_bytes_per_launch: 123456\n")


def test_traffic_reported_only_for_the_captured_sources(bench, tmp_path, monkeypatch):
    sources = {"a.cu": "kernel a\n", "b.cuh": "helper b\n"}
    digest = hashlib.sha1(b"kernel a\nhelper b\n").hexdigest()
    _tree(tmp_path, sources, digest)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic(["a.cu", "b.cuh"], "k.md") == 123456.0
    # the digest covers the files in the given order
    assert bench.profiled_traffic(["b.cuh", "a.cu"], "k.md") is None
    # a changed source makes the capture stale
    (tmp_path / "paper_2509_10226_gb300" / "csrc" / "a.cu").write_text("kernel a, changed\n")
    assert bench.profiled_traffic(["a.cu", "b.cuh"], "k.md") is None
    # missing summary or source
    assert bench.profiled_traffic(["a.cu", "b.cuh"], "missing.md") is None
    assert bench.profiled_traffic(["a.cu", "c.cu"], "k.md") is None


def test_byte_and_flop_counts(bench):
    # CG: 4 nd index bytes and 6 metric words per cell, u read and y written once per DoF
    assert bench.cg_bytes(10, 7, 20, "fp32") == 10 * (80 + 24) + 2 * 4 * 7
    assert bench.cg_bytes(10, 7, 20, "fp64") == 10 * (80 + 48) + 2 * 8 * 7
    # Eq. 6 per cell: 2 (3 nq nd 2) + 33 nq + nd
    assert bench.cg_flops(1, 20, 35) == 2 * (3 * 35 * 20 * 2) + 33 * 35 + 20
    # DG: per cell index + metric, 2 vectors of nd values, per face ids/code and geometry
    assert bench.dg_bytes(2, 3, 1, 10, "fp32") == 2 * (4 + 24) + 2 * 4 * 2 * 10 + 3 * (12 + 32) + (8 + 20)
