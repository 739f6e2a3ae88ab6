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


def test_executed_flop_count(bench):
    # per point: 3 nd FMAs for the gradient, 3 nd for the integration, metric 3 x (mul + 2 FMA), 3 weight muls
    assert bench.cg_flops_executed(1, 20, 35) == 35 * (2 * 3 * 20 + 2 * 3 * 20 + 15 + 3)


def test_flat_summary_keeps_the_comparison(bench):
    variants = {"fp64": {"gdofs": 0.61234567, "frac_measured": 0.93, "frac_measured_executed": 0.88},
                "tf32": {"gdofs": 61.0, "rel_l2_vs_fp64": 9.7e-4}, "csr_fp64": {"gdofs": 4.28, "rel_l2_vs_fp64": 1e-15},
                "dg_p2_48_tf32": {"gdofs": 54.0, "rel_l2_vs_fp64": 1.1e-3},
                "solve_sweep_48": {"p3": {"ir_tf32": {"seconds": 0.3}, "pcg_fp64": {"seconds": 5.7}, "n_dofs": 5}}}
    out = bench.flat_summary(variants, {"fp64": 1.3})
    assert out["fp64_gdofs"] == 0.6123 and out["tf32_rel_l2"] == 9.7e-4 and out["csr_fp64_gdofs"] == 4.28
    assert out["dg_p2_48_tf32_gdofs"] == 54.0 and out["fp64_frac_of_measured_fp64_peak"] == 0.93
    assert out["peak_fp64_tflops_measured"] == 1.3
    assert out["solve_p3_48_s"] == {"ir_tf32": 0.3, "pcg_fp64": 5.7}


def test_oracle_split_over_processes_equals_one_process():
    """The multi-core CPU baseline splits the cells over processes and sums the chunk results: that sum is
    the one-process oracle apply (the same operator, up to summation order)."""
    import sys

    sys.path.insert(0, ROOT)
    import bench as bench_main  # importable by name, so that spawned workers find the worker function
    import synth
    from oracle import cg, topology

    xyz, cells = synth.kuhn_cube(3, jitter=0.2, seed=0)
    dofs, keys = topology.cg_numbering(cells, 2)
    u = synth.uniform_vector(keys.shape[0], 1)
    y1 = cg.apply(xyz, cells, u, 2, dofs=dofs)
    pool = bench_main.OracleCores(xyz, cells, u, 2, dofs, 2)
    try:
        y2, _ = pool.apply()
    finally:
        pool.close()
    assert abs(y2 - y1).max() <= 1e-13 * abs(y1).max()
    assert bench_main.host_cores() >= 1 and isinstance(bench_main.cpu_model(), str)
