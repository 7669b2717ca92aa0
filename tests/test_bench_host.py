"""Host-side logic of bench.py (no GPU): the algorithmic byte counts of the metric and the rule
that committed ncu counters are reported only while the profiled kernel's source is unchanged."""
import os
import shutil

import pytest

import bench


def test_sweep_and_score_bytes():
    # 128^3 grid, K = 32, FP32: the per-sweep and scoring byte counts of the metric
    n, nnz_g, nnz_p, e_off = 2_097_152, 12_484_608, 4_194_302, 4_145_153
    assert bench.sweep_bytes(n, nnz_g) == 4 * (n + 1) + 8 * nnz_g + 4 * n + 2 * n * 32 * 4
    assert bench.sweep_bytes(n, nnz_g) == 653_524_996
    assert bench.sweep_bytes(n, nnz_p) == 587_202_548
    assert bench.score_bytes(n, e_off) == 16 * e_off + 2 * n * 32 * 4
    # BF16 blocks halve the vector bytes (2 N K s) only
    assert bench.sweep_bytes(n, nnz_g, s=2) == bench.sweep_bytes(n, nnz_g) - 2 * n * 32 * 2


def test_mlp_roofline_constants():
    assert bench.MLP_FLOP_PER_ROW == 2 * (16 * 64 + 64 * 64 + 64) == 10_368
    assert bench.MLP_BYTES_PER_ROW == 68


@pytest.mark.parametrize("kernel", sorted(bench.KERNEL_SOURCES))
def test_kernel_source_regions_exist(kernel):
    h = bench.kernel_source_hash(kernel)
    assert len(h) == 64 and h == bench.kernel_source_hash(kernel)


def test_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    summary = "k_jacobi_grid3d128_k32.txt"
    src = os.path.join(bench.ROOT, "profiles", summary)
    fake_root = tmp_path
    (fake_root / "profiles").mkdir()
    text = open(src).read()
    shas = set(__import__("re").findall(r"source_sha256:\s*([0-9a-f]{64})", text))
    assert len(shas) == 1
    sha = shas.pop()
    (fake_root / "profiles" / summary).write_text(text)
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: sha)
    t = bench.ncu_traffic("k_jacobi", summary)
    vals = [float(x) for x in __import__("re").findall(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)]
    assert t == sum(vals) / len(vals)
    # an edited kernel makes the committed counters stale: no traffic is reported
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: "0" * 64)
    assert bench.ncu_traffic("k_jacobi", summary) is None
    # a missing summary reports none either
    assert bench.ncu_traffic("k_jacobi", "absent.txt") is None
