"""Host logic of bench.py that needs no GPU: the committed ncu traffic record is used only while
the source files it was taken from are unchanged, and the workload description follows n."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_record_of_the_dominant_kernel():
    """The committed record of the benchmark's dominant kernel holds DRAM and algorithmic bytes
    of one captured launch; while its sources are unchanged the two agree (no re-reads)."""
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)["kernels"]["k_mdot"]
    assert rec["dram_bytes_per_launch"] > 0 and rec["algorithmic_bytes_per_launch"] > 0
    k = bench.ncu_traffic("k_mdot")
    if k is None:
        pytest.skip("k_mdot changed since its counters were taken: the bench reports traffic null")
    assert 0.95 <= k["dram_bytes_per_launch"] / k["algorithmic_bytes_per_launch"] <= 1.1


def test_traffic_record_goes_stale_when_a_source_changes(tmp_path, monkeypatch):
    rec = {"kernels": {"k": {"dram_bytes_per_launch": 1.0, "algorithmic_bytes_per_launch": 1,
                             "source_files": {"src.cu": "0" * 16}}}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    (tmp_path / "src.cu").write_text("// kernel\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("k") is None                      # hash differs: stale
    rec["kernels"]["k"]["source_files"]["src.cu"] = bench.file_hash("src.cu")
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    assert bench.ncu_traffic("k")["dram_bytes_per_launch"] == 1.0
    assert bench.ncu_traffic("missing") is None


def test_workload_config_follows_n():
    for n in (128, 256):
        c = bench.workload_config(n)
        assert c["unknowns"] == (n + 1) ** 3 and f"{(n + 1) ** 3:,}" in c["workload"]
        assert f"{31 * 16 * (n + 1) ** 3 / 1e9:.2f} GB" in c["l2"]
    assert "complex64" in bench.workload_config(128, "mixed")["precision"]
