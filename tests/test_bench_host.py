"""Host logic of bench.py that needs no GPU: the committed ncu traffic records are used only
while the source files they were taken from are unchanged, an ncu CSV capture is turned into
records against the library's own byte counts, the CPU-oracle extrapolation model, and the
workload description."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_records_are_well_formed():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)
    for name, k in rec["kernels"].items():
        assert k["dram_bytes"] > 0 and k["algorithmic_bytes"] > 0, name
        assert abs(k["dram_over_algorithmic"] - k["dram_bytes"] / k["algorithmic_bytes"]) < 1e-9, name
        assert k["source_files"], name


def test_traffic_record_goes_stale_when_a_source_changes(tmp_path, monkeypatch):
    rec = {"kernels": {"k": {"dram_over_algorithmic": 1.0, "source_files": {"src.cu": "0" * 16}}}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    (tmp_path / "src.cu").write_text("// kernel\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("k") is None                      # hash differs: stale
    rec["kernels"]["k"]["source_files"]["src.cu"] = bench.file_hash("src.cu")
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    assert bench.ncu_traffic("k")["dram_over_algorithmic"] == 1.0
    assert bench.ncu_traffic("missing") is None


CSV = '''==PROF== Connected to process
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","python","h","void helm::(anonymous namespace)::k_smooth0<double, true, double>(helm::Grid)","1","7","(32, 8, 1)","(9, 33, 5)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Mbyte","600.00"
"0","1","python","h","void helm::(anonymous namespace)::k_smooth0<double, true, double>(helm::Grid)","1","7","(32, 8, 1)","(9, 33, 5)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","Mbyte","200.00"
"0","1","python","h","void helm::(anonymous namespace)::k_smooth0<double, true, double>(helm::Grid)","1","7","(32, 8, 1)","(9, 33, 5)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","usecond","150.00"
"1","1","python","h","void helm::(anonymous namespace)::k_smooth0<double, true, double>(helm::Grid)","1","7","(32, 8, 1)","(9, 33, 5)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Mbyte","80.00"
"1","1","python","h","void helm::(anonymous namespace)::k_smooth0<double, true, double>(helm::Grid)","1","7","(32, 8, 1)","(9, 33, 5)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","Mbyte","20.00"
"1","1","python","h","void helm::(anonymous namespace)::k_smooth0<double, true, double>(helm::Grid)","1","7","(32, 8, 1)","(9, 33, 5)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","usecond","20.00"
"2","1","python","h","void helm::(anonymous namespace)::k_stencil<double, 2, true, double, double, double, false>(helm::Grid)","1","7","(32, 8, 1)","(9, 33, 5)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Gbyte","1.00"
"2","1","python","h","void helm::(anonymous namespace)::k_stencil<double, 2, true, double, double, double, false>(helm::Grid)","1","7","(32, 8, 1)","(9, 33, 5)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","Mbyte","250.00"
"2","1","python","h","void helm::(anonymous namespace)::k_stencil<double, 2, true, double, double, double, false>(helm::Grid)","1","7","(32, 8, 1)","(9, 33, 5)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","usecond","300.00"
'''


def test_write_traffic_from_an_ncu_csv(tmp_path, monkeypatch):
    """The finest level's down-sweep kernel is the first launch of its family in the region and
    its up-sweep kernel the last; each record holds DRAM bytes over the library's count."""
    (tmp_path / "profiles").mkdir()
    (tmp_path / "regions").mkdir()
    for f in bench.SOURCES["vcycle64"]:
        os.makedirs(tmp_path / os.path.dirname(f), exist_ok=True)
        (tmp_path / f).write_text("// source\n")
    region = {"region": "vcycle64", "workload": "w", "families": {
        "k_smooth0 (finest)": {"launches": 1, "bytes": 1.0e9}, "k_smooth0": {"launches": 1, "bytes": 1e8},
        "k_stencil(jacobi) (finest)": {"launches": 1, "bytes": 1.25e9}}}
    (tmp_path / "regions" / "ncu_region_vcycle64.json").write_text(json.dumps(region))
    (tmp_path / "cap.csv").write_text(CSV)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "REGION_OUT", str(tmp_path / "regions"))
    bench.write_traffic(str(tmp_path / "cap.csv"), "vcycle64")
    rec = json.loads((tmp_path / "profiles" / "ncu_traffic.json").read_text())["kernels"]
    assert rec["k_smooth0 (finest)"]["dram_bytes"] == pytest.approx(8e8)
    assert rec["k_smooth0 (finest)"]["dram_over_algorithmic"] == pytest.approx(0.8)
    assert rec["k_stencil(jacobi) (finest)"]["dram_over_algorithmic"] == pytest.approx(1.0)
    assert rec["k_stencil(jacobi) (finest)"]["duration_us"] == pytest.approx(300.0)
    assert bench.ncu_traffic("k_smooth0 (finest)") is not None


def test_kernel_families_from_ncu_names():
    assert bench._family_of("void helm::(anonymous namespace)::k_stencil<float, 1, false, float, double, float, "
                            "false>(helm::Grid)") == "k_stencil(resid)"
    assert bench._family_of("k_gs_update_sums(const cx<double>*)") == "k_gs_update"
    assert bench._family_of("k_mdot<cx<double>, AccD3>(int)") == "k_mdot"
    assert bench._template_real("k_stencil<double, 0, false>(x)") == "double"
    assert bench._family_of("void k_restrict2<float>(Grid, Grid)") == "k_restrict"
    assert bench._family_of("void k_prolong2<double>(Grid, Grid)") == "k_prolong_add"
    assert bench._family_of("void k_rr<double, true, double>(Grid)") == "k_rr"
    assert bench._family_of("k_givens(int)") is None


def test_oracle_step_model_and_extrapolation():
    # samples of 1 and 4 steps: T = overhead + steps * step with step 2 s, overhead 3 s
    samples = [[1, 5.0], [4, 11.0], [1, 5.0], [4, 11.0]]
    step, over = bench.step_model(samples)
    assert step == pytest.approx(2.0) and over == pytest.approx(3.0)
    # 61 steps of GMRES(30): three restart cycles
    assert bench.extrapolate(step, over, 61) == pytest.approx(61 * 2.0 + 3 * 3.0)
    assert bench.step_model([[2, 4.0]]) == (2.0, 0.0)


def test_stored_oracle_counts_are_read():
    path = os.path.join(ROOT, "tests", "golden", "wedge_oracle_counts.txt")
    if not os.path.exists(path):
        pytest.skip("no stored counts")
    for ln in open(path):
        if ln.strip() and not ln.startswith("#"):
            name, n, it = ln.split()
            assert bench.oracle_count(name, int(n)) == int(it) > 0


def test_workload_config_follows_n():
    for n in (128, 256):
        c = bench.workload_config(n)
        assert c["unknowns"] == (n + 1) ** 3 and f"{n + 1}^3 unknowns" in c["workload"]
        assert c["workload"].startswith(f"wedge n={n},")
        assert f"{31 * 16 * (n + 1) ** 3 / 1e9:.2f} GB" in c["l2"]
    assert "complex64" in bench.workload_config(128, "mixed")["precision"]
