"""Host logic of bench.py that needs no GPU: the committed ncu traffic is
used only while the CUDA sources still hash to the profiled build."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _tree(tmp_path):
    for d in ("paper_2008_11578_gb300/csrc", "include", "profiles"):
        os.makedirs(tmp_path / d, exist_ok=True)
    src = os.path.join(ROOT, "paper_2008_11578_gb300", "csrc")
    for f in os.listdir(src):
        if f.endswith((".cu", ".cuh")):
            shutil.copy(os.path.join(src, f), tmp_path / "paper_2008_11578_gb300" / "csrc" / f)
    shutil.copy(os.path.join(ROOT, "include", "orca.h"), tmp_path / "include" / "orca.h")


def test_profiled_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench._source_hash()
    prof = tmp_path / "profiles" / "solve_kernel_clusters_1m.md"
    prof.write_text(f"# x\n\nkernel_source_hash: {h}\ntraffic_bytes_per_launch: 12345\n"
                    "issue_active_pct: 70.5\nsimt_efficiency_pct: 27.4\n")
    assert bench._profiled_traffic("clusters_1m") == 12345
    assert bench._profiled("clusters_1m") == {"traffic_bytes_per_launch": 12345,
                                              "issue_active_pct": 70.5,
                                              "simt_efficiency_pct": 27.4}
    # any change of a CUDA source invalidates the captured traffic
    k = tmp_path / "paper_2008_11578_gb300" / "csrc" / "orca_math.cuh"
    k.write_text(k.read_text() + "\n// edited\n")
    assert bench._source_hash() != h
    assert bench._profiled_traffic("clusters_1m") is None
    assert bench._profiled("clusters_1m") == {}
    # no profile, no traffic
    prof.unlink()
    assert bench._profiled_traffic("clusters_1m") is None
