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


def test_binning_traffic_comes_from_its_own_capture(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench._source_hash()
    (tmp_path / "profiles" / "bin_kernel_clusters_1m.md").write_text(
        f"# x\n\nkernel_source_hash: {h}\ntraffic_bytes_per_launch: 54539008\n")
    assert bench._profiled("clusters_1m", "bin_kernel") == {"traffic_bytes_per_launch": 54539008}
    assert bench._profiled("clusters_1m") == {}   # the solve kernel has no capture here
    (tmp_path / "profiles" / "bin_kernel_clusters_1m.md").write_text(
        "# x\n\nkernel_source_hash: 0000000000000000\ntraffic_bytes_per_launch: 1\n")
    assert bench._profiled("clusters_1m", "bin_kernel") == {}


def test_parity_stats_of_the_cpu_baseline_leg():
    """The bench's parity statistics (oracle sample of the timed workload
    against one GPU step) on CPU: a GPU result equal to the oracle's FP32
    rounding is exact; a planted velocity error and a swapped neighbour are
    reported."""
    import numpy as np

    import oracle
    from paper_2008_11578_gb300 import scenes
    s = scenes.open_square(300, 25.0, seed=3)
    sel = np.arange(0, s.n, 3)
    r = oracle.step(s, sel=sel)
    full = oracle.step(s)
    gpu = dict(pos=full.pos.astype(np.float32), vel=full.vel.astype(np.float32),
               nbr=full.nbr.copy(), cnt=full.cnt.copy(), flags=full.flags.copy())
    st = bench._parity_stats(s, r, gpu, sel)
    assert st["neighbour_lists_bit_exact"] and st["agents"] == len(sel)
    assert st["max_dv_m_s"] <= 1e-7 and st["max_dp_beyond_half_ulp_m"] <= 1e-9
    gpu["vel"][sel[4], 1] += 3e-4
    gpu["nbr"][sel[7], [0, 1]] = gpu["nbr"][sel[7], [1, 0]]
    st = bench._parity_stats(s, r, gpu, sel)
    assert not st["neighbour_lists_bit_exact"]
    assert abs(st["max_dv_m_s"] - 3e-4) <= 1e-6
