"""Host logic of bench.py that needs no GPU: the DRAM traffic read from the
committed ncu summaries, and its refusal of summaries taken on another kernel
source."""

import os
import shutil

import bench


def test_traffic_is_the_launch_weighted_mean_of_the_summary():
    mix = {5: 101, 8: 2}
    t = bench.kernel_traffic("gemm_tc.cu", "ozaki_tc_kernel_n8192.md", mix)
    assert t is not None
    vals = {}
    for line in open(os.path.join(bench.ROOT, "profiles", "ozaki_tc_kernel_n8192.md")):
        if line.strip().startswith("- traffic_bytes_per_launch_s"):
            k, v = line.strip()[2:].split(":", 1)
            vals[int(k.rsplit("s", 1)[1])] = float(v)
    assert abs(t - (101 * vals[5] + 2 * vals[8]) / 103) <= 1e-6 * t
    # a slice count the summary does not list gives no number
    assert bench.kernel_traffic("gemm_tc.cu", "ozaki_tc_kernel_n8192.md", {6: 10}) is None


def test_stale_summary_gives_no_traffic(tmp_path, monkeypatch):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    (root / "paper_2407_13299_gb300" / "csrc").mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "ozaki_tc_kernel_n8192.md"), root / "profiles")
    (root / "paper_2407_13299_gb300" / "csrc" / "gemm_tc.cu").write_text("// another source\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.kernel_traffic("gemm_tc.cu", "ozaki_tc_kernel_n8192.md", {5: 1}) is None
