"""Host logic of bench.py that needs no GPU: the DRAM traffic read from the
committed ncu summaries, and its refusal of summaries taken on another kernel
source."""

import os
import shutil

import bench


def _summary_for(root, source_text):
    """A copy of the committed summary whose source hash names `source_text`."""
    import hashlib

    (root / "profiles").mkdir(parents=True)
    (root / "paper_2407_13299_gb300" / "csrc").mkdir(parents=True)
    (root / "paper_2407_13299_gb300" / "csrc" / "gemm_tc.cu").write_text(source_text)
    digest = hashlib.sha256(source_text.encode()).hexdigest()[:16]
    lines = []
    for line in open(os.path.join(bench.ROOT, "profiles", "ozaki_tc_kernel_n8192.md")):
        if line.strip().lstrip("- ").startswith("source_sha256"):
            line = f"- source_sha256: {digest} (test copy)\n"
        lines.append(line)
    (root / "profiles" / "ozaki_tc_kernel_n8192.md").write_text("".join(lines))


def test_traffic_is_the_launch_weighted_mean_of_the_summary(tmp_path, monkeypatch):
    vals = {}
    for line in open(os.path.join(bench.ROOT, "profiles", "ozaki_tc_kernel_n8192.md")):
        if line.strip().startswith("- traffic_bytes_per_launch_s"):
            k, v = line.strip()[2:].split(":", 1)
            vals[int(k.rsplit("s", 1)[1])] = float(v.split()[0])
    assert 5 in vals and 8 in vals
    root = tmp_path / "repo"
    _summary_for(root, "// the kernel source the counters were taken on\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    mix = {5: 101, 8: 2}
    t = bench.kernel_traffic("gemm_tc.cu", "ozaki_tc_kernel_n8192.md", mix)
    assert t is not None
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


def test_fermi_occupations_match_the_oracle():
    """The benchmark's exact occupations (the reference its finite-temperature
    errors are measured against) equal the oracle's Fermi function, without
    overflow far from mu."""
    import numpy as np

    from oracle import foe as fo

    e = np.concatenate([np.linspace(-1.5, 1.5, 1001), [-1e4, 1e4]])
    for mu, kT in ((0.0, 0.05), (-0.0346, 0.05), (0.3, 0.001)):
        got = bench.fermi_occupations(e, mu, kT)
        assert np.all(np.isfinite(got)) and got[-2] == 1.0 and got[-1] == 0.0
        assert np.max(np.abs(got - fo.fermi(e, mu, kT))) <= 1e-16
