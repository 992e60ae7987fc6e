"""bench.py takes a kernel's measured DRAM traffic from its committed ncu summary only
while the kernel source still has the hash recorded at capture time."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_read_from_summary_when_source_unchanged():
    t = bench.measured_traffic("grid_dual", "c5")
    assert t is None or t > 0          # None only if the kernel changed since the capture
    assert bench.measured_traffic("grid_dual", "small") is None   # captured on c5 only
    assert bench.measured_traffic("select", "c5") is None         # no summary for it


def test_traffic_dropped_once_the_kernel_source_changes(tmp_path, monkeypatch):
    name = bench.PROFILE_OF_PHASE["grid_dual"]
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", name), tmp_path / "profiles" / name)
    src_rel = "paper_1610_08895_gb300/csrc/gridding.cu"
    (tmp_path / os.path.dirname(src_rel)).mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, src_rel), tmp_path / src_rel)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    orig = bench.measured_traffic("grid_dual", "c5")
    with open(tmp_path / src_rel, "a") as f:
        f.write("\n// an edit elsewhere in the file keeps the kernel's counters\n")
    assert bench.measured_traffic("grid_dual", "c5") == orig
    text = (tmp_path / src_rel).read_text()
    edited = text.replace("const int gam = c0 & 7;", "const int gam = (c0 & 7) + 0;")
    assert edited != text
    (tmp_path / src_rel).write_text(edited)
    assert bench.measured_traffic("grid_dual", "c5") is None
    if orig is not None:       # the copy matched its recorded hash before the edit
        assert orig > 0
