"""bench.py reports ncu DRAM traffic only for the kernel sources it was taken on."""
import os

import bench


def test_traffic_row_needs_matching_fingerprint(tmp_path, monkeypatch):
    fp = bench.source_fingerprint()
    f = tmp_path / "traffic.md"
    f.write_text("| w | yz_cluster | k | %s | 123 | 456 |\n| w | x_forward | k | 0000000000000000 | 7 | 8 |\n" % fp)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.recorded_traffic("yz_cluster", "w") == 123.0
    assert bench.recorded_traffic("x_forward", "w") is None      # taken on other sources
    assert bench.recorded_traffic("yz_cluster", "other") is None


def test_fingerprint_changes_with_any_kernel_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2406_16064_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for fn in bench.KERNEL_SOURCES:
        (csrc / fn).write_text("x")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    f1 = bench.source_fingerprint()
    for fn in bench.KERNEL_SOURCES:
        (csrc / fn).write_text("y" + fn)
        f2 = bench.source_fingerprint()
        assert f2 != f1
        f1 = f2
    assert os.path.exists(str(csrc / "passes.cuh"))
