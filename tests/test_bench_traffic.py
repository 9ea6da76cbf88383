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


def test_algorithmic_bytes_of_the_film_by_hand():
    """512x512x4 film, FP32: per launch the cluster pass reads and writes the x-transformed
    rows once (3 nz ny Kx complex = 25,214,976 B) and reads the blocked tensor once
    ((4 nz + 2 (nz - 1)) (Py/2 + 1) Kx floats = 23,158,872 B); the x inverse of stage s
    reads the rows and the stage state and writes k_s (plus the partial error at s = 7)."""
    import numpy as np
    import synth
    mesh = synth.Mesh(512, 512, 4, 2e-9, 2e-9, 1e-9)
    mat = synth.Material(Ms=5.8e5, A=1.5e-11, D=3e-3, dmi=1, Ku=8e5)
    w = synth.Workload("film", [synth.Sim(mesh, mat, np.zeros((3,) + mesh.shape))], "f32", 1e-5)
    e, n, Kx = 4, mesh.ncells, 513
    rows = 3 * 4 * 512 * Kx * 2 * e
    tens = (4 * 4 + 2 * 3) * (1024 // 2 + 1) * Kx * e
    assert (rows, tens) == (25_214_976, 23_158_872)
    kb = bench.kernel_bytes(w, e)
    assert kb["yz_cluster"] / 7 == 2 * rows + tens == 73_588_824
    assert kb["x_inverse_epilogue"] == 7 * (rows + 6 * e * n) + 3 * e * n
    assert kb["x_forward"] == sum(3 * e * n * s + (3 * e * n if s > 1 else 0) + (3 * e * n if s == 7 else 0)
                                  for s in range(1, 8)) + 7 * rows
    assert kb["project"] == 6 * e * n and not kb["z_fused"] and not kb["y_fused"]
    alg = bench.kernel_bytes(w, e, spectrum=False)
    assert alg["yz_cluster"] / 7 == tens
    assert alg["x_inverse_epilogue"] == 7 * 6 * e * n + 3 * e * n
    assert kb["x_forward"] - alg["x_forward"] == 7 * rows
