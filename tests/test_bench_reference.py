"""bench.py --impl reference: the oracle on the host cores, W untimed and exactly K
timed steps on a bounded block of the workload (no GPU)."""
import argparse

import numpy as np

import bench
import synth


def test_reference_arm_runs_exactly_the_requested_steps():
    args = argparse.Namespace(workload="film_relax_32", steps=4, warmup=3)
    line = bench.run_reference(args, 0, 1)
    assert line["impl"] == "reference" and line["steps"] == 4 and line["warmup"] == 3
    assert line["unit"] == bench.UNIT and line["metric"] == bench.METRIC and line["higher_is_better"]
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    # one oracle process per host core (fewer only when memory is short)
    assert 1 <= line["cpu_baseline"]["cores"] <= bench.host_cores()
    assert line["cpu_baseline"]["cores"] == bench.oracle_workers(bench.workload("film_relax_32").sims[0])
    assert bench.run_reference(args, 1, 2) is None          # other ranks do no work


def test_reference_block_is_a_power_of_two_crop_of_the_workload():
    w = synth.skyrmion_film(nx=64, ny=48, nz=2)
    s = w.sims[0]
    assert bench.reference_block(s, 1.0) is s
    b = bench.reference_block(s, 0.2)                 # sqrt(0.2) * (64, 48) = (28.6, 21.5)
    assert (b.mesh.nx, b.mesh.ny, b.mesh.nz) == (16, 16, 2)
    assert np.array_equal(b.m0, s.m0[:, :, :16, :16]) and b.mat is s.mat
    tiny = bench.reference_block(s, 1e-6)
    assert (tiny.mesh.nx, tiny.mesh.ny) == (8, 8)


def test_extended_workload_switch():
    """--ext: per-cell A and D within 10 % of the material's and a Zhang-Li drift on the
    same meshes and states; the x inverse reads 2 more values a cell per stage; the
    reference arm runs the oracle on it."""
    args = argparse.Namespace(workload="film_relax_32", steps=2, warmup=3, ext=True)
    w0 = bench.workload("film_relax_32")
    w = bench.workload_for(args)
    assert w.name == w0.name + "_ext"
    s, s0 = w.sims[0], w0.sims[0]
    assert np.array_equal(s.m0, s0.m0) and s.mesh == s0.mesh and s0.mat.A_cells is None
    assert np.all(np.abs(s.mat.A_cells / s0.mat.A - 1) <= 0.1) and s.mat.u_stt == (50.0, 0.0, 0.0)
    kb, kb0 = bench.kernel_bytes(w, 8), bench.kernel_bytes(w0, 8)
    assert kb["x_inverse_epilogue"] - kb0["x_inverse_epilogue"] == 7 * 2 * 8 * s.mesh.ncells
    line = bench.run_reference(args, 0, 1)
    assert line["config"]["workload"].endswith("_ext") and line["value"] > 0
