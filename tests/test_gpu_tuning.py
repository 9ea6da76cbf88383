"""Autotuned tile shapes and schedules: every selectable tuning gives the oracle's field,
and mm_autotune picks one no slower than the fixed rule.

Tolerances: FP64 fields 1e-10 relative (max over cells); FP32 fields 1e-5 relative RMS.
"""
import itertools

import numpy as np
import pytest

import synth
from paper_2406_16064_gb300 import mm
from tests.gpu_util import max_rel, oracle_rhs, rms_rel

pytestmark = pytest.mark.gpu


def _mat():
    return synth.Material(Ms=8e5, A=1.3e-11, D=3e-3, dmi=1, Ku=4e5, u=(0.2, 0.3, 0.9), Kc=1e4,
                          H=(1e4, -2e4, 3e4), alpha=0.3)


# a cluster-pass film (3 planes), a single-plane film, a mesh with separate y and z passes
MESHES = [(40, 24, 3), (48, 40, 1), (20, 12, 10)]


def _tunings(nz):
    """Every kx block width, one or two row tiles, three CTA widths, both column groups and
    every cluster-kernel build (2, 3 or 4 CTAs per SM)."""
    for ty, rx, xt in itertools.product((1, 2, 4, 8, 16, 32), (1, 3), (0, 128, 512)):
        for g, occ in (itertools.product((1, 2), (0, 3, 4)) if 1 < nz <= 8 else ((0, 0),)):
            yield {"Ty": ty, "Rx": rx, "x_threads": xt, "col_threads": xt if nz == 1 or nz > 8 else 0,
                   "col_group": g, "col_occ": occ, "x_stage": (ty + rx) % 2}


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("dims", MESHES)
def test_every_selectable_tuning_gives_the_oracle_field(precision, dims):
    mesh = synth.Mesh(*dims, 2e-9, 2e-9, 1e-9)
    sim = synth.Sim(mesh, _mat(), synth.random_state(13, mesh))
    ref_k, ref_H = oracle_rhs(sim, method="direct")
    ran = 0
    for t in _tunings(mesh.nz):
        if precision == "f64" and (t["x_threads"] > 512 or t["col_threads"] > 512):
            continue
        ctx = mm.Context(precision)
        ctx.add_sim(mesh, sim.mat)
        try:
            ctx.set_tuning(0, t)
        except mm.MMError as e:                  # tiles that do not fit are refused up front
            assert e.code == mm.MM_EINVAL
            ctx.close()
            continue
        ctx.precompute()
        got = ctx.get_tuning(0)
        assert got["Ty"] == t["Ty"] and got["Rx"] == min(t["Rx"], mesh.ny) and got["col_occ"] == t["col_occ"]
        dmdt, heff = ctx.rhs_host(sim.m0.ravel())
        ctx.close()
        if precision == "f64":
            assert max_rel(heff, ref_H) < 1e-10 and max_rel(dmdt, ref_k) < 1e-10, t
        else:
            assert rms_rel(heff, ref_H) < 1e-5 and rms_rel(dmdt, ref_k) < 1e-5, t
        ran += 1
    assert ran >= 12


def test_autotune_picks_no_slower_than_the_rule_and_keeps_parity():
    mesh = synth.Mesh(128, 96, 2, 2e-9, 2e-9, 2e-9)
    sim = synth.Sim(mesh, _mat(), synth.random_state(14, mesh))
    ctx = mm.Context("f32")
    ctx.add_sim(mesh, sim.mat)
    ctx.add_sim(mesh, sim.mat)                   # a second simulation of the same mesh
    t, best, rule = ctx.autotune(0, reps=4)
    assert best <= rule and best > 0
    got = ctx.get_tuning(0)
    assert got == ctx.get_tuning(1)
    assert (got["Ty"], got["Rx"], got["col_group"]) == (t["Ty"], t["Rx"], t["col_group"])
    assert t["x_threads"] in (0, got["x_threads"])
    ctx.precompute()
    dmdt, heff = ctx.rhs_host(np.concatenate([sim.m0.ravel()] * 2))
    ref_k, ref_H = oracle_rhs(sim, method="fft")
    n = 3 * mesh.ncells
    for i in range(2):
        assert rms_rel(heff[i * n:(i + 1) * n], ref_H) < 1e-5
        assert rms_rel(dmdt[i * n:(i + 1) * n], ref_k) < 1e-5
    ctx.close()


def test_tuning_cache_round_trip(tmp_path):
    from paper_2406_16064_gb300 import tuning
    path = str(tmp_path / "tune.json")
    mesh = synth.Mesh(64, 64, 1, 2e-9, 2e-9, 2e-9)
    ctx = mm.Context("f32")
    ctx.add_sim(mesh, _mat())
    first = tuning.tune_context(ctx, [mesh], "gpu", reps=3, path=path)
    (k, e), = first.items()
    assert k.endswith("|64x64x1|64x64x1*1")
    assert e["cached"] is False and e["ms_per_attempt"] <= e["rule_ms_per_attempt"]
    t0 = ctx.get_tuning(0)
    ctx.close()
    ctx = mm.Context("f32")
    ctx.add_sim(mesh, _mat())
    again = tuning.tune_context(ctx, [mesh], "gpu", reps=3, path=path)
    assert again[k]["cached"] is True and ctx.get_tuning(0) == t0
    ctx.close()


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("dims", [(64, 48, 3), (64, 40, 1), (32, 16, 12), (33, 17, 2), (48, 5, 4)])
def test_staged_x_inverse_rows_are_bitwise_the_loaded_ones(precision, dims):
    """The x-inverse pass with its state rows staged by bulk copies (x_stage = 1) computes
    exactly what the direct loads give: right-hand side and three RK45 attempts bit for
    bit, energies up to the order of their atomic FP64 sums, and the oracle's field.  (33 cells a row in FP32 is 132 bytes, not a
    multiple of 16: that mesh takes the direct loads whatever the tuning says.)"""
    mesh = synth.Mesh(*dims, 2e-9, 2e-9, 1e-9)
    sim = synth.Sim(mesh, _mat(), synth.random_state(19, mesh))
    out = {}
    for stage in (0, 1):
        for rx in (1, 2, 5):
            if rx > mesh.ny:
                continue
            ctx = mm.Context(precision)
            ctx.add_sim(mesh, sim.mat)
            ctx.set_tuning(0, {"Rx": rx, "x_stage": stage})
            ctx.precompute()
            assert ctx.get_tuning(0)["x_stage"] == stage
            dmdt, heff = ctx.rhs_host(sim.m0.ravel())
            ctx.set_m(sim.m0.ravel())
            E = ctx.energy(0)
            ctx.reset_time()
            ctx.rk45_setup(1e-5 if precision == "f32" else 1e-6)
            ctx.rk45_attempts(3)
            out[(stage, rx)] = (dmdt, heff, E, ctx.get_m(0), ctx.status(0)["n_accepted"])
            ctx.close()
    ref_k, ref_H = oracle_rhs(sim, method="direct")
    for (stage, rx), (dmdt, heff, E, m, nacc) in out.items():
        base = out[(0, rx)]
        assert np.array_equal(dmdt, base[0]) and np.array_equal(heff, base[1])
        assert np.array_equal(m, base[3]) and nacc == base[4]
        # energies are FP64 sums combined across CTAs by atomics: equal up to summation order
        for k in E:
            assert abs(E[k] - base[2][k]) <= 1e-12 * max(abs(v) for v in base[2].values())
        if precision == "f64":
            assert max_rel(heff, ref_H) < 1e-10
        else:
            assert rms_rel(heff, ref_H) < 1e-5
