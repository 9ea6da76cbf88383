"""GPU parity of the steepest-descent minimiser (mm_minimize) against oracle.minimize.

The step sequence depends on the Barzilai-Borwein sums, so parity of whole
trajectories is checked over the first steps (FP64, fields agree to ~1e-13);
converged states are compared by energy and position (one minimum).
"""
import numpy as np
import pytest

import synth
from oracle import demag as D
from oracle import fields as F
from oracle import minimize as SD
from tests.gpu_util import make_ctx

pytestmark = pytest.mark.gpu


def _film_sim(nx=12, ny=10, nz=1, seed=3):
    mesh = synth.Mesh(nx, ny, nz, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, D=1e-3, dmi=1, Ku=5e5, u=(0, 0, 1), H=(5e4, 0, 2e4), alpha=0.5,
                         precession=0, demag=1)
    m0 = synth.tilt(synth.uniform_state(mesh, (0, 0, 1)), seed, 0.2)
    return synth.Sim(mesh, mat, m0)


def _oracle(sim, max_dmdt, max_steps):
    Ms = F.ms_array(sim.mesh, sim.mat, sim.Ms_cells)
    Nt = D.mesh_tensor(sim.mesh)
    field = lambda y: F.h_eff(sim.mesh, sim.mat, y, Ms, Nt, "fft")
    m, st = SD.minimize(field, sim.m0.copy(), sim.mat, Ms, max_dmdt=max_dmdt, max_steps=max_steps)
    E = F.energies(sim.mesh, sim.mat, m, Ms, Nt, "fft")["total"]
    return m, st, E


@pytest.mark.parametrize("dims", [(12, 10, 1), (9, 7, 3)])
def test_first_steps_match_the_oracle_f64(dims):
    sim = _film_sim(*dims)
    ctx = make_ctx("f64", [sim])
    ctx.set_m(sim.m0.ravel())
    steps, conv = ctx.minimize(0.0, max_steps=12, sync_every=4)
    assert steps == 12 and not conv
    m_ref, st, _ = _oracle(sim, 0.0, 12)
    info = ctx.minimize_info(0)
    assert abs(info["tau"] - st.tau) <= 1e-7 * st.tau
    assert np.abs(ctx.get_m(0) - m_ref.ravel()).max() < 1e-8


def test_converged_film_matches_the_oracle_minimum_f64():
    sim = _film_sim()
    ctx = make_ctx("f64", [sim])
    ctx.set_m(sim.m0.ravel())
    steps, conv = ctx.minimize(1e4, max_steps=3000)
    assert conv and steps < 600, steps
    m_ref, st, E_ref = _oracle(sim, 1e4, 3000)
    assert st.converged
    m = ctx.get_m(0)
    E = ctx.energy(0)["total"]
    assert abs(E - E_ref) <= 1e-9 * abs(E_ref)
    assert np.abs(m - m_ref.ravel()).max() < 1e-5
    assert ctx.minimize_info(0)["max_dmdt"] < 1e4


def test_converged_film_f32_reaches_the_fp64_minimum():
    sim = _film_sim()
    ctx = make_ctx("f32", [sim])
    ctx.set_m(sim.m0.ravel())
    steps, conv = ctx.minimize(1e5, max_steps=3000)
    assert conv, ctx.minimize_info(0)
    _, _, E_ref = _oracle(sim, 1e4, 3000)
    E = ctx.energy(0)["total"]
    assert abs(E - E_ref) <= 1e-5 * abs(E_ref)
    m = ctx.get_m(0).reshape(3, -1)
    assert np.abs(np.sqrt((m ** 2).sum(0)) - 1).max() < 2 * 2.0 ** -23


def test_macrospin_stoner_wohlfarth_angle_on_gpu():
    mesh = synth.Mesh(1, 1, 1, 2e-9, 2e-9, 2e-9)
    Ku, Ms0 = 5e5, 8e5
    HK = 2 * Ku / (F.MU0 * Ms0)
    mat = synth.Material(Ms=Ms0, Ku=Ku, u=(0, 0, 1), H=(0.3 * HK, 0, 0), alpha=0.5, precession=0, demag=0)
    sim = synth.Sim(mesh, mat, synth.uniform_state(mesh, (0.2, 0.1, 1.0)))
    ctx = make_ctx("f64", [sim])
    ctx.set_m(sim.m0.ravel())
    steps, conv = ctx.minimize(1.0, max_steps=500)
    assert conv and steps < 100
    m = ctx.get_m(0)
    assert abs(m[0] - 0.3) < 1e-8 and abs(m[1]) < 1e-8 and abs(m[2] - np.sqrt(0.91)) < 1e-8


def test_uneven_batch_each_simulation_reaches_its_own_minimum():
    """Per-simulation step sizes and stopping: three meshes and materials in one context."""
    sims = [_film_sim(12, 10, 1, seed=3), _film_sim(9, 7, 3, seed=4), _film_sim(16, 6, 1, seed=5)]
    sims[2].mat.Ku = 3e5
    sims[2].mat.H = (0.0, 3e4, 4e4)
    ctx = make_ctx("f64", sims)
    ctx.set_m(np.concatenate([s.m0.ravel() for s in sims]))
    steps, conv = ctx.minimize(1e4, max_steps=3000)
    assert conv
    for i, s in enumerate(sims):
        m_ref, st, E_ref = _oracle(s, 1e4, 3000)
        assert st.converged
        E = ctx.energy(i)["total"]
        assert abs(E - E_ref) <= 1e-9 * abs(E_ref), i
        assert np.abs(ctx.get_m(i) - m_ref.ravel()).max() < 1e-5, i
        assert ctx.minimize_info(i)["status"] == 2


def test_random_start_reaches_the_rk45_minimum_f64():
    """The 32x32x1 film of random directions: steepest descent converges (step cap)
    to the energy the damped RK45 relaxation reaches, in far fewer field evaluations."""
    w = synth.film_relax_32()
    sim = w.sims[0]
    ctx = make_ctx("f64", [sim])
    ctx.set_m(sim.m0.ravel())
    steps, conv = ctx.minimize(1e7, max_steps=5000)
    assert conv and steps < 2000, (steps, ctx.minimize_info(0))
    E_sd = ctx.energy(0)["total"]
    ctx.set_m(sim.m0.ravel())
    ctx.reset_time()
    attempts = ctx.relax(w.rtol, max_dmdt=1e7, max_steps=20000, sync_every=64)
    assert ctx.status(0)["status"] == 2
    E_rk = ctx.energy(0)["total"]
    # both stop at the first state below 1e7 rad/s (RK45 at rtol 1e-6 cannot resolve much
    # lower: its error-controller noise is ~2e6 rad/s here), so they agree to the energy
    # error of that threshold, not to rounding (2.5e-6 measured)
    assert abs(E_sd - E_rk) <= 1e-5 * abs(E_rk), (E_sd, E_rk)
    assert steps < 7 * attempts / 5


def test_masked_cells_stay_fixed_on_gpu():
    mesh = synth.Mesh(6, 5, 1, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, Ku=2e5, H=(3e4, 0, 0), precession=0, demag=1)
    Ms_cells = np.full(mesh.shape, 8e5)
    Ms_cells[0, 2, 3] = 0.0
    sim = synth.Sim(mesh, mat, synth.random_state(4, mesh), Ms_cells)
    ctx = make_ctx("f64", [sim])
    ctx.set_m(sim.m0.ravel())
    ctx.minimize(0.0, max_steps=20)
    m = ctx.get_m(0).reshape(3, *mesh.shape)
    assert np.array_equal(m[:, 0, 2, 3], sim.m0[:, 0, 2, 3])
    Ms = F.ms_array(mesh, mat, Ms_cells)
    Nt = D.mesh_tensor(mesh)
    m_ref, _ = SD.minimize(lambda y: F.h_eff(mesh, mat, y, Ms, Nt, "fft"), sim.m0.copy(), mat, Ms, max_steps=20)
    assert np.abs(m - m_ref).max() < 1e-8
