"""Pins for oracle.minimize: the paper's update equation, a closed-form minimum,
agreement with the damped RK45 relaxation (no GPU)."""
import numpy as np

import synth
from oracle import demag as D
from oracle import fields as F
from oracle import integrate as I
from oracle import minimize as SD


def _cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def test_update_solves_the_implicit_midpoint_step_and_keeps_the_norm():
    """m' = m - tau (m + m')/2 x f with f = m x H, and |m'| = |m| (Sec. 'Steepest descent')."""
    rng = np.random.default_rng(5)
    m = rng.standard_normal((3, 7, 5))
    m /= np.sqrt((m * m).sum(axis=0))[None]
    H = rng.standard_normal((3, 7, 5)) * 1e5
    f = _cross(m, H)
    g = _cross(m, f)
    for tau in (1e-7, 3e-6, 4e-5):                 # tau |f| from ~0.01 to a few radians
        m1 = SD.update(m, f, g, tau)
        resid = m1 - m + tau * _cross(0.5 * (m + m1), f)
        assert np.abs(resid).max() < 1e-14
        assert np.abs(np.sqrt((m1 * m1).sum(axis=0)) - 1.0).max() < 1e-14
    # g is the descent direction: to first order in tau |f| the change is -tau g
    # (the next term, -(tau |f|)^2 m / 2, is ~1e-4 of it at tau |f| ~ 2e-4)
    tau = 1e-9
    m1 = SD.update(m, f, g, tau)
    assert np.abs((m1 - m) + tau * g).max() < 1e-3 * np.abs(tau * g).max()


def test_macrospin_relaxes_to_the_stoner_wohlfarth_angle():
    """Easy axis z, field along x: sin(theta) = mu0 Ms H / (2 Ku) below the anisotropy field."""
    mesh = synth.Mesh(1, 1, 1, 2e-9, 2e-9, 2e-9)
    Ku, Ms0 = 5e5, 8e5
    HK = 2 * Ku / (F.MU0 * Ms0)
    mat = synth.Material(Ms=Ms0, Ku=Ku, u=(0, 0, 1), H=(0.3 * HK, 0, 0), alpha=0.5, precession=0, demag=0)
    Ms = F.ms_array(mesh, mat)
    m0 = synth.uniform_state(mesh, (0.2, 0.1, 1.0))
    m, st = SD.minimize(lambda y: F.h_eff(mesh, mat, y, Ms), m0, mat, Ms, max_dmdt=1.0, max_steps=500)
    assert st.converged, st.last_maxdmdt
    assert abs(m[0].item() - 0.3) < 1e-8
    assert abs(m[1].item()) < 1e-8
    assert abs(m[2].item() - np.sqrt(1 - 0.09)) < 1e-8
    assert st.k < 100                               # BB steps: far fewer than damped dynamics


def test_film_minimum_matches_the_damped_relaxation():
    """Same start, same minimum: the steepest-descent result has the energy of the
    RK45 relaxation with precession off (which needs ~30x more right-hand sides and
    still sits above the stopping threshold: 2 nm exchange modes make it stiff)."""
    mesh = synth.Mesh(12, 10, 1, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, Ku=5e5, u=(0, 0, 1), H=(5e4, 0, 2e4), alpha=0.5,
                         precession=0, demag=1)
    Ms = F.ms_array(mesh, mat)
    Nt = D.mesh_tensor(mesh)
    m0 = synth.tilt(synth.uniform_state(mesh, (0, 0, 1)), 3, 0.2)
    field = lambda y: F.h_eff(mesh, mat, y, Ms, Nt, "fft")
    m_sd, st = SD.minimize(field, m0, mat, Ms, max_dmdt=1e4, max_steps=2000)
    assert st.converged and st.k < 400, (st.k, st.last_maxdmdt)
    f = lambda y: F.rhs(mesh, mat, y, Ms, Nt, "fft")[0]
    m_rk, st_rk = I.run(f, m0.copy(), 1e-6, max_dmdt=1e6, max_steps=3000)
    assert st_rk.last_maxdmdt < 1e7
    E_sd = F.energies(mesh, mat, m_sd, Ms, Nt, "fft")["total"]
    E_rk = F.energies(mesh, mat, m_rk, Ms, Nt, "fft")["total"]
    assert abs(E_sd - E_rk) <= 1e-9 * abs(E_rk)
    assert np.abs(m_sd - m_rk).max() < 1e-4
    assert np.abs(np.sqrt((m_sd ** 2).sum(axis=0)) - 1.0).max() < 1e-13


def test_random_start_settles_into_a_minimum():
    """From random directions (exchange-dominated, non-convex) the capped steps settle:
    the run converges and ends far below the start energy, with every cell turned
    by at most ~1 rad a step."""
    mesh = synth.Mesh(16, 12, 1, 2.5e-9, 2.5e-9, 3e-9)
    mat = synth.Material(Ms=8.6e5, A=1.3e-11, H=(7958.0, 0, 0), alpha=0.5, precession=1, demag=1)
    Ms = F.ms_array(mesh, mat)
    Nt = D.mesh_tensor(mesh)
    m0 = synth.random_state(11, mesh)
    field = lambda y: F.h_eff(mesh, mat, y, Ms, Nt, "fft")
    E0 = F.energies(mesh, mat, m0, Ms, Nt, "fft")["total"]
    m, st = SD.minimize(field, m0, mat, Ms, max_dmdt=1e7, max_steps=4000)
    assert st.converged, (st.k, st.last_maxdmdt)
    E = F.energies(mesh, mat, m, Ms, Nt, "fft")["total"]
    assert E < 0.01 * E0
    g = st.g_prev
    assert st.tau * np.sqrt((g * g).sum(axis=0)).max() <= SD.MAX_TURN * (1 + 1e-12)


def test_masked_cells_do_not_move():
    mesh = synth.Mesh(4, 3, 1, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, Ku=2e5, H=(3e4, 0, 0), precession=0, demag=0)
    Ms_cells = np.full(mesh.shape, 8e5)
    Ms_cells[0, 1, 2] = 0.0
    Ms = F.ms_array(mesh, mat, Ms_cells)
    m0 = synth.random_state(4, mesh)
    m, st = SD.minimize(lambda y: F.h_eff(mesh, mat, y, Ms), m0, mat, Ms, max_steps=20)
    assert np.array_equal(m[:, 0, 1, 2], m0[:, 0, 1, 2])
