"""Pins for oracle.fields: closed forms and energy-gradient consistency (no GPU)."""
import math

import numpy as np
import pytest

import synth
from oracle import demag as D
from oracle import fields as F


def test_spin_spiral_exchange_closed_form():
    nx, ny, nz = 24, 3, 2
    dx = 2e-9
    mesh = synth.Mesh(nx, ny, nz, dx, 3e-9, 1e-9)
    A, Ms = 1.3e-11, 8e5
    mat = synth.Material(Ms=Ms, A=A, demag=0)
    k = 2 * math.pi / (11 * dx)
    x = np.arange(nx) * dx
    m = np.zeros((3, nz, ny, nx))
    m[0] = np.cos(k * x)
    m[1] = np.sin(k * x)
    Msa = F.ms_array(mesh, mat)
    E = F.energies(mesh, mat, m, Msa)["exchange"]
    V = dx * 3e-9 * 1e-9
    expect = (nx - 1) * ny * nz * V * 2 * A * (1 - math.cos(k * dx)) / dx ** 2
    assert abs(E - expect) < 1e-12 * expect
    H = F.h_exchange(mesh, mat, m, Msa)
    interior = (2 * A / (F.MU0 * Ms)) * (2 * math.cos(k * dx) - 2) / dx ** 2 * m[:, :, :, 5:-5]
    np.testing.assert_allclose(H[:, :, :, 5:-5], interior, rtol=0, atol=1e-9 * np.abs(interior).max())


def test_cycloid_dmi_closed_form():
    nx, ny, nz = 30, 2, 1
    dx = 1e-9
    mesh = synth.Mesh(nx, ny, nz, dx, 1e-9, 0.5e-9)
    Dm, Ms = 3e-3, 5.8e5
    mat = synth.Material(Ms=Ms, D=Dm, dmi=1, demag=0)
    k = 2 * math.pi / (17 * dx)
    x = np.arange(nx) * dx
    m = np.zeros((3, nz, ny, nx))
    m[0] = np.sin(k * x)
    m[2] = np.cos(k * x)
    E = F.energies(mesh, mat, m, F.ms_array(mesh, mat))["dmi"]
    V = dx * 1e-9 * 0.5e-9
    expect = -(nx - 1) * ny * nz * V * Dm * math.sin(k * dx) / dx
    assert abs(E - expect) < 1e-12 * abs(expect)


def test_cubic_energy_gap_100_111():
    mesh = synth.Mesh(1, 1, 1, 3e-9, 3e-9, 3e-9)
    K1 = 4.8e4
    mat = synth.Material(Ms=1.7e6, Kc=-K1 / 2, demag=0)
    V = 27e-27
    Msa = F.ms_array(mesh, mat)
    e100 = F.energies(mesh, mat, synth.uniform_state(mesh, (1, 0, 0)), Msa)["cubic"]
    e111 = F.energies(mesh, mat, synth.uniform_state(mesh, (1, 1, 1)), Msa)["cubic"]
    assert abs((e111 - e100) / V - K1 / 3) < 1e-9 * K1


TERMS = ["exchange", "dmi", "uniaxial", "cubic", "zeeman", "demag"]


@pytest.mark.parametrize("masked", [False, True])
def test_fields_are_energy_gradients(masked):
    """H_term,i = -(1/(mu0 Ms_i V)) dE_term/dm_i by central differences."""
    mesh = synth.Mesh(6, 5, 3, 2e-9, 2.5e-9, 1.5e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, D=3e-3, dmi=1, Ku=5e5, u=(0.3, 0.4, 0.866), Kc=1e4,
                         H=(1e4, -2e4, 3e4), alpha=0.3)
    m = synth.random_state(7, mesh)
    Ms = F.ms_array(mesh, mat)
    if masked:
        Ms = Ms.copy()
        Ms[1, 2, 2] = 0.0
        Ms[0, 0, :2] = 0.0
        Ms[2, 4, 5] = 3e5
    Nt = D.mesh_tensor(mesh)
    H = F.field_terms(mesh, mat, m, Ms, Nt, "direct")
    V = mesh.dx * mesh.dy * mesh.dz
    h = 1e-6
    for term in TERMS:
        scale = np.abs(H[term]).max()
        for (c, iz, iy, ix) in [(0, 1, 2, 3), (1, 0, 0, 3), (2, 2, 4, 5), (0, 2, 3, 1), (1, 1, 2, 1)]:
            if Ms[iz, iy, ix] == 0:
                continue
            mp = m.copy(); mp[c, iz, iy, ix] += h
            mm = m.copy(); mm[c, iz, iy, ix] -= h
            g = (F.energies(mesh, mat, mp, Ms, Nt, "direct")[term]
                 - F.energies(mesh, mat, mm, Ms, Nt, "direct")[term]) / (2 * h)
            Hn = -g / (F.MU0 * Ms[iz, iy, ix] * V)
            assert abs(Hn - H[term][c, iz, iy, ix]) < 1e-6 * scale, (term, c, iz, iy, ix)


def test_masked_cells_carry_no_field_or_torque():
    mesh = synth.Mesh(5, 4, 2, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, D=3e-3, dmi=1, Ku=5e5, H=(1e4, 0, 0))
    Ms = F.ms_array(mesh, mat).copy()
    Ms[0, 1, 1] = 0.0
    m = synth.random_state(3, mesh)
    dmdt, H = F.rhs(mesh, mat, m, Ms, method="direct")
    assert np.all(H[:, 0, 1, 1] == 0) and np.all(dmdt[:, 0, 1, 1] == 0)


def test_ll_torque_properties():
    mesh = synth.Mesh(4, 3, 2, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, Ku=5e5, H=(1e4, 2e4, 0), alpha=0.2)
    Ms = F.ms_array(mesh, mat)
    m = synth.random_state(5, mesh)
    dmdt, H = F.rhs(mesh, mat, m, Ms, method="direct")
    assert np.abs((dmdt * m).sum(axis=0)).max() < 1e-12 * np.abs(dmdt).max()
    # |dm/dt| = gamma/(1+a^2) * sqrt(1+a^2) |m x H| for unit m
    mxH = F._cross(m, H)
    expect = mat.gamma / math.sqrt(1 + mat.alpha ** 2) * np.sqrt((mxH ** 2).sum(axis=0))
    np.testing.assert_allclose(np.sqrt((dmdt ** 2).sum(axis=0)), expect, rtol=1e-12)
    # precession off leaves only the damping term, which lowers the Zeeman-like energy
    mat0 = synth.Material(**{**mat.__dict__, "precession": 0})
    d0 = F.ll_rhs(mat0, m, H, Ms)
    assert ((d0 * H).sum(axis=0) >= -1e-9 * np.abs(d0 * H).max()).all()
