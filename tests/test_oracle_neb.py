"""Pins for oracle.neb: single-cell uniaxial chain vs Stoner-Wohlfarth energy (no GPU)."""
import numpy as np

import synth
from oracle import fields as F
from oracle import neb as NB


def test_single_cell_chain_relaxes_to_equal_angles_on_sw_profile():
    mesh = synth.Mesh(1, 1, 1, 3e-9, 3e-9, 3e-9)
    Ku, Ms0 = 5e5, 8e5
    H = 0.3 * 2 * Ku / (F.MU0 * Ms0)                 # h = 0.3 along the easy axis
    mat = synth.Material(Ms=Ms0, Ku=Ku, u=(0, 0, 1), H=(0, 0, H), alpha=0.5, precession=0, demag=0)
    Ms = F.ms_array(mesh, mat)
    n = 11
    up = synth.uniform_state(mesh, (0, 0, 1))
    dn = synth.uniform_state(mesh, (0, 0, -1))
    chain = synth.geodesic_chain(up, dn, n)
    for i in range(1, n - 1):
        chain[i] = synth.tilt(chain[i], 100 + i, 0.2)
    c, E, st = NB.relax(mesh, mat, Ms, chain, k_spring=1e5, rtol=1e-6, steps=600)
    assert np.array_equal(c[0], chain[0]) and np.array_equal(c[-1], chain[-1])
    assert np.abs(np.sqrt((c ** 2).sum(axis=1)) - 1).max() < 1e-14
    V = 27e-27
    th = np.linspace(0, np.pi, n)
    expect = -Ku * V * np.cos(th) ** 2 - F.MU0 * Ms0 * V * H * np.cos(th)
    assert np.abs(E - expect).max() < 1e-3 * Ku * V
    # barrier from the reversed end equals Ku V (1 - h)^2 at the interpolated maximum
    h = 0.3
    assert abs((E.max() - E[-1]) - Ku * V * (1 - h) ** 2) < 0.05 * Ku * V


def test_tangent_is_perpendicular_and_unit():
    mesh = synth.Mesh(3, 2, 1, 1e-9, 1e-9, 1e-9)
    a = synth.random_state(1, mesh)
    b = synth.random_state(2, mesh)
    chain = synth.geodesic_chain(a, b, 5)
    tau = NB.tangents(chain, np.array([0.0, 1.0, 3.0, 2.0, 0.5]))
    for i in range(1, 4):
        assert abs(np.sqrt((tau[i] ** 2).sum()) - 1) < 1e-14
        assert np.abs((tau[i] * chain[i]).sum(axis=0)).max() < 1e-14
