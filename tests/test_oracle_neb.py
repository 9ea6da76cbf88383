"""Pins for oracle.neb (no GPU): a single-cell uniaxial chain against the
Stoner-Wohlfarth energy, a two-particle chain against the closed-form energy
profile of its sequential minimum energy path, and the geodesic distance
against closed forms."""
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


def _sw_energy(Ku, V, h, th):
    """Stoner-Wohlfarth energy of one particle at angle th from the easy axis, field
    h H_K along the axis (mu0 Ms H = 2 Ku h)."""
    return -Ku * V * np.cos(th) ** 2 - 2 * Ku * V * h * np.cos(th)


def test_two_particle_chain_takes_the_sequential_path():
    """Two uncoupled single-domain particles reversing in a field along the easy axis: the
    minimum energy path turns one particle, then the other (through the intermediate
    minimum with one particle reversed), never both at once.  At equal geodesic spacing
    (path length 2 pi) image i at arc length s_i has E = e(min(s_i, pi)) + e(max(s_i - pi, 0))
    with e the Stoner-Wohlfarth energy; the highest image lies below the coherent
    (both at once) barrier."""
    mesh = synth.Mesh(2, 1, 1, 3e-9, 3e-9, 3e-9)
    Ku, Ms0, h = 5e5, 8e5, 0.3
    H = h * 2 * Ku / (F.MU0 * Ms0)
    mat = synth.Material(Ms=Ms0, Ku=Ku, u=(0, 0, 1), H=(0, 0, H), alpha=0.5, precession=0, demag=0)
    Ms = F.ms_array(mesh, mat)
    n = 13
    s = np.linspace(0, 2 * np.pi, n)
    chain = np.zeros((n, 3, 1, 1, 2))
    for i, si in enumerate(s):
        t1, t2 = min(si, np.pi), max(si - np.pi, 0.0)
        chain[i, :, 0, 0, 0] = [np.sin(t1) * np.cos(0.3), np.sin(t1) * np.sin(0.3), np.cos(t1)]
        chain[i, :, 0, 0, 1] = [np.sin(t2) * np.cos(1.1), np.sin(t2) * np.sin(1.1), np.cos(t2)]
        if 0 < i < n - 1:
            chain[i] = synth.tilt(chain[i], 200 + i, 0.15)
    c, E, st = NB.relax(mesh, mat, Ms, chain, k_spring=1e5, rtol=1e-6, steps=1500)
    V = 27e-27
    L = np.array([NB.geodesic_distance(c[i], c[i + 1]) for i in range(n - 1)])
    assert abs(L.sum() - 2 * np.pi) < 1e-6 and L.max() - L.min() < 1e-5
    expect = _sw_energy(Ku, V, h, np.minimum(s, np.pi)) + _sw_energy(Ku, V, h, np.maximum(s - np.pi, 0.0))
    assert np.abs(E - expect).max() < 1e-5 * Ku * V
    mid = c[(n - 1) // 2]
    assert abs(mid[2, 0, 0, 0] + 1) < 1e-6 and abs(mid[2, 0, 0, 1] - 1) < 1e-6
    top = 2 * _sw_energy(Ku, V, h, np.arccos(-h))          # both particles at their saddle
    assert E.max() < top - 0.5 * Ku * V


def test_geodesic_distance_closed_forms():
    """sqrt(sum over cells of theta^2): N cells each turned by theta are theta sqrt(N)
    apart; reversing every cell is pi sqrt(N); one turned cell alone counts theta."""
    mesh = synth.Mesh(4, 3, 2, 1e-9, 1e-9, 1e-9)
    N = mesh.ncells
    a = synth.random_state(3, mesh)
    th = 0.37
    # turn every cell by th about an axis perpendicular to it
    ref = np.broadcast_to(np.array([0.3, -0.5, 0.8])[:, None, None, None], a.shape)
    ax = F._cross(a, ref)
    ax = ax / np.sqrt((ax ** 2).sum(0))[None]
    b = a * np.cos(th) + F._cross(ax, a) * np.sin(th)
    assert abs(NB.geodesic_distance(a, b) - th * np.sqrt(N)) < 1e-12
    assert abs(NB.geodesic_distance(a, -a) - np.pi * np.sqrt(N)) < 1e-12
    one = a.copy()
    one[:, 1, 2, 3] = b[:, 1, 2, 3]
    assert abs(NB.geodesic_distance(a, one) - th) < 1e-12
