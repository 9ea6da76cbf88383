"""Pins for oracle.demag (no GPU)."""
import numpy as np
import pytest

import synth
from oracle import demag as D
from oracle import newell as nw


def test_direct_sum_equals_fft_convolution():
    mesh = synth.Mesh(7, 5, 3, 2e-9, 2.5e-9, 1.5e-9)
    M = synth.random_state(11, mesh) * 8e5
    Nt = D.mesh_tensor(mesh)
    a = D.demag_direct(mesh, M, Nt)
    b = D.demag_fft(mesh, M, Nt)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_direct_at_matches_full_direct():
    mesh = synth.Mesh(6, 4, 2, 1e-9, 1e-9, 1e-9)
    M = synth.random_state(12, mesh) * 5e5
    Nt = D.mesh_tensor(mesh)
    full = D.demag_direct(mesh, M, Nt)
    cells = [(0, 0, 0), (1, 3, 5), (1, 2, 2)]
    got = D.demag_direct_at(mesh, M, cells, Nt)
    for k, c in enumerate(cells):
        np.testing.assert_allclose(got[:, k], full[:, c[0], c[1], c[2]], rtol=0, atol=1e-12 * np.abs(full).max())


@pytest.mark.parametrize("n", [2, 5, 8])
def test_uniform_cube_mean_field_is_minus_third(n):
    """Sum rule: for uniform M in a cube the mean demag field is exactly -M/3."""
    mesh = synth.Mesh(n, n, n, 1e-9, 1e-9, 1e-9)
    Ms = 1e6
    m = synth.uniform_state(mesh, (0.3, -0.5, 0.8))
    H = D.demag_fft(mesh, m * Ms)
    mean = H.reshape(3, -1).mean(axis=1)
    np.testing.assert_allclose(mean, -m[:, 0, 0, 0] * Ms / 3.0, rtol=0, atol=1e-12 * Ms)


def test_uniform_box_mean_field_matches_box_factor():
    mesh = synth.Mesh(12, 6, 2, 2e-9, 2e-9, 1e-9)
    Ms = 7e5
    m = synth.uniform_state(mesh, (1.0, 1.0, 1.0))
    H = D.demag_fft(mesh, m * Ms)
    box = nw.as_matrix(nw.tensor_exact(0.0, 0.0, 0.0, 24e-9, 12e-9, 2e-9))
    expect = -box @ (m[:, 0, 0, 0] * Ms)
    np.testing.assert_allclose(H.reshape(3, -1).mean(axis=1), expect, rtol=0, atol=1e-11 * Ms)


def test_single_cell_is_self_term():
    mesh = synth.Mesh(1, 1, 1, 2e-9, 3e-9, 1e-9)
    M = np.array([1.0, 2.0, -3.0]).reshape(3, 1, 1, 1) * 1e5
    H = D.demag_direct(mesh, M)
    t = nw.as_matrix(nw.tensor_exact(0.0, 0.0, 0.0, 2e-9, 3e-9, 1e-9))
    np.testing.assert_allclose(H[:, 0, 0, 0], -t @ M[:, 0, 0, 0], rtol=1e-14)
