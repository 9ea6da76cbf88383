"""Pins for oracle.potential (no GPU): the scalar-potential demag field.

The kernel is pinned to numerical quadrature of its defining cell integral and to
the point dipole far away; the superposition of a box's cells to the closed form of
the whole box (exact: inner face charges cancel); the FFT convolution to the direct
sum; the centre field of a uniformly magnetised cube to -M/3 at second order in the
cell size.  The last test records how far this discretisation lies from the Newell
cell-averaged field (Sec. "Magnetostatic energy", Eq. 8) on the workloads' kinds of
mesh.
"""
import math

import numpy as np
import pytest

import synth
from oracle import demag as D
from oracle import potential as P

D3 = (2e-9, 3e-9, 1.5e-9)


def _quad(R, d, n=48):
    """(1/4 pi) int_cell (R - s)/|R - s|^3 d^3 s by n-point Gauss-Legendre per axis."""
    x, w = np.polynomial.legendre.leggauss(n)
    X, Y, Z = R[0] - 0.5 * d[0] * x, R[1] - 0.5 * d[1] * x, R[2] - 0.5 * d[2] * x
    XX, YY, ZZ = np.meshgrid(X, Y, Z, indexing="ij")
    W = np.einsum("i,j,k->ijk", w, w, w) * d[0] * d[1] * d[2] / 8.0
    r3 = (XX ** 2 + YY ** 2 + ZZ ** 2) ** 1.5
    return np.array([(W * XX / r3).sum(), (W * YY / r3).sum(), (W * ZZ / r3).sum()]) / (4.0 * math.pi)


@pytest.mark.parametrize("ijk", [(2, 0, 0), (1, 1, 0), (3, -2, 1), (0, 0, 1), (-5, 4, -3), (0, -1, -1)])
def test_kernel_matches_quadrature(ijk):
    R = [ijk[a] * D3[a] for a in range(3)]
    s = P.potential_kernel(*R, *D3)
    q = _quad(R, D3)
    assert np.abs(s - q).max() <= 1e-10 * np.abs(q).max()


def test_kernel_centre_parities_and_axis_permutation():
    assert np.abs(P.potential_kernel(0.0, 0.0, 0.0, *D3)).max() == 0.0
    R = np.array([3.0, 1.0, -2.0]) * np.array(D3)
    s = P.potential_kernel(*R, *D3)
    # S_x odd in X, even in Y and Z
    assert np.isclose(P.potential_kernel(-R[0], R[1], R[2], *D3)[0], -s[0], rtol=1e-13)
    assert np.isclose(P.potential_kernel(R[0], -R[1], R[2], *D3)[0], s[0], rtol=1e-13)
    assert np.isclose(P.potential_kernel(R[0], R[1], -R[2], *D3)[0], s[0], rtol=1e-13)
    # S_y(X, Y, Z; dx, dy, dz) = S_x(Y, X, Z; dy, dx, dz)
    t = P.potential_kernel(R[1], R[0], R[2], D3[1], D3[0], D3[2])
    assert np.isclose(t[0], s[1], rtol=1e-13) and np.isclose(t[1], s[0], rtol=1e-13)


def test_box_superposition_is_exact():
    """A 3 x 2 x 4 block of cells with uniform M: the cells' potentials add up to the
    potential of one 3dx x 2dy x 4dz cell (the charges of the inner faces cancel)."""
    nb = (3, 2, 4)
    M = np.array([0.3, -0.7, 0.6]) * 8e5
    cx = [(i - (nb[a] - 1) / 2.0) * D3[a] for a, n in enumerate(nb) for i in range(n)]
    centres = [np.array([(i - (nb[0] - 1) / 2.0) * D3[0], (j - (nb[1] - 1) / 2.0) * D3[1],
                         (k - (nb[2] - 1) / 2.0) * D3[2]])
               for i in range(nb[0]) for j in range(nb[1]) for k in range(nb[2])]
    big = [nb[a] * D3[a] for a in range(3)]
    del cx
    for r in ([0.0, 0.5 * D3[1], 0.5 * D3[2]], [2 * D3[0], -1.5 * D3[1], 0.5 * D3[2]],
              [-4 * D3[0], 2.5 * D3[1], -3.5 * D3[2]], [1 * D3[0], 0.5 * D3[1], 1.5 * D3[2]]):
        r = np.array(r)
        u = sum(P.potential_kernel(*(r - c), *D3) @ M for c in centres)
        ub = P.potential_kernel(*r, *big) @ M
        assert abs(u - ub) <= 1e-11 * abs(ub)


def test_far_field_is_the_point_dipole():
    V = D3[0] * D3[1] * D3[2]
    for k in (20.0, 40.0):
        R = np.array([0.6, -0.5, 0.3]) * k * max(D3)
        s = P.potential_kernel(*R, *D3)
        dip = V * R / (4 * math.pi * np.linalg.norm(R) ** 3)
        rel = np.abs(s - dip).max() / np.abs(dip).max()
        assert rel < 2.0 * (max(D3) / np.linalg.norm(R)) ** 2


@pytest.mark.parametrize("dims", [(5, 4, 3), (6, 5, 1), (1, 7, 2)])
def test_direct_sum_equals_fft(dims):
    mesh = synth.Mesh(*dims, *D3)
    M = synth.random_state(21, mesh) * 8e5
    M[:, 0, 0, 0] = 0.0                                  # a hole
    ud = P.potential_direct(mesh, M)
    uf = P.potential_fft(mesh, M)
    assert ud.shape == (dims[2] + 2, dims[1] + 2, dims[0] + 2)
    assert np.abs(ud - uf).max() <= 1e-12 * np.abs(ud).max()


def test_cube_centre_field_converges_to_minus_m_over_three():
    """Uniformly magnetised cube of n^3 cells, central difference at the centre cell:
    -M/3 (the point field at the centre of a cube) plus an O(1/n^2) error."""
    M = np.array([0.0, 0.0, 1e6])
    err = []
    for n in (5, 9, 17):
        d = 1e-9
        mesh = synth.Mesh(n, n, n, d, d, d)
        c = n // 2
        # u at the centre's z neighbours: by the superposition identity, the potential of
        # the whole cube
        up = P.potential_kernel(0.0, 0.0, d, n * d, n * d, n * d) @ M
        dn = P.potential_kernel(0.0, 0.0, -d, n * d, n * d, n * d) @ M
        Hz = -(up - dn) / (2 * d)
        err.append(abs(Hz + M[2] / 3.0) / (M[2] / 3.0))
        if n == 5:                                       # and the same through the FFT convolution
            H = P.h_demag_potential(mesh, np.broadcast_to(M[:, None, None, None], (3, n, n, n)).copy(), "fft")
            assert abs(H[2, c, c, c] - Hz) <= 1e-11 * M[2]
    assert err[2] < err[1] < err[0] and err[2] < 5e-3
    assert 2.5 < err[1] / err[2] < 5.0                   # (17/9)^2 = 3.6: second order


def test_difference_from_the_newell_field():
    """The scalar-potential field against the Newell cell-averaged field (the method's
    result on the workloads' kinds of mesh): a uniformly magnetised 16^3 cube and a
    16x16x1 film with M in-plane and out of plane.  Deep inside the cube the two agree
    to a fraction of a percent; at the surfaces and in the single-plane film they differ
    by several percent of Ms, far above the FP32 field tolerance (1e-5): the methods are
    different discretisations, not two evaluations of one sum."""
    rows = {}
    for name, dims, mdir in (("cube", (16, 16, 16), (0, 0, 1)), ("film_perp", (16, 16, 1), (0, 0, 1)),
                             ("film_inplane", (16, 16, 1), (1, 0, 0))):
        mesh = synth.Mesh(*dims, 2e-9, 2e-9, 2e-9)
        Ms = 8e5
        M = Ms * synth.uniform_state(mesh, mdir)
        Hn = D.demag_fft(mesh, M)
        Hp = P.h_demag_potential(mesh, M, "fft")
        diff = np.sqrt(((Hn - Hp) ** 2).sum(0)) / Ms
        rows[name] = diff
    inner = rows["cube"][4:-4, 4:-4, 4:-4]
    assert inner.max() < 5e-3
    assert rows["cube"].max() > 1e-2                     # surfaces
    assert rows["film_perp"].max() > 1e-2
    assert rows["film_inplane"].max() > 1e-3
