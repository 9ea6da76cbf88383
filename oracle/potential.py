"""Demagnetising field through the magnetic scalar potential (oracle, FP64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Paper: Sec. "Magnetostatic energy" -- with the scalar potential the three
inverse transforms of the FFT demag reduce to one (the remark after Eq. 8;
the paper cites the method and gives no formulas).  Reading used here:

* potential at cell centres, u_i = sum_j S(r_i - r_j) . M_j, with S the exact
  potential of one uniformly magnetised cell: for unit magnetisation along x
  the cell carries charge +1 on its +x face and -1 on its -x face, so
  S_x(R) = (1/4 pi) [P(X - dx/2; Y, Z) - P(X + dx/2; Y, Z)], P(a; Y, Z) the
  potential of a unit-density dy x dz rectangle at normal distance a (closed
  form: the mixed antiderivative F(y, z) = y ln(z + r) + z ln(y + r) -
  a atan(y z / (a r)) of 1/r, r = sqrt(a^2 + y^2 + z^2), at the four corners);
  S_y, S_z by permuting the axes;
* field H_d = -grad u by central differences at every cell, with u taken at
  the cell centres one step outside the mesh where a neighbour lies outside
  (the potential is defined everywhere), so the convolution produces u on
  the mesh extended by one cell on each side of every axis with more than
  zero cells (a single-plane film gets the planes above and below).

This is a different discretisation from the Newell cell-averaged field of
oracle.demag (point potential, difference quotient), so the two fields agree
in the interior of a smooth magnetisation to O(Delta^2) and differ at the
surfaces; test_oracle_potential.py reports the difference.

* potential_kernel   S(R) for offsets R (closed form)
* potential_direct   u on the extended grid by the direct sum (small meshes)
* potential_fft      the same by zero-padded FFT convolution (padding 2n + 2)
* field_from_potential   -grad u by central differences
* h_demag_potential  the whole field (direct or FFT)

Parity: pinned by tests/test_oracle_potential.py -- the closed form against
numerical quadrature of the cell integral; S(0) = 0 and the parities; the
superposition identity (the cells of a box with uniform M sum exactly to the
potential of the whole box: the inner face charges cancel); the far field
against the point dipole; direct sum against FFT; the centre field of a
uniformly magnetised cube against -M/3 at second order in the cell size.
"""
from __future__ import annotations

import math

import numpy as np


def _log_sum(z, r, rest2):
    """ln(z + r) with r = sqrt(z^2 + rest2), rest2 > 0; for z < 0 through
    z + r = rest2 / (r - z), which does not cancel."""
    return np.where(z >= 0, np.log(np.abs(z) + r), np.log(rest2) - np.log(r + np.abs(z)))


def _corner(a, y, z):
    """F(y, z) with d^2F/(dy dz) = 1/sqrt(a^2 + y^2 + z^2) (a != 0)."""
    a, y, z = np.broadcast_arrays(np.asarray(a, float), np.asarray(y, float), np.asarray(z, float))
    r = np.sqrt(a * a + y * y + z * z)
    return (y * _log_sum(z, r, a * a + y * y) + z * _log_sum(y, r, a * a + z * z)
            - a * np.arctan(y * z / (a * r)))


def rect_potential(a, Y, Z, dy, dz):
    """Integral of 1/|r - s| over s in the rectangle [Y - dy/2, Y + dy/2] x [Z - dz/2,
    Z + dz/2] of the plane at normal distance a (r at the origin of the plane)."""
    a = np.asarray(a, float)
    y1, y2 = -Y - dy / 2.0, -Y + dy / 2.0
    z1, z2 = -Z - dz / 2.0, -Z + dz / 2.0
    return _corner(a, y2, z2) - _corner(a, y1, z2) - _corner(a, y2, z1) + _corner(a, y1, z1)


def potential_kernel(X, Y, Z, dx, dy, dz):
    """S(R) = (S_x, S_y, S_z): potential at offset R = (X, Y, Z) from the centre of a
    dx x dy x dz cell magnetised with unit magnetisation along x, y or z; shape
    (3,) + X.shape."""
    X, Y, Z = np.broadcast_arrays(np.asarray(X, float), np.asarray(Y, float), np.asarray(Z, float))
    c = 1.0 / (4.0 * math.pi)
    # the rectangle is centred at the cell's transverse offset (0, 0): the target sits
    # at transverse position (Y, Z) relative to it
    sx = c * (rect_potential(X - dx / 2, Y, Z, dy, dz) - rect_potential(X + dx / 2, Y, Z, dy, dz))
    sy = c * (rect_potential(Y - dy / 2, X, Z, dx, dz) - rect_potential(Y + dy / 2, X, Z, dx, dz))
    sz = c * (rect_potential(Z - dz / 2, X, Y, dx, dy) - rect_potential(Z + dz / 2, X, Y, dx, dy))
    return np.stack([sx, sy, sz])


def potential_direct(mesh, M):
    """u on the extended grid (nz + 2, ny + 2, nx + 2) by the direct sum; M (3, nz, ny, nx)
    in A/m; index 0 along each axis is the cell centre one step below the mesh."""
    nz, ny, nx = mesh.nz, mesh.ny, mesh.nx
    src = np.argwhere(np.abs(M).sum(axis=0) > 0)          # (k, j, i) of magnetised cells
    kz, jy, ix = np.meshgrid(np.arange(-1, nz + 1), np.arange(-1, ny + 1), np.arange(-1, nx + 1), indexing="ij")
    u = np.zeros(kz.shape)
    for (k, j, i) in src:
        S = potential_kernel((ix - i) * mesh.dx, (jy - j) * mesh.dy, (kz - k) * mesh.dz, mesh.dx, mesh.dy, mesh.dz)
        u += S[0] * M[0, k, j, i] + S[1] * M[1, k, j, i] + S[2] * M[2, k, j, i]
    return u


def potential_fft(mesh, M):
    """The same u by circular convolution on a grid padded to 2n + 2 along every axis
    (the extended grid's n + 2 points need offsets -n .. n, 2n + 1 of them)."""
    nz, ny, nx = mesh.nz, mesh.ny, mesh.nx
    P = (2 * nz + 2, 2 * ny + 2, 2 * nx + 2)
    off = [np.arange(-n, n + 1) for n in (nz, ny, nx)]          # the 2n + 1 offsets
    Kz, Ky, Kx = np.meshgrid(*off, indexing="ij")
    S = np.zeros((3,) + P)                                     # position n + 1 stays empty
    pos = [o % p for o, p in zip(off, P)]
    S[(slice(None),) + np.ix_(*pos)] = potential_kernel(Kx * mesh.dx, Ky * mesh.dy, Kz * mesh.dz,
                                                        mesh.dx, mesh.dy, mesh.dz)
    Sk = np.fft.fftn(S, axes=(1, 2, 3))
    Mk = np.fft.fftn(M, s=P, axes=(1, 2, 3))
    u = np.real(np.fft.ifftn((Sk * Mk).sum(axis=0)))
    # extended index e = -1 .. n along each axis sits at circular position e mod P
    idx = [np.arange(-1, n + 1) % p for n, p in zip((nz, ny, nx), P)]
    return u[np.ix_(*idx)]


def field_from_potential(mesh, u):
    """H = -grad u by central differences at the mesh cells (u on the extended grid)."""
    H = np.empty((3, mesh.nz, mesh.ny, mesh.nx))
    H[0] = -(u[1:-1, 1:-1, 2:] - u[1:-1, 1:-1, :-2]) / (2.0 * mesh.dx)
    H[1] = -(u[1:-1, 2:, 1:-1] - u[1:-1, :-2, 1:-1]) / (2.0 * mesh.dy)
    H[2] = -(u[2:, 1:-1, 1:-1] - u[:-2, 1:-1, 1:-1]) / (2.0 * mesh.dz)
    return H


def h_demag_potential(mesh, M, method="auto"):
    """Demag field (A/m) of M (3, nz, ny, nx) through the scalar potential."""
    if method == "auto":
        method = "direct" if mesh.ncells <= 512 else "fft"
    u = potential_direct(mesh, M) if method == "direct" else potential_fft(mesh, M)
    return field_from_potential(mesh, u)
