"""Demagnetising field as a discrete convolution (oracle, FP64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Paper: Sec. "Magnetostatic energy", Eq. 8: H_d,i = -sum_j N_{i-j} M_j with
M_j = Ms_j m_j, and the FFT evaluation of the same sum (three forward and
three inverse transforms, zero padding).

* demag_direct   the sum of Eq. 8 written out, O(N^2); for small meshes.
* demag_direct_at  the same sum for a list of target cells only.
* demag_fft      the same sum by circular convolution on a grid padded to
                 2n along every axis with n > 1 (numpy's FFT is the only
                 library step).

Parity: pinned by tests/test_oracle_demag.py (direct sum == FFT to 1e-12,
the uniform-box sum rule, thin-film limit, reciprocity of the pair
tensor).  N comes from oracle.newell.mesh_tensor.
"""
from __future__ import annotations

import numpy as np

from . import newell


def mesh_tensor(mesh):
    return newell.mesh_tensor(mesh.nx, mesh.ny, mesh.nz, mesh.dx, mesh.dy, mesh.dz)


def _window(Ntab, mesh, iz, iy, ix):
    """N(r_i - r_j) for target cell i and all sources j: shape (6, nz, ny, nx)."""
    nz, ny, nx = mesh.nz, mesh.ny, mesh.nx
    w = Ntab[:, iz:iz + nz, iy:iy + ny, ix:ix + nx]
    return w[:, ::-1, ::-1, ::-1]


def _apply(w, M):
    xx, yy, zz, xy, xz, yz = (w[c] for c in range(6))
    hx = -(xx * M[0] + xy * M[1] + xz * M[2]).sum()
    hy = -(xy * M[0] + yy * M[1] + yz * M[2]).sum()
    hz = -(xz * M[0] + yz * M[1] + zz * M[2]).sum()
    return hx, hy, hz


def demag_direct(mesh, M, Ntab=None):
    """H_d for every cell by the direct sum.  M: (3, nz, ny, nx) in A/m."""
    if Ntab is None:
        Ntab = mesh_tensor(mesh)
    H = np.zeros_like(M)
    for iz in range(mesh.nz):
        for iy in range(mesh.ny):
            for ix in range(mesh.nx):
                H[:, iz, iy, ix] = _apply(_window(Ntab, mesh, iz, iy, ix), M)
    return H


def demag_direct_at(mesh, M, cells, Ntab=None):
    """H_d at the listed cells [(iz, iy, ix), ...] by the direct sum; shape (3, K)."""
    if Ntab is None:
        Ntab = mesh_tensor(mesh)
    return np.array([_apply(_window(Ntab, mesh, *c), M) for c in cells]).T


def padded(n):
    return 2 * n if n > 1 else 1


def demag_fft(mesh, M, Ntab=None):
    """H_d for every cell by zero-padded circular convolution (padding 2n)."""
    if Ntab is None:
        Ntab = mesh_tensor(mesh)
    nz, ny, nx = mesh.nz, mesh.ny, mesh.nx
    P = (padded(nz), padded(ny), padded(nx))
    # place offsets -(n-1)..(n-1) circularly
    Nc = np.zeros((6,) + P)
    iz = np.r_[np.arange(nz), np.arange(-nz + 1, 0)] % P[0]
    iy = np.r_[np.arange(ny), np.arange(-ny + 1, 0)] % P[1]
    ix = np.r_[np.arange(nx), np.arange(-nx + 1, 0)] % P[2]
    src_z = np.r_[np.arange(nz), np.arange(-nz + 1, 0)] + nz - 1
    src_y = np.r_[np.arange(ny), np.arange(-ny + 1, 0)] + ny - 1
    src_x = np.r_[np.arange(nx), np.arange(-nx + 1, 0)] + nx - 1
    Nc[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]] = \
        Ntab[:, src_z[:, None, None], src_y[None, :, None], src_x[None, None, :]]
    Nk = np.fft.rfftn(Nc, axes=(1, 2, 3))
    Mk = np.fft.rfftn(M, s=P, axes=(1, 2, 3))
    xx, yy, zz, xy, xz, yz = Nk
    Hk = np.stack([xx * Mk[0] + xy * Mk[1] + xz * Mk[2],
                   xy * Mk[0] + yy * Mk[1] + yz * Mk[2],
                   xz * Mk[0] + yz * Mk[1] + zz * Mk[2]])
    H = -np.fft.irfftn(Hk, s=P, axes=(1, 2, 3))
    return H[:, :nz, :ny, :nx].copy()
