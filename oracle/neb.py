"""Geodesic nudged elastic band (oracle, FP64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Paper: Sec. "Miscellaneous" -- a chain of images between two fixed end
states is relaxed like LLG with the precession term switched off; the
effective field of each image also feels its neighbours through the
tangent, and only the part of the field perpendicular to the tangent is
kept.  The paper defers the details to a thesis that is not available, so
the published geodesic NEB (Bessarab, Uzdin & Jonsson, CPC 196, 335
(2015)) fills them in:

  * tangent: the energy-weighted upwind tangent of Henkelman & Jonsson
    (2000) built from tau+ = m_{i+1} - m_i and tau- = m_i - m_{i-1},
    projected cell by cell onto the tangent plane of m_i and normalised
    over the whole image;
  * distance between images: sqrt(sum over cells of theta^2), theta the
    angle between the two cells' unit vectors;
  * force (field units, A/m): F_i = H_i - (H_i . tau_i) tau_i
    + k (L_{i,i+1} - L_{i-1,i}) tau_i, with k in A/m per radian;
  * dynamics: dm_i/dt = -alpha g~ m_i x (m_i x F_i) for the free images,
    0 for the two end images; the whole chain is one state for the
    adaptive RK45 of oracle.integrate (a single h, the error is the max
    over all images).

Parity: pinned by tests/test_oracle_neb.py -- a single-cell uniaxial chain
(in a field along the axis) against the Stoner-Wohlfarth energy at equally
spaced angles, fixed ends and |m| = 1; a chain of two uncoupled particles
(a multi-cell image whose path turns one cell, then the other) against the
closed-form energy of every image at equal geodesic spacing, the path
length 2 pi and the intermediate minimum (this fails with the tangent
normalised per cell or a wrong spring sign); the geodesic distance against
theta sqrt(N) for N cells turned by theta.
"""
from __future__ import annotations

import numpy as np

from . import fields as F
from . import integrate as I


def _cross(a, b):
    return F._cross(a, b)


def geodesic_distance(ma, mb):
    c = _cross(ma, mb)
    s = np.sqrt((c * c).sum(axis=0))
    d = (ma * mb).sum(axis=0)
    th = np.arctan2(s, d)
    return float(np.sqrt((th * th).sum()))


def tangents(chain, energies):
    """Unit tangents for the free images (ends get zeros)."""
    n = chain.shape[0]
    tau = np.zeros_like(chain)
    for i in range(1, n - 1):
        tp = chain[i + 1] - chain[i]
        tm = chain[i] - chain[i - 1]
        Ep, E0, Em = energies[i + 1], energies[i], energies[i - 1]
        if Ep > E0 > Em:
            t = tp
        elif Ep < E0 < Em:
            t = tm
        else:
            dmax = max(abs(Ep - E0), abs(Em - E0))
            dmin = min(abs(Ep - E0), abs(Em - E0))
            t = tp * dmax + tm * dmin if Ep > Em else tp * dmin + tm * dmax
        m = chain[i]
        t = t - (t * m).sum(axis=0)[None] * m
        nrm = np.sqrt((t * t).sum())
        tau[i] = t / nrm if nrm > 0 else t
    return tau


def image_field_energy(mesh, mat, Ms, m, Ntab=None, method="auto"):
    """Effective field and total energy of one image."""
    return F.h_eff(mesh, mat, m, Ms, Ntab, method), F.energies(mesh, mat, m, Ms, Ntab, method)["total"]


def chain_forces(mat, Ms, chain, H, E, k_spring):
    """d(chain)/dt of the images 1..n-2 of `chain` (shape (n, 3, nz, ny, nx)) from their
    fields H[i] and the energies E of all n images; images 0 and n-1 get zeros (the
    chain's fixed ends, or neighbours owned by another process)."""
    n = chain.shape[0]
    tau = tangents(chain, E)
    L = [geodesic_distance(chain[i], chain[i + 1]) for i in range(n - 1)]
    gt = mat.gamma / (1.0 + mat.alpha ** 2)
    out = np.zeros_like(chain)
    for i in range(1, n - 1):
        Ht = float((H[i] * tau[i]).sum())
        Fi = H[i] - Ht * tau[i] + k_spring * (L[i] - L[i - 1]) * tau[i]
        m = chain[i]
        out[i] = -mat.alpha * gt * _cross(m, _cross(m, Fi)) * (Ms > 0)[None]
    return out


def chain_rhs(mesh, mat, Ms, chain, k_spring, Ntab=None, method="auto"):
    """d(chain)/dt and the image energies for a chain of shape (n, 3, nz, ny, nx)."""
    n = chain.shape[0]
    HE = [image_field_energy(mesh, mat, Ms, chain[i], Ntab, method) for i in range(n)]
    H = np.stack([h for h, _ in HE])
    E = np.array([e for _, e in HE])
    return chain_forces(mat, Ms, chain, H, E, k_spring), E


def relax(mesh, mat, Ms, chain, k_spring, rtol, steps, Ntab=None, method="auto"):
    """`steps` attempted RK45 steps of the whole chain; returns (chain, energies, stepper)."""
    st = I.Stepper(rtol=rtol)
    # the integrator wants components on axis 0: carry the chain as (3, n, ...)
    f = lambda c: chain_rhs(mesh, mat, Ms, c.swapaxes(0, 1), k_spring, Ntab, method)[0].swapaxes(0, 1)
    c = chain.swapaxes(0, 1).copy()
    for _ in range(steps):
        c, _ = I.step(f, c, st)
        c[:, 0], c[:, -1] = chain[0], chain[-1]
    c = np.ascontiguousarray(c.swapaxes(0, 1))
    E = chain_rhs(mesh, mat, Ms, c, k_spring, Ntab, method)[1]
    return c, E, st
