"""Effective field, energies and the LL right-hand side (oracle, FP64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Paper passages followed (arXiv 2406.16064):
  exchange    Sec. "Exchange energy", Eqs. 2-5: H_ex,i = 2/(mu0 Ms_i)
              sum_j A (m_j - m_i)/Delta_ij^2 over the six face neighbours.
  DMI         Sec. "Dzyaloshinskii-Moriya Energy", Eq. 14: H_dmi,i =
              -1/(mu0 Ms_i) sum_j D (e_ij x m_j)/Delta_ij, interfacial e_ij
              = {-e_y, e_y, e_x, -e_x, 0, 0} for {-x, +x, -y, +y, -z, +z}.
  anisotropy  Sec. "Anisotropy": uniaxial H = 2K (m.u) u / (mu0 Ms),
              E = -K (m.u)^2; cubic E = Kc (mx^4 + my^4 + mz^4), H = -4Kc
              m^3 / (mu0 Ms) (the atomistic forms with mu_s -> mu0 Ms V).
  Zeeman      Sec. "Zeeman energy": H = H_ext, E = -mu0 Ms m.H.
  demag       oracle.demag (Eq. 8).
  LL          Sec. "LLG equation", LL form: dm/dt = -g~ m x H - alpha g~
              m x (m x H), g~ = gamma/(1+alpha^2); precession off drops
              the first term (the NEB/relax mode of Sec. "Miscellaneous").

Readings where the paper is silent: free boundaries -- a neighbour outside
the mesh or with Ms_j = 0 is dropped from the exchange and DMI sums; cells
with Ms_i = 0 carry no field and no torque; mu0 = 4e-7*pi exactly.

Parity: pinned by tests/test_oracle_fields.py (spin-spiral and cycloid
closed forms, H = -dE/dm / (mu0 Ms V) by finite differences of the
independently written energies, macrospin closed form, cubic <100>/<111>
energy gap).
"""
from __future__ import annotations

import math

import numpy as np

from . import demag as _demag

MU0 = 4e-7 * math.pi

# neighbour directions: (axis index in (z, y, x) array order, step)
_AXES = {"x": 2, "y": 1, "z": 0}


def _shift(a, axis, step):
    """b[i] = a[i + step] along `axis` (array axis), zero where i+step is outside."""
    b = np.zeros_like(a)
    n = a.shape[axis]
    src = [slice(None)] * a.ndim
    dst = [slice(None)] * a.ndim
    if step > 0:
        src[axis] = slice(step, n)
        dst[axis] = slice(0, n - step)
    else:
        src[axis] = slice(0, n + step)
        dst[axis] = slice(-step, n)
    b[tuple(dst)] = a[tuple(src)]
    return b


def ms_array(sim_mesh, mat, Ms_cells=None):
    if Ms_cells is not None:
        return np.asarray(Ms_cells, dtype=np.float64)
    return np.full(sim_mesh.shape, float(mat.Ms))


def _inv_mu0Ms(Ms):
    return np.where(Ms > 0, 1.0 / (MU0 * np.where(Ms > 0, Ms, 1.0)), 0.0)


def h_exchange(mesh, mat, m, Ms):
    """Eq. 5 with A_ij = A and free boundaries."""
    H = np.zeros_like(m)
    if mat.A == 0.0:
        return H
    has = (Ms > 0).astype(np.float64)
    for name, d in (("x", mesh.dx), ("y", mesh.dy), ("z", mesh.dz)):
        ax = _AXES[name]
        for step in (-1, 1):
            nb = _shift(has, ax, step)                      # neighbour exists and is magnetic
            for c in range(3):
                H[c] += nb * (_shift(m[c], ax, step) - m[c]) / (d * d)
    return H * (2.0 * mat.A * _inv_mu0Ms(Ms))[None]


def _cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def h_dmi(mesh, mat, m, Ms):
    """Eq. 14 with the interfacial DMI vectors and free boundaries."""
    H = np.zeros_like(m)
    if mat.D == 0.0 or mat.dmi == 0:
        return H
    has = (Ms > 0).astype(np.float64)
    ex = np.array([1.0, 0.0, 0.0])[:, None, None, None]
    ey = np.array([0.0, 1.0, 0.0])[:, None, None, None]
    # (axis, step, e_ij, Delta)
    table = (("x", -1, -ey, mesh.dx), ("x", 1, ey, mesh.dx),
             ("y", -1, ex, mesh.dy), ("y", 1, -ex, mesh.dy))
    for name, step, e, d in table:
        ax = _AXES[name]
        nb = _shift(has, ax, step)
        mj = np.stack([_shift(m[c], ax, step) for c in range(3)])
        H += nb[None] * _cross(np.broadcast_to(e, m.shape), mj) / d
    return -mat.D * _inv_mu0Ms(Ms)[None] * H


def h_uniaxial(mat, m, Ms):
    if mat.Ku == 0.0:
        return np.zeros_like(m)
    u = np.asarray(mat.u, dtype=np.float64)
    u = u / np.linalg.norm(u)
    mu = m[0] * u[0] + m[1] * u[1] + m[2] * u[2]
    return (2.0 * mat.Ku * _inv_mu0Ms(Ms) * mu)[None] * u[:, None, None, None]


def h_cubic(mat, m, Ms):
    if mat.Kc == 0.0:
        return np.zeros_like(m)
    return -4.0 * mat.Kc * _inv_mu0Ms(Ms)[None] * m ** 3


def h_zeeman(mat, m, Ms):
    H = np.zeros_like(m)
    has = Ms > 0
    for c in range(3):
        H[c] = np.where(has, mat.H[c], 0.0)
    return H


def h_demag(mesh, mat, m, Ms, Ntab=None, method="auto"):
    if not mat.demag:
        return np.zeros_like(m)
    M = m * Ms[None]
    if method == "auto":
        method = "direct" if mesh.ncells <= 1024 else "fft"
    if method == "direct":
        return _demag.demag_direct(mesh, M, Ntab)
    return _demag.demag_fft(mesh, M, Ntab)


def field_terms(mesh, mat, m, Ms, Ntab=None, method="auto"):
    """Every term of H_eff (A/m) as a dict; 'total' is their sum (Eq. 1)."""
    t = {
        "exchange": h_exchange(mesh, mat, m, Ms),
        "dmi": h_dmi(mesh, mat, m, Ms),
        "uniaxial": h_uniaxial(mat, m, Ms),
        "cubic": h_cubic(mat, m, Ms),
        "zeeman": h_zeeman(mat, m, Ms),
        "demag": h_demag(mesh, mat, m, Ms, Ntab, method),
    }
    tot = sum(t.values())
    tot = tot * (Ms > 0)[None]
    t["total"] = tot
    return t


def h_eff(mesh, mat, m, Ms, Ntab=None, method="auto"):
    return field_terms(mesh, mat, m, Ms, Ntab, method)["total"]


def ll_rhs(mat, m, H, Ms):
    """LL form of the LLG equation; zero where Ms = 0."""
    gt = mat.gamma / (1.0 + mat.alpha ** 2)
    mxH = _cross(m, H)
    out = -mat.alpha * gt * _cross(m, mxH)
    if mat.precession:
        out = out - gt * mxH
    return out * (Ms > 0)[None]


def rhs(mesh, mat, m, Ms, Ntab=None, method="auto"):
    """dm/dt and H_eff for a state m: the LLG right-hand side."""
    H = h_eff(mesh, mat, m, Ms, Ntab, method)
    return ll_rhs(mat, m, H, Ms), H


# ---------------------------------------------------------------- energies

def energies(mesh, mat, m, Ms, Ntab=None, method="auto"):
    """Energies in J, written from the energy densities of the paper.

    exchange  V sum_i sum_j A m_i.(m_i - m_j)/Delta^2   (Eq. 4, w_i summed)
    dmi       V/2 sum_i sum_j D/Delta m_i.(e_ij x m_j)   (bilinear form whose
              derivative is Eq. 14)
    uniaxial  -V sum_i Ku (m_i.u)^2
    cubic     V sum_i Kc (mx^4 + my^4 + mz^4)
    zeeman    -mu0 V sum_i Ms_i m_i.H
    demag     -(mu0/2) V sum_i Ms_i m_i.H_d,i             (Eqs. 6-7)
    """
    V = mesh.dx * mesh.dy * mesh.dz
    has = (Ms > 0).astype(np.float64)
    E = {}
    ex = 0.0
    if mat.A != 0.0:
        for name, d in (("x", mesh.dx), ("y", mesh.dy), ("z", mesh.dz)):
            ax = _AXES[name]
            for step in (-1, 1):
                nb = _shift(has, ax, step) * has
                mj = np.stack([_shift(m[c], ax, step) for c in range(3)])
                ex += (nb * (m * (m - mj)).sum(axis=0)).sum() * mat.A / (d * d)
    E["exchange"] = V * ex
    dm = 0.0
    if mat.D != 0.0 and mat.dmi:
        exv = np.array([1.0, 0.0, 0.0])[:, None, None, None]
        eyv = np.array([0.0, 1.0, 0.0])[:, None, None, None]
        for name, step, e, d in (("x", -1, -eyv, mesh.dx), ("x", 1, eyv, mesh.dx),
                                 ("y", -1, exv, mesh.dy), ("y", 1, -exv, mesh.dy)):
            ax = _AXES[name]
            nb = _shift(has, ax, step) * has
            mj = np.stack([_shift(m[c], ax, step) for c in range(3)])
            dm += (nb * (m * _cross(np.broadcast_to(e, m.shape), mj)).sum(axis=0)).sum() * mat.D / d
    E["dmi"] = 0.5 * V * dm
    if mat.Ku != 0.0:
        u = np.asarray(mat.u, float) / np.linalg.norm(mat.u)
        mu = m[0] * u[0] + m[1] * u[1] + m[2] * u[2]
        E["uniaxial"] = -V * mat.Ku * (has * mu * mu).sum()
    else:
        E["uniaxial"] = 0.0
    E["cubic"] = V * mat.Kc * (has * (m ** 4).sum(axis=0)).sum() if mat.Kc != 0.0 else 0.0
    E["zeeman"] = -MU0 * V * (Ms * (m[0] * mat.H[0] + m[1] * mat.H[1] + m[2] * mat.H[2])).sum()
    if mat.demag:
        Hd = h_demag(mesh, mat, m, Ms, Ntab, method)
        E["demag"] = -0.5 * MU0 * V * (Ms * (m * Hd).sum(axis=0)).sum()
    else:
        E["demag"] = 0.0
    E["total"] = sum(E.values())
    return E
