"""Effective field, energies and the LL right-hand side (oracle, FP64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Paper passages followed (arXiv 2406.16064):
  exchange    Sec. "Exchange energy", Eqs. 2-5: H_ex,i = 2/(mu0 Ms_i)
              sum_j A_ij (m_j - m_i)/Delta_ij^2 over the six face neighbours;
              A_ij = A, or 2 A_i A_j / (A_i + A_j) for cell-based A.
  DMI         Sec. "Dzyaloshinskii-Moriya Energy", the unified form: H_dmi,i =
              -1/(mu0 Ms_i) sum_j D_ij (e_ij x m_j)/Delta_ij for the neighbours
              {-x, +x, -y, +y, -z, +z} with e_ij = {-e_y, e_y, e_x, -e_x, 0, 0}
              (interfacial, C_nv), r_ij = {-e_x, e_x, -e_y, e_y, -e_z, e_z}
              (bulk, T/O) or {e_x, -e_x, -e_y, e_y, 0, 0} (D_2d); D_ij = D,
              or 2 D_i D_j / (D_i + D_j) for cell-based D.
  torques     Sec. "Spin transfer torques": the Zhang-Li terms
              -(u.grad)m + beta m x (u.grad)m, with -(u.grad)m written as
              m x [m x (u.grad)m], and the Slonczewski / spin-orbit terms
              -a_J m x (m x p) - b_J m x p, added to the implicit (Gilbert)
              equation and solved for dm/dt (ll_rhs).
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
with Ms_i = 0 carry no field and no torque; mu0 = 4e-7*pi exactly; a pair
constant whose two cell values sum to 0 is 0; (u.grad)m is the central
difference (m_+ - m_-)/(2 Delta) along each axis, a neighbour outside the
mesh or with Ms = 0 replaced by m_i; the spin torques act whether or not the
precession term is on.

Parity: pinned by tests/test_oracle_fields.py (spin-spiral and cycloid
closed forms, H = -dE/dm / (mu0 Ms V) by finite differences of the
independently written energies, macrospin closed form, cubic <100>/<111>
energy gap) and tests/test_oracle_fields_ext.py (bulk and D_2d helix closed
forms, the continuum DMI fields of the paper on a smooth texture, energy
gradients with every DMI class and cell-based A / D, the Gilbert-form torques
solved per cell, spin-orbit macrospin closed forms, uniform translation at
beta = alpha, and the head-to-head wall of Sec. "Domain-wall motion under
currents" under the paper's time-dependent current, whose centre and tilt
follow the closed form).
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


def _pair(C, ax, step):
    """Harmonic mean 2 C_i C_j / (C_i + C_j) with the neighbour at `step` along `ax`
    (0 where C_i + C_j = 0 or the neighbour is outside the mesh)."""
    Cj = _shift(C, ax, step)
    s = C + Cj
    return np.where(s != 0, 2.0 * C * Cj / np.where(s != 0, s, 1.0), 0.0)


def _pair_const(mat, cells, uniform, shape, ax, step):
    if cells is None:
        return np.full(shape, float(uniform))
    return _pair(np.asarray(cells, dtype=np.float64), ax, step)


def _has_exchange(mat):
    return mat.A != 0.0 or (mat.A_cells is not None and np.any(np.asarray(mat.A_cells) != 0))


def _has_dmi(mat):
    return mat.dmi != 0 and (mat.D != 0.0 or (mat.D_cells is not None and np.any(np.asarray(mat.D_cells) != 0)))


def h_exchange(mesh, mat, m, Ms):
    """Eq. 5 with A_ij (uniform or cell-based) and free boundaries."""
    H = np.zeros_like(m)
    if not _has_exchange(mat):
        return H
    has = (Ms > 0).astype(np.float64)
    for name, d in (("x", mesh.dx), ("y", mesh.dy), ("z", mesh.dz)):
        ax = _AXES[name]
        for step in (-1, 1):
            nb = _shift(has, ax, step)                      # neighbour exists and is magnetic
            Aij = _pair_const(mat, mat.A_cells, mat.A, Ms.shape, ax, step)
            for c in range(3):
                H[c] += nb * Aij * (_shift(m[c], ax, step) - m[c]) / (d * d)
    return H * (2.0 * _inv_mu0Ms(Ms))[None]


def _cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


_EX = np.array([1.0, 0.0, 0.0])[:, None, None, None]
_EY = np.array([0.0, 1.0, 0.0])[:, None, None, None]
_EZ = np.array([0.0, 0.0, 1.0])[:, None, None, None]


def dmi_table(kind):
    """(axis, step, e_ij) of the DMI class: 1 interfacial e_z x r_ij, 2 bulk r_ij,
    3 D_2d; neighbours without a DMI vector are left out."""
    if kind == 1:
        return (("x", -1, -_EY), ("x", 1, _EY), ("y", -1, _EX), ("y", 1, -_EX))
    if kind == 2:
        return (("x", -1, -_EX), ("x", 1, _EX), ("y", -1, -_EY), ("y", 1, _EY), ("z", -1, -_EZ), ("z", 1, _EZ))
    if kind == 3:
        return (("x", -1, _EX), ("x", 1, -_EX), ("y", -1, -_EY), ("y", 1, _EY))
    raise ValueError("DMI kind must be 1, 2 or 3")


def _delta(mesh, name):
    return {"x": mesh.dx, "y": mesh.dy, "z": mesh.dz}[name]


def h_dmi(mesh, mat, m, Ms):
    """The unified DMI field with the vectors of the material's class and free boundaries."""
    H = np.zeros_like(m)
    if not _has_dmi(mat):
        return H
    has = (Ms > 0).astype(np.float64)
    for name, step, e in dmi_table(mat.dmi):
        ax = _AXES[name]
        nb = _shift(has, ax, step)
        Dij = _pair_const(mat, mat.D_cells, mat.D, Ms.shape, ax, step)
        mj = np.stack([_shift(m[c], ax, step) for c in range(3)])
        H += (nb * Dij)[None] * _cross(np.broadcast_to(e, m.shape), mj) / _delta(mesh, name)
    return -_inv_mu0Ms(Ms)[None] * H


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


def has_spin_torque(mat):
    return any(v != 0.0 for v in mat.u_stt) or mat.aJ != 0.0 or mat.bJ != 0.0


def u_grad_m(mesh, mat, m, Ms):
    """(u.grad)m by central differences; a missing or non-magnetic neighbour is m_i."""
    has = (Ms > 0).astype(np.float64)
    G = np.zeros_like(m)
    for name, d, uc in (("x", mesh.dx, mat.u_stt[0]), ("y", mesh.dy, mat.u_stt[1]), ("z", mesh.dz, mat.u_stt[2])):
        if uc == 0.0:
            continue
        ax = _AXES[name]
        side = []
        for step in (1, -1):
            nb = _shift(has, ax, step)[None]
            mj = np.stack([_shift(m[c], ax, step) for c in range(3)])
            side.append(nb * mj + (1.0 - nb) * m)
        G += uc * (side[0] - side[1]) / (2.0 * d)
    return G


def gilbert_torques(mesh, mat, m, Ms):
    """The extra torques of the implicit equation dm/dt = -gamma m x H + alpha m x dm/dt + T:
    T = m x (m x (u.grad)m) + beta m x (u.grad)m - a_J m x (m x p) - b_J m x p."""
    T = np.zeros_like(m)
    if any(v != 0.0 for v in mat.u_stt):
        if mesh is None:
            raise ValueError("the Zhang-Li torque needs the mesh")
        G = u_grad_m(mesh, mat, m, Ms)
        mG = _cross(m, G)
        T += _cross(m, mG) + mat.beta * mG
    if mat.aJ != 0.0 or mat.bJ != 0.0:
        p = np.asarray(mat.p, dtype=np.float64)
        p = np.broadcast_to((p / np.linalg.norm(p))[:, None, None, None], m.shape)
        mp = _cross(m, p)
        T += -mat.aJ * _cross(m, mp) - mat.bJ * mp
    return T


def ll_rhs(mat, m, H, Ms, mesh=None):
    """LL form of the LLG equation; zero where Ms = 0.

    With A = -gamma m x H + T (T of gilbert_torques, perpendicular to m) the
    implicit equation X = A + alpha m x X has X = (A + alpha m x A)/(1 + alpha^2)
    for |m| = 1; without precession the -gamma m x H part of A is dropped from
    the first term only (the damping-only relaxation mode)."""
    gt = mat.gamma / (1.0 + mat.alpha ** 2)
    mxH = _cross(m, H)
    out = -mat.alpha * gt * _cross(m, mxH)
    if mat.precession:
        out = out - gt * mxH
    if has_spin_torque(mat):
        T = gilbert_torques(mesh, mat, m, Ms)
        out = out + (T + mat.alpha * _cross(m, T)) / (1.0 + mat.alpha ** 2)
    return out * (Ms > 0)[None]


def rhs(mesh, mat, m, Ms, Ntab=None, method="auto"):
    """dm/dt and H_eff for a state m: the LLG right-hand side."""
    H = h_eff(mesh, mat, m, Ms, Ntab, method)
    return ll_rhs(mat, m, H, Ms, mesh), H


# ---------------------------------------------------------------- energies

def energies(mesh, mat, m, Ms, Ntab=None, method="auto"):
    """Energies in J, written from the energy densities of the paper.

    exchange  V sum_i sum_j A_ij m_i.(m_i - m_j)/Delta^2  (Eq. 4, w_i summed)
    dmi       V/2 sum_i sum_j D_ij/Delta m_i.(e_ij x m_j)  (bilinear form whose
              derivative is the DMI field)
    uniaxial  -V sum_i Ku (m_i.u)^2
    cubic     V sum_i Kc (mx^4 + my^4 + mz^4)
    zeeman    -mu0 V sum_i Ms_i m_i.H
    demag     -(mu0/2) V sum_i Ms_i m_i.H_d,i             (Eqs. 6-7)
    """
    V = mesh.dx * mesh.dy * mesh.dz
    has = (Ms > 0).astype(np.float64)
    E = {}
    ex = 0.0
    if _has_exchange(mat):
        for name, d in (("x", mesh.dx), ("y", mesh.dy), ("z", mesh.dz)):
            ax = _AXES[name]
            for step in (-1, 1):
                nb = _shift(has, ax, step) * has
                Aij = _pair_const(mat, mat.A_cells, mat.A, Ms.shape, ax, step)
                mj = np.stack([_shift(m[c], ax, step) for c in range(3)])
                ex += (nb * Aij * (m * (m - mj)).sum(axis=0)).sum() / (d * d)
    E["exchange"] = V * ex
    dm = 0.0
    if _has_dmi(mat):
        for name, step, e in dmi_table(mat.dmi):
            ax = _AXES[name]
            nb = _shift(has, ax, step) * has
            Dij = _pair_const(mat, mat.D_cells, mat.D, Ms.shape, ax, step)
            mj = np.stack([_shift(m[c], ax, step) for c in range(3)])
            dm += (nb * Dij * (m * _cross(np.broadcast_to(e, m.shape), mj)).sum(axis=0)).sum() / _delta(mesh, name)
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
