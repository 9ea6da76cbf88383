"""Pins for the extended terms of oracle.fields: bulk and D_2d DMI, cell-based
exchange and DMI constants, Zhang-Li and Slonczewski / spin-orbit torques
(Sec. "Dzyaloshinskii-Moriya Energy", Sec. "Exchange energy", Sec. "Spin
transfer torques").  No GPU."""
import math

import numpy as np
import pytest

import synth
from oracle import fields as F

E = np.eye(3)


def _helix(mesh, axis, k):
    """m = cos(k s) e1 + sin(k s) e2 along `axis` (s the cell coordinate), (e1, e2, e_axis)
    right-handed."""
    a = "xyz".index(axis)
    e1, e2 = E[(a + 1) % 3], E[(a + 2) % 3]
    n = (mesh.nx, mesh.ny, mesh.nz)[a]
    d = (mesh.dx, mesh.dy, mesh.dz)[a]
    s = np.arange(n) * d
    shape = [1, 1, 1]
    shape[2 - a] = n                                     # array order (z, y, x)
    c = np.cos(k * s).reshape(shape)
    sn = np.sin(k * s).reshape(shape)
    m = c[None] * e1[:, None, None, None] + sn[None] * e2[:, None, None, None]
    return np.broadcast_to(m, (3,) + mesh.shape).copy(), d, n


# discrete closed forms of the DMI field of a helix about each axis (interior cells) and
# of its energy, from the DMI vectors of each class: (field factor, energy factor) times
# D sin(k Delta) / Delta, per axis
CLOSED = {
    2: {"x": (2, -1), "y": (2, -1), "z": (2, -1)},      # bulk: e_ij = r_ij
    3: {"x": (-2, 1), "y": (2, -1), "z": (0, 0)},       # D_2d
    1: {"z": (0, 0)},                                   # interfacial: no z neighbours
}


@pytest.mark.parametrize("kind,axis", [(2, "x"), (2, "y"), (2, "z"), (3, "x"), (3, "y"), (3, "z"), (1, "z")])
def test_dmi_helix_closed_forms(kind, axis):
    mesh = synth.Mesh(*{"x": (20, 3, 3), "y": (3, 20, 3), "z": (3, 3, 20)}[axis], 2e-9, 2.5e-9, 1.5e-9)
    Ms, D = 8e5, 3e-3
    mat = synth.Material(Ms=Ms, D=D, dmi=kind, demag=0)
    k = 2 * math.pi / (13 * (mesh.dx, mesh.dy, mesh.dz)["xyz".index(axis)])
    m, d, n = _helix(mesh, axis, k)
    Msa = F.ms_array(mesh, mat)
    H = F.h_dmi(mesh, mat, m, Msa)
    fh, fe = CLOSED[kind][axis]
    expect = fh * D * math.sin(k * d) / (F.MU0 * Ms * d) * m
    sl = (slice(None), slice(1, -1), slice(1, -1), slice(1, -1))   # interior cells
    scale = 2 * D / (F.MU0 * Ms * d)
    np.testing.assert_allclose(H[sl], expect[sl], rtol=0, atol=1e-12 * scale)
    Et = F.energies(mesh, mat, m, Msa)["dmi"]
    V = mesh.dx * mesh.dy * mesh.dz
    bonds = (n - 1) * mesh.ncells // n
    Ee = fe * V * D * math.sin(k * d) / d * bonds
    assert abs(Et - Ee) <= 1e-12 * V * D / d * bonds


def _smooth(mesh, seed):
    """A smooth (unnormalised) vector field and its analytic x, y, z derivatives."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(mesh.nz) * mesh.dz, np.arange(mesh.ny) * mesh.dy,
                          np.arange(mesh.nx) * mesh.dx, indexing="ij")
    kv = rng.uniform(-1, 1, (3, 3)) * 2 * math.pi / (80 * mesh.dx)
    ph = rng.uniform(0, 2 * math.pi, 3)
    arg = [kv[c, 0] * x + kv[c, 1] * y + kv[c, 2] * z + ph[c] for c in range(3)]
    m = np.stack([np.sin(a) for a in arg])
    dm = [np.stack([kv[c, ax] * np.cos(arg[c]) for c in range(3)]) for ax in range(3)]
    return m, dm


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_dmi_matches_the_continuum_fields_of_the_paper(kind):
    """Bulk: H = -2D/(mu0 Ms) curl m; interfacial: -2D/(mu0 Ms)(e_y x dm/dx - e_x x dm/dy);
    D_2d: -2D/(mu0 Ms)(e_y x dm/dy - e_x x dm/dx): the discrete field on a smooth texture
    agrees to O(Delta^2) away from the boundaries."""
    mesh = synth.Mesh(24, 22, 20, 1e-9, 1e-9, 1e-9)
    Ms, D = 8e5, 3e-3
    mat = synth.Material(Ms=Ms, D=D, dmi=kind, demag=0)
    m, (mx, my, mz) = _smooth(mesh, 4)
    H = F.h_dmi(mesh, mat, m, F.ms_array(mesh, mat))
    bc = lambda v: np.broadcast_to(v[:, None, None, None], m.shape)
    ex, ey, ez = bc(E[0]), bc(E[1]), bc(E[2])
    if kind == 2:
        curl = F._cross(ex, mx) + F._cross(ey, my) + F._cross(ez, mz)
        cont = -2 * D / (F.MU0 * Ms) * curl
    elif kind == 1:
        cont = -2 * D / (F.MU0 * Ms) * (F._cross(ey, mx) - F._cross(ex, my))
    else:
        cont = -2 * D / (F.MU0 * Ms) * (F._cross(ey, my) - F._cross(ex, mx))
    inner = (slice(None), slice(1, -1), slice(1, -1), slice(1, -1))
    err = np.abs(H[inner] - cont[inner]).max() / np.abs(cont[inner]).max()
    assert err < 3e-3, err


TERMS = ["exchange", "dmi"]


@pytest.mark.parametrize("kind,cells,masked", [(2, False, False), (3, False, True), (1, True, False),
                                               (2, True, True), (3, True, False)])
def test_extended_fields_are_energy_gradients(kind, cells, masked):
    """H_term,i = -(1/(mu0 Ms_i V)) dE_term/dm_i by central differences."""
    mesh = synth.Mesh(6, 5, 3, 2e-9, 2.5e-9, 1.5e-9)
    rng = np.random.default_rng(11)
    A_cells = rng.uniform(0.5e-11, 2e-11, mesh.shape) if cells else None
    D_cells = rng.uniform(1e-3, 4e-3, mesh.shape) if cells else None
    if cells:
        A_cells[1, 2, 2] = 0.0                          # a cell decoupled from its neighbours
    mat = synth.Material(Ms=8e5, A=1.3e-11, D=3e-3, dmi=kind, demag=0, A_cells=A_cells, D_cells=D_cells)
    m = synth.random_state(7, mesh)
    Ms = F.ms_array(mesh, mat).copy()
    if masked:
        Ms[1, 2, 3] = 0.0
        Ms[2, 4, 5] = 3e5
    H = F.field_terms(mesh, mat, m, Ms)
    V = mesh.dx * mesh.dy * mesh.dz
    h = 1e-6
    for term in TERMS:
        scale = np.abs(H[term]).max()
        for (c, iz, iy, ix) in [(0, 1, 2, 3), (1, 0, 0, 3), (2, 2, 4, 5), (0, 2, 3, 1), (1, 1, 2, 1), (2, 1, 2, 2)]:
            if Ms[iz, iy, ix] == 0:
                continue
            mp = m.copy(); mp[c, iz, iy, ix] += h
            mm = m.copy(); mm[c, iz, iy, ix] -= h
            g = (F.energies(mesh, mat, mp, Ms)[term] - F.energies(mesh, mat, mm, Ms)[term]) / (2 * h)
            Hn = -g / (F.MU0 * Ms[iz, iy, ix] * V)
            assert abs(Hn - H[term][c, iz, iy, ix]) < 1e-6 * scale, (term, c, iz, iy, ix)


def test_cell_constants_harmonic_mean_by_hand():
    """A chain A = (A1, A1, A2, A2): cell 1 couples to cell 0 with A1 and to cell 2 with
    2 A1 A2 / (A1 + A2); uniform cell values reproduce the uniform constant; a cell with
    A = 0 is decoupled."""
    mesh = synth.Mesh(4, 1, 1, 2e-9, 2e-9, 2e-9)
    A1, A2, Ms = 1e-11, 3e-11, 8e5
    m = synth.random_state(2, mesh)
    cells = np.array([A1, A1, A2, A2]).reshape(mesh.shape)
    mat = synth.Material(Ms=Ms, A=0.0, demag=0, A_cells=cells)
    Msa = F.ms_array(mesh, mat)
    H = F.h_exchange(mesh, mat, m, Msa)
    A12 = 2 * A1 * A2 / (A1 + A2)
    c = 2 / (F.MU0 * Ms * mesh.dx ** 2)
    want = c * (A1 * (m[:, 0, 0, 0] - m[:, 0, 0, 1]) + A12 * (m[:, 0, 0, 2] - m[:, 0, 0, 1]))
    np.testing.assert_allclose(H[:, 0, 0, 1], want, rtol=1e-14, atol=0)
    uni = synth.Material(Ms=Ms, A=A1, demag=0)
    same = synth.Material(Ms=Ms, A=0.0, demag=0, A_cells=np.full(mesh.shape, A1))
    np.testing.assert_allclose(F.h_exchange(mesh, same, m, Msa), F.h_exchange(mesh, uni, m, Msa), rtol=1e-15)
    cells0 = cells.copy()
    cells0[0, 0, 2] = 0.0
    H0 = F.h_exchange(mesh, synth.Material(Ms=Ms, demag=0, A_cells=cells0), m, Msa)
    assert np.all(H0[:, 0, 0, 2] == 0)
    np.testing.assert_allclose(H0[:, 0, 0, 1], c * A1 * (m[:, 0, 0, 0] - m[:, 0, 0, 1]), rtol=1e-14)
    Dm = synth.Material(Ms=Ms, D=0.0, dmi=2, demag=0, D_cells=np.array([2e-3, -2e-3, 1e-3, 3e-3]).reshape(mesh.shape))
    # D_01 = 2 (2e-3)(-2e-3) / 0 -> 0 (the pair of opposite values sums to 0)
    Hd = F.h_dmi(mesh, Dm, m, Msa)
    D12 = 2 * (-2e-3) * 1e-3 / (-1e-3)
    want = -(D12 * np.cross(E[0], m[:, 0, 0, 2])) / (F.MU0 * Ms * mesh.dx)
    np.testing.assert_allclose(Hd[:, 0, 0, 1], want, rtol=1e-14)


def _skew(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


@pytest.mark.parametrize("precession", [1, 0])
def test_torques_solve_the_implicit_gilbert_equation(precession):
    """dm/dt from the LL form equals the per-cell solution of
    (I - alpha [m]x) X = -gamma m x H + T (T: the torques of Sec. "Spin transfer torques")."""
    mesh = synth.Mesh(5, 4, 3, 2e-9, 2e-9, 3e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, D=2e-3, dmi=2, Ku=3e5, H=(1e4, 2e4, -3e4), alpha=0.3,
                         precession=precession, demag=0, u_stt=(60.0, -25.0, 10.0), beta=0.1,
                         aJ=2e9, bJ=-7e8, p=(0.2, -0.5, 1.0))
    m = synth.random_state(3, mesh)
    Ms = F.ms_array(mesh, mat).copy()
    Ms[1, 2, 2] = 0.0
    dmdt, H = F.rhs(mesh, mat, m, Ms, method="direct")
    G = F.u_grad_m(mesh, mat, m, Ms)
    p = np.array(mat.p) / np.linalg.norm(mat.p)
    gam, al = mat.gamma, mat.alpha
    for iz in range(mesh.nz):
        for iy in range(mesh.ny):
            for ix in range(mesh.nx):
                mi, Hi, Gi = m[:, iz, iy, ix], H[:, iz, iy, ix], G[:, iz, iy, ix]
                if Ms[iz, iy, ix] == 0:
                    assert np.all(dmdt[:, iz, iy, ix] == 0)
                    continue
                T = (np.cross(mi, np.cross(mi, Gi)) + mat.beta * np.cross(mi, Gi)
                     - mat.aJ * np.cross(mi, np.cross(mi, p)) - mat.bJ * np.cross(mi, p))
                if precession:
                    X = np.linalg.solve(np.eye(3) - al * _skew(mi), -gam * np.cross(mi, Hi) + T)
                else:
                    # damping-only mode: the precession term of the LL form is dropped
                    Xh = np.linalg.solve(np.eye(3) - al * _skew(mi), -gam * np.cross(mi, Hi))
                    Xp = -gam / (1 + al ** 2) * np.cross(mi, Hi)
                    X = (Xh - Xp) + np.linalg.solve(np.eye(3) - al * _skew(mi), T)
                np.testing.assert_allclose(dmdt[:, iz, iy, ix], X, rtol=0, atol=1e-12 * np.abs(X).max())


def _macrospin_run(mat, m0, t, n):
    mesh = synth.Mesh(1, 1, 1, 2e-9, 2e-9, 2e-9)
    Ms = F.ms_array(mesh, mat)
    f = lambda y: F.rhs(mesh, mat, y, Ms)[0]
    m = m0.reshape(3, 1, 1, 1).astype(float)
    h = t / n
    for _ in range(n):
        k1 = f(m); k2 = f(m + 0.5 * h * k1); k3 = f(m + 0.5 * h * k2); k4 = f(m + h * k3)
        m = m + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return m.ravel()


def test_spin_orbit_macrospin_closed_forms():
    """No field, alpha = 0: b_J alone turns m about p at the rate b_J; a_J alone pulls m
    towards p with m.p = tanh(a_J t + atanh(m0.p))."""
    p = np.array([0.0, 0.0, 1.0])
    m0 = np.array([math.sin(1.0), 0.0, math.cos(1.0)])
    bJ, t = 3e9, 1e-9
    mat = synth.Material(Ms=8e5, alpha=0.0, demag=0, bJ=bJ, p=tuple(p))
    m = _macrospin_run(mat, m0, t, 2000)
    ang = bJ * t
    want = np.array([math.sin(1.0) * math.cos(ang), math.sin(1.0) * math.sin(ang), math.cos(1.0)])
    assert np.abs(m - want).max() < 1e-9
    aJ = 2e9
    mat = synth.Material(Ms=8e5, alpha=0.0, demag=0, aJ=aJ, p=tuple(p))
    m = _macrospin_run(mat, m0, t, 2000)
    assert abs(m[2] - math.tanh(aJ * t + math.atanh(math.cos(1.0)))) < 1e-9
    assert abs(m[1]) < 1e-12


def _unit_texture(mesh, seed):
    """m = (sin t cos f, sin t sin f, cos t) with t, f linear in position, and its
    analytic x, y, z derivatives."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(mesh.nz) * mesh.dz, np.arange(mesh.ny) * mesh.dy,
                          np.arange(mesh.nx) * mesh.dx, indexing="ij")
    a, b = rng.uniform(-1, 1, (2, 3)) * 2 * math.pi / (80 * mesh.dx)
    t = a[0] * x + a[1] * y + a[2] * z + 0.7
    f = b[0] * x + b[1] * y + b[2] * z + 0.3
    m = np.stack([np.sin(t) * np.cos(f), np.sin(t) * np.sin(f), np.cos(t)])
    mt = np.stack([np.cos(t) * np.cos(f), np.cos(t) * np.sin(f), -np.sin(t)])
    mf = np.stack([-np.sin(t) * np.sin(f), np.sin(t) * np.cos(f), np.zeros_like(t)])
    return m, [a[i] * mt + b[i] * mf for i in range(3)]


def test_zhang_li_uniform_translation_and_gradient():
    """beta = alpha and no field: dm/dt = m x (m x (u.grad)m), i.e. -(u.grad)m for |m| = 1
    and a gradient along m of zero; the central difference matches the analytic gradient
    of a smooth texture to O(Delta^2); a missing neighbour is the cell itself."""
    mesh = synth.Mesh(30, 4, 3, 1e-9, 1e-9, 1e-9)
    u = (80.0, -30.0, 20.0)
    mat = synth.Material(Ms=8e5, alpha=0.2, beta=0.2, demag=0, u_stt=u)
    m, dr = _unit_texture(mesh, 9)
    Ms = F.ms_array(mesh, mat)
    dmdt, _ = F.rhs(mesh, mat, m, Ms)
    G = F.u_grad_m(mesh, mat, m, Ms)
    np.testing.assert_allclose(dmdt, F._cross(m, F._cross(m, G)), rtol=0, atol=1e-12 * np.abs(G).max())
    Gr = sum(uc * dr[a] for a, uc in enumerate(u))
    inner = (slice(None), slice(1, -1), slice(1, -1), slice(1, -1))
    assert np.abs(G[inner] - Gr[inner]).max() < 5e-3 * np.abs(Gr[inner]).max()
    np.testing.assert_allclose(dmdt[inner], -Gr[inner], rtol=0, atol=5e-3 * np.abs(Gr[inner]).max())
    # one-cell-thick mesh along z: the z term vanishes; a boundary cell is one-sided /(2 Delta)
    thin = synth.Mesh(5, 4, 1, 1e-9, 1e-9, 1e-9)
    mt = synth.random_state(5, thin)
    Mt = synth.Material(Ms=8e5, demag=0, u_stt=(0.0, 0.0, 50.0))
    assert np.all(F.u_grad_m(thin, Mt, mt, F.ms_array(thin, Mt)) == 0)
    Mx = synth.Material(Ms=8e5, demag=0, u_stt=(50.0, 0.0, 0.0))
    Gx = F.u_grad_m(thin, Mx, mt, F.ms_array(thin, Mx))
    np.testing.assert_allclose(Gx[:, 0, 1, 0], 50.0 * (mt[:, 0, 1, 1] - mt[:, 0, 1, 0]) / 2e-9, rtol=1e-14)


@pytest.mark.parametrize("beta", [0.0, 0.3])
def test_head_to_head_wall_under_time_dependent_current(beta):
    """Sec. "Domain-wall motion under currents": a 1D head-to-head wall (uniaxial K along
    the wire, no demag) driven by u(t) = u0 exp(-b t) cos(w t) with b = 5e8 1/s, w = 2e9 1/s,
    Permalloy constants, alpha = 0.1.  For dm/dt = -gamma m x H + alpha m x dm/dt
    - (u.grad)m + beta m x (u.grad)m the rigid wall moves with dz/dt = (1 + alpha beta) u /
    (1 + alpha^2) and tilts with dphi/dt = (beta - alpha) u / ((1 + alpha^2) Delta),
    Delta = sqrt(A/K) (the paper prints both with u of the opposite sign; magnitudes and
    their ratio agree)."""
    from dataclasses import replace
    nx, dx = 200, 1e-9
    mesh = synth.Mesh(nx, 1, 1, dx, dx, dx)
    A, K, al = 1.3e-11, 1e5, 0.1
    Dw = math.sqrt(A / K)
    mat = synth.Material(Ms=8e5, A=A, Ku=K, u=(1, 0, 0), alpha=al, beta=beta, demag=0)
    u0, b, w = 100.0, 5e8, 2e9
    u = lambda t: u0 * math.exp(-b * t) * math.cos(w * t)
    Iu = lambda t: u0 * (math.exp(-b * t) * (w * math.sin(w * t) - b * math.cos(w * t)) + b) / (b * b + w * w)
    x = (np.arange(nx) + 0.5) * dx
    th = 2 * np.arctan(np.exp((x - 60e-9) / Dw))            # +x on the left, -x on the right
    m = np.stack([np.cos(th), np.sin(th) * np.cos(0.4), np.sin(th) * np.sin(0.4)]).reshape(3, 1, 1, nx)
    Ms = F.ms_array(mesh, mat)
    f = lambda t, y: F.rhs(mesh, replace(mat, u_stt=(u(t), 0.0, 0.0)), y, Ms)[0]
    centre = lambda m: nx * dx - ((1 - m[0].ravel()) / 2).sum() * dx
    tilt = lambda m: math.atan2(m[2].sum(), m[1].sum())
    z0, p0 = centre(m), tilt(m)
    h, n = 8e-14, 5000
    t = 0.0
    dz, dp, ez, ep = [], [], [], []
    for i in range(n):                                    # classical RK4 with u at the stage times
        k1 = f(t, m); k2 = f(t + h / 2, m + h / 2 * k1); k3 = f(t + h / 2, m + h / 2 * k2); k4 = f(t + h, m + h * k3)
        m = m + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        m = m / np.sqrt((m ** 2).sum(0))[None]
        t += h
        if (i + 1) % 250 == 0:
            dz.append(centre(m) - z0); ez.append((1 + al * beta) / (1 + al * al) * Iu(t))
            dp.append(tilt(m) - p0); ep.append((beta - al) / ((1 + al * al) * Dw) * Iu(t))
    dz, ez, dp, ep = map(np.array, (dz, ez, dp, ep))
    assert np.abs(dz - ez).max() < 0.01 * np.abs(ez).max()
    assert np.abs(dp - ep).max() < 0.02 * np.abs(ep).max()
