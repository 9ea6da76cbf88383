"""Pins for oracle.newell against results the mathematics fixes (no GPU)."""
import math
import os

import numpy as np
import pytest

from oracle import newell as nw

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def aharoni_z(a, b, c):
    """Aharoni (1998) Eq. 1: demag factor along c of a 2a x 2b x 2c prism."""
    r = math.sqrt(a * a + b * b + c * c)
    ab, bc, ac = math.hypot(a, b), math.hypot(b, c), math.hypot(a, c)
    s = (b * b - c * c) / (2 * b * c) * math.log((r - a) / (r + a))
    s += (a * a - c * c) / (2 * a * c) * math.log((r - b) / (r + b))
    s += b / (2 * c) * math.log((ab + a) / (ab - a)) + a / (2 * c) * math.log((ab + b) / (ab - b))
    s += c / (2 * a) * math.log((bc - b) / (bc + b)) + c / (2 * b) * math.log((ac - a) / (ac + a))
    s += 2 * math.atan(a * b / (c * r))
    s += (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c) + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
    s += c / (a * b) * (ac + bc) - (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c)
    return s / math.pi


def test_cube_self_term_is_one_third():
    t = nw.tensor_exact(0.0, 0.0, 0.0, 1.0, 1.0, 1.0)
    with open(os.path.join(GOLDEN, "aharoni_prism.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    expect = float(rows[0][3])
    np.testing.assert_allclose(t[:3], expect, rtol=0, atol=1e-15)
    np.testing.assert_allclose(t[3:], 0.0, atol=1e-15)


@pytest.mark.parametrize("abc", [(1, 2, 3), (5, 5, 0.5), (0.3, 2, 1.7), (10, 0.2, 0.2)])
def test_self_term_matches_aharoni(abc):
    a, b, c = abc
    t = nw.tensor_exact(0.0, 0.0, 0.0, 2 * a, 2 * b, 2 * c)
    # both closed forms cancel at large aspect ratios (~3e-13 at 50:1)
    assert abs(t[2] - aharoni_z(a, b, c)) < 1e-12
    # and the other axes by relabelling the prism
    assert abs(t[0] - aharoni_z(b, c, a)) < 1e-12
    assert abs(t[1] - aharoni_z(c, a, b)) < 1e-12
    assert abs(t[:3].sum() - 1.0) < 1e-12


def test_trace_vanishes_off_centre():
    rng = np.random.default_rng(1)
    for _ in range(20):
        d = rng.uniform(0.3, 3.0, 3)
        off = rng.integers(-6, 7, 3) * d
        if not off.any():
            continue
        t = nw.tensor(*off, *d)
        # closed-form cancellation grows like (r/d_min)^6 for elongated cells
        assert abs(t[:3].sum()) < 1e-11 * np.abs(t).max()


def test_parities_and_axis_relabelling():
    d = (1.0, 1.3, 0.7)
    X, Y, Z = 2.0, 3.9, 1.4
    t = nw.tensor(X, Y, Z, *d)
    for sx, sy, sz in [(-1, 1, 1), (1, -1, 1), (1, 1, -1), (-1, -1, -1)]:
        u = nw.tensor(sx * X, sy * Y, sz * Z, *d)
        for c in range(6):
            px, py, pz = nw.PARITY[c]
            sign = (px if sx < 0 else 1) * (py if sy < 0 else 1) * (pz if sz < 0 else 1)
            assert abs(u[c] - sign * t[c]) <= 1e-13 * np.abs(t).max()
    # swap x <-> y: xx<->yy, xz<->yz, xy stays
    s = nw.tensor(Y, X, Z, d[1], d[0], d[2])
    np.testing.assert_allclose(s[[1, 0, 2, 3, 5, 4]], t, rtol=0, atol=1e-13 * np.abs(t).max())


@pytest.mark.parametrize("cell", [(1, 1, 1), (1, 1, 0.5), (1, 1, 0.25), (2.5, 2.5, 3)])
def test_closed_form_and_quadrature_agree_across_switch(cell):
    rng = np.random.default_rng(2)
    dirs = rng.normal(size=(30, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    dm = max(cell)
    for r in (nw.SWITCH, nw.SWITCH + 0.5):
        X, Y, Z = (dirs * r * dm).T
        ex = nw.tensor_exact(X, Y, Z, *cell)
        qu = nw.tensor_far(X, Y, Z, *cell, 12)
        scale = np.abs(qu).max(axis=0)
        assert (np.abs(ex - qu).max(axis=0) / scale).max() < 1e-10   # closed-form cancellation


@pytest.mark.parametrize("cell", [(1, 1, 1), (1, 1, 0.25), (2.5, 2.5, 3)])
def test_quadrature_bands_converged(cell):
    rng = np.random.default_rng(3)
    dirs = rng.normal(size=(20, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    dm = max(cell)
    for r in (3.01, 4.0, 6.0, 12.0, 32.0, 128.0, 500.0):
        q = int(nw.far_order(r))
        X, Y, Z = (dirs * r * dm).T
        ref = nw.tensor_far(X, Y, Z, *cell, 16)
        got = nw.tensor_far(X, Y, Z, *cell, q)
        assert (np.abs(got - ref).max(axis=0) / np.abs(ref).max(axis=0)).max() < 1e-13


def test_far_field_is_point_dipole():
    d = (1.0, 2.0, 0.5)
    V = d[0] * d[1] * d[2]
    R = np.array([700.0, -400.0, 250.0])
    t = nw.tensor(*R, *d)
    r = np.linalg.norm(R)
    G = V / (4 * math.pi) * (np.eye(3) * r * r - 3 * np.outer(R, R)) / r ** 5
    g6 = np.array([G[0, 0], G[1, 1], G[2, 2], G[0, 1], G[0, 2], G[1, 2]])
    assert np.abs(t - g6).max() < 1e-5 * np.abs(g6).max()       # (d/r)^2 corrections


@pytest.mark.parametrize("mesh", [(6, 5, 3, 1.0, 1.5, 0.8), (24, 20, 2, 1.0, 1.0, 0.5), (9, 1, 1, 2.0, 1.0, 1.0)])
def test_prism_sum_rule(mesh):
    """mean over the box of sum_j N(r_i - r_j) == self term of the whole box."""
    nx, ny, nz, dx, dy, dz = mesh
    Nt = nw.mesh_tensor(nx, ny, nz, dx, dy, dz)
    oz = np.arange(-nz + 1, nz)
    oy = np.arange(-ny + 1, ny)
    ox = np.arange(-nx + 1, nx)
    mult = ((nz - np.abs(oz))[:, None, None] * (ny - np.abs(oy))[None, :, None]
            * (nx - np.abs(ox))[None, None, :])
    total = (Nt * mult[None]).sum(axis=(1, 2, 3)) / (nx * ny * nz)
    box = nw.tensor_exact(0.0, 0.0, 0.0, nx * dx, ny * dy, nz * dz)
    np.testing.assert_allclose(total, box, rtol=0, atol=1e-12)


def test_wide_thin_film_limit():
    Nt = nw.mesh_tensor(64, 64, 1, 1.0, 1.0, 0.2)
    # field at the centre of a uniformly magnetised (along z) wide film -> N_zz ~ 1
    # sum over all offsets = field factor at the centre of a 127 x 127 x 1 film
    tz = Nt[2].sum()
    assert 0.99 < tz < 1.0


def _clenshaw_curtis(n):
    """Clenshaw-Curtis nodes and weights on [0, 1] (n + 1 Chebyshev points, n even): a
    quadrature family independent of the oracle's Gauss-Legendre tent rule."""
    k = np.arange(n + 1)
    theta = np.pi * k / n
    x = 0.5 * (1.0 - np.cos(theta))
    w = np.zeros(n + 1)
    for i in range(n + 1):
        s = 0.0
        for j in range(1, n // 2 + 1):
            b = 1.0 if 2 * j == n else 2.0
            s += b * np.cos(2 * j * theta[i]) / (4 * j * j - 1)
        c = 1.0 if i in (0, n) else 2.0
        w[i] = c / n * (1.0 - s)
    return x, 0.5 * w


def _far_reference(R, d, n=32):
    """Tent average of the point-dipole kernel, each half-tent by Clenshaw-Curtis."""
    x, w = _clenshaw_curtis(n)
    axes = []
    for dc in d:
        t = np.concatenate([dc * x, -dc * x])
        wt = np.concatenate([w * (1.0 - x), w * (1.0 - x)])   # density (1 - |t|/d)/d, dt = d du
        axes.append((t, wt))
    TX, TY, TZ = np.meshgrid(axes[0][0], axes[1][0], axes[2][0], indexing="ij")
    W = np.einsum("i,j,k->ijk", axes[0][1], axes[1][1], axes[2][1])
    rx, ry, rz = R[0] + TX, R[1] + TY, R[2] + TZ
    r2 = rx * rx + ry * ry + rz * rz
    inv5 = W / (r2 * r2 * np.sqrt(r2))
    out = np.array([(inv5 * (r2 - 3 * rx * rx)).sum(), (inv5 * (r2 - 3 * ry * ry)).sum(),
                    (inv5 * (r2 - 3 * rz * rz)).sum(), (inv5 * (-3 * rx * ry)).sum(),
                    (inv5 * (-3 * rx * rz)).sum(), (inv5 * (-3 * ry * rz)).sum()])
    return out * (d[0] * d[1] * d[2] / (4.0 * math.pi))


@pytest.mark.parametrize("cell", [(1.0, 1.0, 1.0), (2.0, 2.0, 1.0), (1.0, 1.0, 0.25)])
def test_far_bands_against_an_independent_quadrature(cell):
    """The oracle's tensor beyond the switch (its band table of Gauss-Legendre orders)
    against the same cell-pair average integrated by Clenshaw-Curtis on each half-tent,
    at radii inside every band."""
    rng = np.random.default_rng(11)
    dm = max(cell)
    for r in (3.5, 5.0, 9.0, 20.0, 60.0, 200.0):
        dirv = rng.normal(size=3)
        R = dirv / np.linalg.norm(dirv) * r * dm
        got = nw.tensor(*R, *cell)
        ref = _far_reference(R, cell)
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), (r, got, ref)
