"""Newell demagnetisation tensor of a regular cell mesh (oracle, FP64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Paper: Sec. "Magnetostatic energy", Eqs. 6-8.  The demag field is the
cell-averaged field H_d,i = -sum_j N_{i-j} M_j, N a symmetric 3x3 tensor
that depends only on the offset between two equal rectangular cells
(Newell, Williams & Dunlop, JGR 98, 9551 (1993), cited by the paper).

Two evaluations of the same quantity are used:

* near field -- Newell's closed form: N_xx is the 27-point second
  difference of f(x,y,z) over the offsets {X-dx, X, X+dx} x ... divided by
  4*pi*dx*dy*dz, N_xy the same second difference of g(x,y,z).  The other
  four components follow by permuting axes.
* far field -- N(R) = V * E_t[ G(R + t) ] with G(r) = (r^2 I - 3 r r^T) /
  (4*pi*r^5) the point-dipole kernel and t the difference of two points
  drawn uniformly from the cell, i.e. t has the tent density
  prod_a (1 - |t_a|/d_a)/d_a on [-d_a, d_a].  Each half-tent is integrated
  with q-point Gauss-Legendre.  The closed form loses about eps*(r/d)^6 to
  cancellation; the quadrature converges geometrically once r >> d, so the
  closed form is used for |R| <= SWITCH * max(d) and quadrature beyond.

Parity: pinned by tests/test_oracle_newell.py -- trace N(0) = 1 for any
prism and 1/3 per axis for a cube, trace N(R != 0) = 0, parity and axis
permutation symmetries, agreement of both evaluations across the switch,
convergence to the point dipole, and the prism sum rule (the mean over a
box of all pair tensors equals the closed-form self term of the box).
"""
from __future__ import annotations

import math

import numpy as np

SWITCH = 3.0          # closed form for |R| <= SWITCH * max(dx, dy, dz)


# ---------------------------------------------------------------- closed form

def _safe_div(a, b):
    return np.where(b > 0, a / np.where(b > 0, b, 1.0), 0.0)


def newell_f(x, y, z):
    """Newell's f(x,y,z); even in each argument (Newell 1993, eq. 27)."""
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    rxz = np.sqrt(x2 + z2)
    rxy = np.sqrt(x2 + y2)
    out = (2.0 * x2 - y2 - z2) * R / 6.0
    out = out + np.where(rxz > 0, 0.5 * y * (z2 - x2) * np.arcsinh(_safe_div(y, rxz)), 0.0)
    out = out + np.where(rxy > 0, 0.5 * z * (y2 - x2) * np.arcsinh(_safe_div(z, rxy)), 0.0)
    out = out - np.where(x * R > 0, x * y * z * np.arctan(_safe_div(y * z, x * R)), 0.0)
    return out


def newell_g(x, y, z):
    """Newell's g(x,y,z); odd in x and in y, even in z (Newell 1993, eq. 32)."""
    sgn = np.sign(x) * np.sign(y)
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    rxy = np.sqrt(x2 + y2)
    ryz = np.sqrt(y2 + z2)
    rxz = np.sqrt(x2 + z2)
    out = -x * y * R / 3.0
    out = out + np.where(rxy > 0, x * y * z * np.arcsinh(_safe_div(z, rxy)), 0.0)
    out = out + np.where(ryz > 0, y / 6.0 * (3.0 * z2 - y2) * np.arcsinh(_safe_div(x, ryz)), 0.0)
    out = out + np.where(rxz > 0, x / 6.0 * (3.0 * z2 - x2) * np.arcsinh(_safe_div(y, rxz)), 0.0)
    out = out - np.where(z * R > 0, z * z2 / 6.0 * np.arctan(_safe_div(x * y, z * R)), 0.0)
    out = out - np.where(y * R > 0, z * y2 / 2.0 * np.arctan(_safe_div(x * z, y * R)), 0.0)
    out = out - np.where(x * R > 0, z * x2 / 2.0 * np.arctan(_safe_div(y * z, x * R)), 0.0)
    return sgn * out


def _second_difference(fun, X, Y, Z, dx, dy, dz):
    """sum over e in {-1,0,1}^3 of prod_a w(e_a) fun(X+e_x dx, ...), w(0)=2, w(+-1)=-1."""
    w = {-1: -1.0, 0: 2.0, 1: -1.0}
    acc = np.zeros(np.broadcast(X, Y, Z).shape)
    for ex in (-1, 0, 1):
        for ey in (-1, 0, 1):
            for ez in (-1, 0, 1):
                acc = acc + w[ex] * w[ey] * w[ez] * fun(X + ex * dx, Y + ey * dy, Z + ez * dz)
    return acc / (4.0 * math.pi * dx * dy * dz)


def nxx_exact(X, Y, Z, dx, dy, dz):
    return _second_difference(newell_f, X, Y, Z, dx, dy, dz)


def nxy_exact(X, Y, Z, dx, dy, dz):
    return _second_difference(newell_g, X, Y, Z, dx, dy, dz)


def tensor_exact(X, Y, Z, dx, dy, dz):
    """Closed-form tensor, components stacked as (xx, yy, zz, xy, xz, yz)."""
    X, Y, Z = np.broadcast_arrays(np.asarray(X, float), np.asarray(Y, float), np.asarray(Z, float))
    return np.stack([
        nxx_exact(X, Y, Z, dx, dy, dz),
        nxx_exact(Y, X, Z, dy, dx, dz),
        nxx_exact(Z, Y, X, dz, dy, dx),
        nxy_exact(X, Y, Z, dx, dy, dz),
        nxy_exact(X, Z, Y, dx, dz, dy),
        nxy_exact(Y, Z, X, dy, dz, dx),
    ])


# ---------------------------------------------------------------- far field

def _tent_rule(d, q):
    """Nodes and weights of E[phi(t)], t with density (1-|t|/d)/d on [-d, d]."""
    x, w = np.polynomial.legendre.leggauss(q)
    u = 0.5 * (1.0 + x)
    wt = 0.5 * w * (1.0 - u)
    return np.concatenate([d * u, -d * u]), np.concatenate([wt, wt])


def tensor_far(X, Y, Z, dx, dy, dz, q):
    """Tent-averaged point-dipole tensor (xx, yy, zz, xy, xz, yz) with q nodes per half-tent."""
    X, Y, Z = np.broadcast_arrays(np.asarray(X, float), np.asarray(Y, float), np.asarray(Z, float))
    tx, wx = _tent_rule(dx, q)
    ty, wy = _tent_rule(dy, q)
    tz, wz = _tent_rule(dz, q)
    acc = np.zeros((6,) + X.shape)
    for a in range(2 * q):
        for b in range(2 * q):
            for c in range(2 * q):
                rx, ry, rz = X + tx[a], Y + ty[b], Z + tz[c]
                r2 = rx * rx + ry * ry + rz * rz
                inv5 = 1.0 / (r2 * r2 * np.sqrt(r2))
                w = wx[a] * wy[b] * wz[c] * inv5
                acc[0] += w * (r2 - 3.0 * rx * rx)
                acc[1] += w * (r2 - 3.0 * ry * ry)
                acc[2] += w * (r2 - 3.0 * rz * rz)
                acc[3] += w * (-3.0 * rx * ry)
                acc[4] += w * (-3.0 * rx * rz)
                acc[5] += w * (-3.0 * ry * rz)
    return acc * (dx * dy * dz / (4.0 * math.pi))


def far_order(r_over_d):
    """Gauss-Legendre nodes per half-tent for a given |R| / max(d).

    Each band is one order above the smallest q whose result agrees with
    q = 16 to ~1e-13 relative for all directions and cell aspect ratios
    down to 1:4 (checked in tests/test_oracle_newell.py).
    """
    r = np.asarray(r_over_d)
    return np.select([r <= 4, r <= 6, r <= 12, r <= 32, r <= 128], [10, 8, 7, 6, 5], 4)


def tensor(X, Y, Z, dx, dy, dz):
    """The oracle's tensor: closed form near, quadrature far; shape (6,) + X.shape."""
    X, Y, Z = np.broadcast_arrays(np.asarray(X, float), np.asarray(Y, float), np.asarray(Z, float))
    dmax = max(dx, dy, dz)
    rr = np.sqrt(X * X + Y * Y + Z * Z) / dmax
    out = np.zeros((6,) + X.shape)
    near = rr <= SWITCH
    if near.any():
        out[:, near] = tensor_exact(X[near], Y[near], Z[near], dx, dy, dz)
    qs = far_order(rr)
    for q in np.unique(qs[~near]):
        sel = (~near) & (qs == q)
        out[:, sel] = tensor_far(X[sel], Y[sel], Z[sel], dx, dy, dz, int(q))
    return out


# ---------------------------------------------------------------- whole mesh

# parity of each component under i -> -i, j -> -j, k -> -k
PARITY = {0: (1, 1, 1), 1: (1, 1, 1), 2: (1, 1, 1), 3: (-1, -1, 1), 4: (-1, 1, -1), 5: (1, -1, -1)}


def mesh_tensor(nx, ny, nz, dx, dy, dz, chunk=200000):
    """N for every offset (i, j, k), |i| < nx etc.

    Returns an array of shape (6, 2nz-1, 2ny-1, 2nx-1) whose entry
    [c, k + nz-1, j + ny-1, i + nx-1] is component c at offset (i dx, j dy, k dz).
    The first octant is evaluated; the rest follows from the parities above.
    """
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    X = (I * dx).ravel(); Y = (J * dy).ravel(); Z = (K * dz).ravel()
    oct_ = np.empty((6, X.size))
    for s in range(0, X.size, chunk):
        oct_[:, s:s + chunk] = tensor(X[s:s + chunk], Y[s:s + chunk], Z[s:s + chunk], dx, dy, dz)
    oct_ = oct_.reshape(6, nx, ny, nz).transpose(0, 3, 2, 1)     # (6, nz, ny, nx)
    full = np.empty((6, 2 * nz - 1, 2 * ny - 1, 2 * nx - 1))
    for c in range(6):
        px, py, pz = PARITY[c]
        for sz in (1, -1):
            for sy in (1, -1):
                for sx in (1, -1):
                    sign = (px if sx < 0 else 1) * (py if sy < 0 else 1) * (pz if sz < 0 else 1)
                    block = oct_[c]
                    if sz < 0:
                        block = block[::-1]
                    if sy < 0:
                        block = block[:, ::-1]
                    if sx < 0:
                        block = block[:, :, ::-1]
                    zs = slice(nz - 1, 2 * nz - 1) if sz > 0 else slice(0, nz)
                    ys = slice(ny - 1, 2 * ny - 1) if sy > 0 else slice(0, ny)
                    xs = slice(nx - 1, 2 * nx - 1) if sx > 0 else slice(0, nx)
                    full[c, zs, ys, xs] = sign * block
    return full


def as_matrix(t6):
    """(6, ...) -> (3, 3, ...) symmetric matrices."""
    xx, yy, zz, xy, xz, yz = t6
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])
