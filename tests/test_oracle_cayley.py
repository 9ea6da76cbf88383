"""Pins for oracle.cayley: the Cayley map, the dcayinv dynamics, fourth-order
convergence and the accuracy claim of Sec. "Cayley transform" (no GPU)."""
import math

import numpy as np

import synth
from oracle import cayley as CY
from oracle import fields as F


def _skew(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def test_cayley_map_matches_its_matrix_definition_and_keeps_the_norm():
    rng = np.random.default_rng(2)
    w = rng.standard_normal((3, 4, 5)) * 1.5
    m = rng.standard_normal((3, 4, 5))
    got = CY.cay(w, m)
    for j in range(4):
        for i in range(5):
            Om = _skew(w[:, j, i])
            Q = np.linalg.solve(np.eye(3) - 0.5 * Om, np.eye(3) + 0.5 * Om)
            np.testing.assert_allclose(got[:, j, i], Q @ m[:, j, i], rtol=0, atol=1e-14 * np.abs(m).max())
            assert abs(np.linalg.det(Q) - 1.0) < 1e-13          # a rotation
    np.testing.assert_allclose(np.sqrt((got ** 2).sum(0)), np.sqrt((m ** 2).sum(0)), rtol=1e-14)


def test_omega_dynamics_reproduce_the_rotation_for_a_constant_f():
    """dQ/dt = skew[f] Q with constant f is the rotation about f by |f| t (Rodrigues)."""
    rng = np.random.default_rng(7)
    f = rng.standard_normal((3, 1, 6))
    m0 = rng.standard_normal((3, 1, 6))
    m0 /= np.sqrt((m0 ** 2).sum(0))[None]
    t = 1.0 / np.sqrt((f ** 2).sum(0)).max()           # about one radian for the largest |f|
    w = np.zeros_like(f)
    n = 200
    h = t / n
    for _ in range(n):                                 # RK4 on omega without restarts
        k1 = CY.omega_rhs(w, f)
        k2 = CY.omega_rhs(w + 0.5 * h * k1, f)
        k3 = CY.omega_rhs(w + 0.5 * h * k2, f)
        k4 = CY.omega_rhs(w + h * k3, f)
        w = w + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    m = CY.cay(w, m0)
    fn = np.sqrt((f ** 2).sum(0))
    k = f / fn[None]
    th = fn * t
    kxm = np.stack([k[1] * m0[2] - k[2] * m0[1], k[2] * m0[0] - k[0] * m0[2], k[0] * m0[1] - k[1] * m0[0]])
    ref = m0 * np.cos(th)[None] + kxm * np.sin(th)[None] + k * (k * m0).sum(0)[None] * (1 - np.cos(th))[None]
    assert np.abs(m - ref).max() < 1e-10


def _macrospin(alpha):
    mesh = synth.Mesh(1, 1, 1, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, H=(0.0, 0.0, 1e5), alpha=alpha, gamma=2.21e5, demag=0)
    Ms = F.ms_array(mesh, mat)
    return mesh, mat, Ms, (lambda y: F.h_eff(mesh, mat, y, Ms))


def _closed(alpha, t):
    gt = 2.21e5 / (1 + alpha ** 2)
    w = gt * 1e5 * t
    return np.array([math.cos(w) / math.cosh(alpha * w), math.sin(w) / math.cosh(alpha * w),
                     math.tanh(alpha * w)])


def test_both_schemes_are_fourth_order_and_cayley_is_more_accurate():
    """The paper's macrospin comparison at t = 1 ns with alpha = 0.05 (figure of the
    absolute error): the Cayley scheme's error is far below the projected scheme's."""
    mesh, mat, Ms, field = _macrospin(0.05)
    m0 = np.array([1.0, 0, 0]).reshape(3, 1, 1, 1)
    ref = _closed(0.05, 1e-9)
    err = {}
    for cay in (True, False):
        for n in (500, 1000):
            m = CY.run(mesh, mat, Ms, field, m0, 1e-9 / n, n, cay)
            err[cay, n] = np.abs(m.ravel() - ref).max()
            assert abs(np.sqrt((m ** 2).sum()) - 1) < 1e-14
        order = math.log2(err[cay, 500] / err[cay, 1000])
        assert 3.7 < order < 4.3, (cay, order)
    assert err[True, 1000] < err[False, 1000] / 5


def test_masked_cells_do_not_move():
    mesh = synth.Mesh(4, 3, 1, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, H=(3e4, 0, 1e4), alpha=0.2, demag=0)
    Ms_cells = np.full(mesh.shape, 8e5)
    Ms_cells[0, 2, 1] = 0.0
    Ms = F.ms_array(mesh, mat, Ms_cells)
    m0 = synth.random_state(9, mesh)
    for cay in (True, False):
        m = CY.run(mesh, mat, Ms, lambda y: F.h_eff(mesh, mat, y, Ms), m0, 1e-13, 5, cay)
        assert np.array_equal(m[:, 0, 2, 1], m0[:, 0, 2, 1])
