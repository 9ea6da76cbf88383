"""Fixed-step classical Runge-Kutta for the LLG equation, with projection and on
the Cayley-transform variable (oracle, FP64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Paper: Sec. "Cayley transform".  The LL equation is written dm/dt = f x m with

    f = gamma (H + alpha m x H) / (1 + alpha^2)

(without precession only the damping part: f = gamma alpha m x H / (1 + alpha^2)),
so m(t) = Q(t) m_n for a rotation Q, taken as the Cayley transform
Q = (I - Omega/2)^-1 (I + Omega/2) of Omega = skew[omega], and omega follows the
vector form of the dcayinv equation

    d omega / dt = f - (omega x f) / 2 + (omega . f) omega / 4.

Classical Runge-Kutta integrates omega from omega = 0 over one step and sets
m_{n+1} = Q(omega_{n+1}) m_n.  The scheme it is compared with is classical
Runge-Kutta on dm/dt itself with projection onto |m| = 1 after the step (the
paper's comparison on the macrospin at t = 1 ns, "classical Runge-Kutta method
with projection" against "one utilizing a Cayley transformation").

Readings where the paper is silent (the CUDA path takes the same ones):
  * "classical Runge-Kutta" is the four-stage RK4 tableau;
  * omega restarts from 0 at every step (the paper requires restarts to keep
    |omega| small and does not say how often);
  * the projection scheme normalises m after each step, not inside the stages.

Parity: pinned by tests/test_oracle_cayley.py -- the closed form of
Q(omega) m equals the matrix definition and keeps |m|; for a constant f the
omega dynamics reproduce the rotation about f by the angle |f| t; both
schemes converge at fourth order to the macrospin closed form, and the Cayley
scheme's error at 1 ns is far below the projected scheme's (the paper's
observation).
"""
from __future__ import annotations

import numpy as np


def _cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def _dot(a, b):
    return (a * b).sum(axis=0)


def cay(omega, m):
    """Q(omega) m per cell, Q = (I - Omega/2)^-1 (I + Omega/2), Omega x = omega x x.
    (I - Omega/2) x = b has x = (b + omega x b / 2 + (omega . b) omega / 4) / (1 + |omega|^2 / 4)."""
    b = m + 0.5 * _cross(omega, m)
    return (b + 0.5 * _cross(omega, b) + 0.25 * _dot(omega, b)[None] * omega) / (1.0 + 0.25 * _dot(omega, omega))[None]


def f_vector(mat, m, H):
    """f of dm/dt = f x m for the LL equation of the material."""
    gt = mat.gamma / (1.0 + mat.alpha ** 2)
    f = mat.alpha * gt * _cross(m, H)
    if mat.precession:
        f = f + gt * H
    return f


def omega_rhs(omega, f):
    """d omega / dt, the vector form of the dcayinv equation."""
    return f - 0.5 * _cross(omega, f) + 0.25 * _dot(omega, f)[None] * omega


def rk4_cayley_step(fvec, m, h):
    """One classical RK4 step on omega (from omega = 0); fvec(m) returns f per cell."""
    k1 = fvec(m)                                   # omega = 0: d omega/dt = f
    w = 0.5 * h * k1
    k2 = omega_rhs(w, fvec(cay(w, m)))
    w = 0.5 * h * k2
    k3 = omega_rhs(w, fvec(cay(w, m)))
    w = h * k3
    k4 = omega_rhs(w, fvec(cay(w, m)))
    return cay(h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4), m)


def rk4_projected_step(rhs, m, h):
    """One classical RK4 step on dm/dt, then m <- m / |m|."""
    k1 = rhs(m)
    k2 = rhs(m + 0.5 * h * k1)
    k3 = rhs(m + 0.5 * h * k2)
    k4 = rhs(m + h * k3)
    y = m + h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    n = np.sqrt(_dot(y, y))
    return y / np.where(n > 0, n, 1.0)[None]


def run(mesh, mat, Ms, field, m, h, n_steps, cayley):
    """n_steps fixed steps of size h; field(m) returns H_eff.  Cells with Ms = 0 do not move."""
    has = (Ms > 0)[None]
    if cayley:
        fvec = lambda y: f_vector(mat, y, field(y)) * has
        for _ in range(n_steps):
            m = rk4_cayley_step(fvec, m, h)
    else:
        from oracle import fields as F
        rhs = lambda y: F.ll_rhs(mat, y, field(y), Ms)
        for _ in range(n_steps):
            y = rk4_projected_step(rhs, m, h)
            m = np.where(has, y, m)
    return m
