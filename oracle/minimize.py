"""Steepest-descent energy minimisation with Barzilai-Borwein steps (oracle, FP64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Paper: Sec. "Steepest descent energy minimization".  Per cell, with
f = m x H_eff(m) and g = m x (m x H_eff(m)), the step

    m_{k+1} = m_k - tau_k (m_k + m_{k+1}) / 2 x f_k

is solved explicitly, as the paper writes it, from

    (1 + tau_k^2 |f_k|^2 / 4) m_{k+1} = (1 - tau_k^2 |f_k|^2 / 4) m_k - tau_k g_k,

which keeps |m| unchanged.  The step size follows the Barzilai-Borwein
rules, with sums over all cells of one simulation,

    tau^1 = sum s.s / sum s.y,     tau^2 = sum s.y / sum y.y,
    s = m_k - m_{k-1},             y = g_k - g_{k-1}.

Readings where the paper is silent (the CUDA path takes the same ones):
  * the two rules alternate: tau^1 on odd steps k, tau^2 on even steps
    k >= 2 (the alternation of the cited Abert et al. 2014);
  * the first step uses tau_0 = 0.01 / max_i |g_i|, so that no cell turns
    by much more than 0.01 rad;
  * where the rule's value is not positive and finite (s.y <= 0: the energy
    is not convex along the last step) the step falls back to the safe size
    0.01 / max_i |g_i| at m_k (keeping the previous tau can freeze a tiny
    step for good: seen from random starts);
  * every step is capped at tau <= 1 / max_i |g_i|, so no cell turns by more
    than about one radian (without it, from a random start the rules produce
    rotations of hundreds of radians and the state never settles; with it the
    32x32x1 random start of the film_relax workload converges in ~850 steps to
    the minimum the damped RK45 relaxation finds);
  * a simulation stops once max_i |dm/dt|_i < max_dmdt (rad/s) at m_k, with
    dm/dt the LL right-hand side of its material (precession flag honoured):
    |dm/dt| = gamma/(1+alpha^2) |g| times alpha, or times sqrt(1+alpha^2)
    with precession;
  * cells with Ms = 0 do not move (f = g = 0 there).

Parity: pinned by tests/test_oracle_minimize.py -- the explicit update
satisfies the implicit midpoint equation above and keeps |m|; a macrospin
with uniaxial anisotropy and a transverse field relaxes to the
Stoner-Wohlfarth angle sin(theta) = mu0 Ms H / (2 Ku); a small film relaxes
to the energy of the damped RK45 relaxation of integrate.run.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


MAX_TURN = 1.0     # rad: cap of tau * max|g| per step


def _cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def update(m, f, g, tau):
    """The norm-preserving step for step size tau (the paper's explicit form)."""
    a = 0.25 * tau * tau * (f * f).sum(axis=0)
    return ((1.0 - a)[None] * m - tau * g) / (1.0 + a)[None]


def dmdt_scale(mat):
    """|dm/dt| / |g| of the LL right-hand side of the material."""
    gt = mat.gamma / (1.0 + mat.alpha ** 2)
    return gt * (np.sqrt(1.0 + mat.alpha ** 2) if mat.precession else mat.alpha)


@dataclass
class Minimizer:
    tau: float = 0.0
    k: int = 0                   # steps taken
    last_maxdmdt: float = np.inf
    converged: bool = False
    m_prev: np.ndarray | None = None
    g_prev: np.ndarray | None = None


def minimize(field, m, mat, Ms, max_dmdt=0.0, max_steps=10 ** 6, st: Minimizer | None = None):
    """Steepest descent from m; field(m) returns H_eff (A/m).  Returns (m, state)."""
    st = st or Minimizer()
    has = (Ms > 0)[None]
    scale = dmdt_scale(mat)
    while st.k < max_steps:
        H = field(m)
        f = _cross(m, H) * has
        g = _cross(m, f)
        maxg = float(np.sqrt((g * g).sum(axis=0).max()))
        st.last_maxdmdt = maxg * scale
        if max_dmdt > 0.0 and st.last_maxdmdt < max_dmdt:
            st.converged = True
            break
        if st.k == 0:
            st.tau = 0.01 / maxg if maxg > 0.0 else 0.0
        else:
            s = m - st.m_prev
            y = g - st.g_prev
            ss, sy, yy = float((s * s).sum()), float((s * y).sum()), float((y * y).sum())
            with np.errstate(divide="ignore", invalid="ignore"):
                cand = ss / sy if st.k % 2 == 1 else sy / yy
            if np.isfinite(cand) and cand > 0.0:
                st.tau = float(cand)
            else:
                st.tau = 0.01 / maxg if maxg > 0.0 else 0.0   # negative curvature: the safe step
        if maxg > 0.0:
            st.tau = min(st.tau, MAX_TURN / maxg)              # no cell turns by more than ~1 rad
        st.m_prev, st.g_prev = m, g
        m = update(m, f, g, st.tau)
        st.k += 1
    return m, st
