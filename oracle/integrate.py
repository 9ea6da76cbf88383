"""Adaptive Dormand-Prince RK45 with projection to |m| = 1 (oracle, FP64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Paper: Sec. "LLG equation" -- the LL form is integrated with the adaptive
Dormand-Prince member of the Runge-Kutta family, and m is projected onto
the unit sphere after every successful step.  The tableau is Dormand &
Prince (1980), RK5(4)7M, which the paper uses without printing it.

Readings where the paper is silent (the CUDA path takes the same ones):
  * error = max over cells and components of |h sum_j (b_j - bhat_j) k_j|,
    divided by rtol (absolute = relative tolerance because |m| = 1);
  * accept when error <= 1; h <- h * clamp(0.9 error^(-1/5), 0.2, 5);
  * h0 = min(1e-12 s, 0.01 / max_i |dm/dt|_i) at the first step;
  * after the projection k1 is recomputed at the projected m (7 right-hand
    sides per attempted step);
  * the last step is clipped to land on t_end;
  * relaxation stops once max_i |dm/dt|_i < max_dmdt (rad/s) at the start
    of an attempt.

Parity: pinned by tests/test_oracle_integrate.py -- the tableau's order
conditions up to fifth order (exact rationals), the macrospin closed form
of Sec. "A magnetic moment under an external magnetic field", the Larmor
frequency at alpha = 0, fifth-order convergence with fixed steps, |m| = 1
after each step, energy decay under damping, and the Stoner-Wohlfarth
switching field of the field sweep of Listing 2.
"""
from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction as Fr

import numpy as np

# Dormand & Prince (1980), RK5(4)7M
C_FR = [Fr(0), Fr(1, 5), Fr(3, 10), Fr(4, 5), Fr(8, 9), Fr(1), Fr(1)]
A_FR = [
    [],
    [Fr(1, 5)],
    [Fr(3, 40), Fr(9, 40)],
    [Fr(44, 45), Fr(-56, 15), Fr(32, 9)],
    [Fr(19372, 6561), Fr(-25360, 2187), Fr(64448, 6561), Fr(-212, 729)],
    [Fr(9017, 3168), Fr(-355, 33), Fr(46732, 5247), Fr(49, 176), Fr(-5103, 18656)],
    [Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84)],
]
B5_FR = [Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84), Fr(0)]
B4_FR = [Fr(5179, 57600), Fr(0), Fr(7571, 16695), Fr(393, 640), Fr(-92097, 339200),
         Fr(187, 2100), Fr(1, 40)]

A = [[float(x) for x in row] for row in A_FR]
B5 = [float(x) for x in B5_FR]
E = [float(b - bh) for b, bh in zip(B5_FR, B4_FR)]


def normalize(m):
    n = np.sqrt((m * m).sum(axis=0))
    return m / np.where(n > 0, n, 1.0)[None]


def attempt(f, m, h, k1=None):
    """One Dormand-Prince attempt from m with step h.

    f(y) returns dm/dt at y.  Returns (y5, errvec, k) with y5 the
    fifth-order solution (not yet projected) and errvec = h sum e_j k_j.
    """
    k = [f(m) if k1 is None else k1]
    for s in range(1, 7):
        y = m.copy()
        for j in range(s):
            if A[s][j] != 0.0:
                y = y + h * A[s][j] * k[j]
        k.append(f(y))
    y5 = m.copy()
    for j in range(7):
        if B5[j] != 0.0:
            y5 = y5 + h * B5[j] * k[j]
    err = np.zeros_like(m)
    for j in range(7):
        if E[j] != 0.0:
            err = err + E[j] * k[j]
    return y5, h * err, k


def max_norm(v):
    """max over cells of the Euclidean norm of a (3, ...) field."""
    return float(np.sqrt((v * v).sum(axis=0)).max()) if v.size else 0.0


@dataclass
class Stepper:
    """State of one adaptive integration (t, h, counters)."""
    rtol: float
    t: float = 0.0
    h: float = 0.0
    t_end: float = 0.0
    n_acc: int = 0
    n_rej: int = 0
    last_err: float = 0.0
    last_maxdmdt: float = 0.0


def done_time(st):
    return st.t_end > 0.0 and st.t_end - st.t <= 1e-12 * st.t_end


def step(f, m, st: Stepper, max_dmdt=0.0, reduce=None):
    """Attempt one step.

    Returns (m, status): status 1 accepted (m projected), 0 rejected,
    2 converged (max|dm/dt| at m below max_dmdt; nothing stepped).
    reduce (optional) turns a maximum over the local state into the maximum over
    a state split across processes (the max|dm/dt| and the error norm); the
    default is the local maximum itself.
    """
    red = reduce if reduce is not None else (lambda x: x)
    k1 = f(m)
    st.last_maxdmdt = red(max_norm(k1))
    if max_dmdt > 0.0 and st.last_maxdmdt < max_dmdt:
        return m, 2
    if st.h <= 0.0:
        st.h = min(1e-12, 0.01 / st.last_maxdmdt) if st.last_maxdmdt > 0 else 1e-12
        if st.t_end > 0.0:
            st.h = min(st.h, st.t_end - st.t)
    h = st.h
    y5, errvec, _ = attempt(f, m, h, k1)
    err = red(float(np.abs(errvec).max()) if errvec.size else 0.0) / st.rtol
    st.last_err = err
    if not np.isfinite(err):
        raise FloatingPointError("non-finite error norm")
    factor = 5.0 if err == 0.0 else min(5.0, max(0.2, 0.9 * err ** -0.2))
    accepted = err <= 1.0
    if accepted:
        m = normalize(y5)
        st.t += h
        st.n_acc += 1
    else:
        st.n_rej += 1
    st.h = h * factor
    if st.t_end > 0.0:
        st.h = min(st.h, st.t_end - st.t)
    return m, int(accepted)


def run(f, m, rtol, t_end=0.0, max_dmdt=0.0, max_steps=10 ** 9, st: Stepper | None = None):
    """Integrate until t_end (if > 0), or until max|dm/dt| < max_dmdt (if > 0).

    Returns (m, stepper).  The relaxation test is made on the k1 of each
    attempt, i.e. at the current (projected) m.
    """
    st = st or Stepper(rtol=rtol)
    st.t_end = t_end
    attempts = 0
    while attempts < max_steps and not done_time(st):
        m, status = step(f, m, st, max_dmdt)
        if status == 2:
            break
        attempts += 1
    return m, st


def fixed_step_rk5(f, m, h, nsteps):
    """Fixed-step fifth-order solution without projection (convergence-order test)."""
    for _ in range(nsteps):
        m, _, _ = attempt(f, m, h)
    return m
