"""Pins for oracle.integrate: tableau, closed forms, convergence order (no GPU)."""
import math
import os
from fractions import Fraction as Fr
from itertools import product

import numpy as np
import pytest

import synth
from oracle import demag as D
from oracle import fields as F
from oracle import integrate as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                out[k] = [float(x) for x in v] if len(v) > 1 else float(v[0])
    return out


def test_tableau_order_conditions():
    """Butcher order conditions: b to order 5, bhat to order 4, row sums = c."""
    A, c, b, bh = I.A_FR, I.C_FR, I.B5_FR, I.B4_FR
    s = 7
    a = [[A[i][j] if j < len(A[i]) else Fr(0) for j in range(s)] for i in range(s)]
    for i in range(s):
        assert sum(a[i]) == c[i]

    def conds(w, order):
        out = []
        ac = [sum(a[i][j] * c[j] for j in range(s)) for i in range(s)]
        ac2 = [sum(a[i][j] * c[j] ** 2 for j in range(s)) for i in range(s)]
        aac = [sum(a[i][j] * ac[j] for j in range(s)) for i in range(s)]
        ac3 = [sum(a[i][j] * c[j] ** 3 for j in range(s)) for i in range(s)]
        acac = [sum(a[i][j] * c[j] * ac[j] for j in range(s)) for i in range(s)]
        aac2 = [sum(a[i][j] * ac2[j] for j in range(s)) for i in range(s)]
        aaac = [sum(a[i][j] * aac[j] for j in range(s)) for i in range(s)]
        S = lambda v: sum(w[i] * v[i] for i in range(s))
        one = [Fr(1)] * s
        out += [(S(one), Fr(1))]
        if order >= 2:
            out += [(S(c), Fr(1, 2))]
        if order >= 3:
            out += [(S([x ** 2 for x in c]), Fr(1, 3)), (S(ac), Fr(1, 6))]
        if order >= 4:
            out += [(S([x ** 3 for x in c]), Fr(1, 4)), (S([c[i] * ac[i] for i in range(s)]), Fr(1, 8)),
                    (S(ac2), Fr(1, 12)), (S(aac), Fr(1, 24))]
        if order >= 5:
            out += [(S([x ** 4 for x in c]), Fr(1, 5)), (S([c[i] ** 2 * ac[i] for i in range(s)]), Fr(1, 10)),
                    (S([ac[i] ** 2 for i in range(s)]), Fr(1, 20)), (S([c[i] * ac2[i] for i in range(s)]), Fr(1, 15)),
                    (S(ac3), Fr(1, 20)), (S([c[i] * aac[i] for i in range(s)]), Fr(1, 30)),
                    (S(acac), Fr(1, 40)), (S(aac2), Fr(1, 60)), (S(aaac), Fr(1, 120))]
        return out

    for got, want in conds(b, 5):
        assert got == want
    for got, want in conds(bh, 4):
        assert got == want
    # the embedded pair differs at fifth order
    assert any(g != w for g, w in conds(bh, 5))
    # FSAL: the last row of A is b
    assert a[6][:6] == b[:6]


def _macrospin(alpha, gamma, Hz):
    mesh = synth.Mesh(1, 1, 1, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, H=(0.0, 0.0, Hz), alpha=alpha, gamma=gamma)
    Ms = F.ms_array(mesh, mat)
    Nt = D.mesh_tensor(mesh)
    f = lambda m: F.rhs(mesh, mat, m, Ms, Nt, "direct")[0]
    return mesh, mat, f


def _closed(alpha, gamma, Hz, t):
    gt = gamma / (1 + alpha ** 2)
    w = gt * Hz * t
    return np.array([math.cos(w) / math.cosh(alpha * w), math.sin(w) / math.cosh(alpha * w),
                     math.tanh(alpha * w)])


def test_macrospin_closed_form_at_1ns():
    g = _golden("macrospin_precession.txt")
    _, mat, f = _macrospin(g["alpha"], g["gamma"], g["Hz"])
    m0 = np.array(g["m0"]).reshape(3, 1, 1, 1)
    m, st = I.run(f, m0, 1e-6, t_end=g["t_end"])
    assert abs(st.t - g["t_end"]) < 1e-21
    err = np.abs(m.ravel() - _closed(g["alpha"], g["gamma"], g["Hz"], st.t)).max()
    assert err < 2e-6
    assert abs(np.linalg.norm(m.ravel()) - 1) < 1e-15


def test_larmor_frequency_without_damping():
    g = _golden("macrospin_precession.txt")
    gamma, Hz = g["gamma"], g["Hz"]
    _, _, f = _macrospin(0.0, gamma, Hz)
    T = 2 * math.pi / (gamma * Hz)
    m, st = I.run(f, np.array([1.0, 0, 0]).reshape(3, 1, 1, 1), 1e-8, t_end=3 * T)
    np.testing.assert_allclose(m.ravel(), [1.0, 0.0, 0.0], atol=1e-6)


def test_fifth_order_convergence():
    _, _, f = _macrospin(0.1, 2.21e5, 1e5)
    m0 = np.array([1.0, 0, 0]).reshape(3, 1, 1, 1)
    t = 2e-10
    errs = []
    for n in (20, 40):
        m = I.fixed_step_rk5(f, m0, t / n, n)
        # the unprojected fixed-step solution is compared with the closed form
        errs.append(np.abs(m.ravel() - _closed(0.1, 2.21e5, 1e5, t)).max())
    order = math.log2(errs[0] / errs[1])
    assert 4.6 < order < 5.4, order


def test_norm_preserved_and_energy_decays():
    mesh = synth.Mesh(6, 6, 1, 2.5e-9, 2.5e-9, 3e-9)
    mat = synth.Material(Ms=8.6e5, A=1.3e-11, alpha=0.5, H=(10 * synth.MT, 0, 0))
    Ms = F.ms_array(mesh, mat)
    Nt = D.mesh_tensor(mesh)
    f = lambda m: F.rhs(mesh, mat, m, Ms, Nt, "direct")[0]
    m = synth.random_state(1, mesh)
    st = I.Stepper(rtol=1e-6)
    E0 = F.energies(mesh, mat, m, Ms, Nt, "direct")["total"]
    for _ in range(40):
        m, acc = I.step(f, m, st)
        assert np.abs(np.sqrt((m * m).sum(axis=0)) - 1).max() < 1e-15
        if acc:
            E1 = F.energies(mesh, mat, m, Ms, Nt, "direct")["total"]
            assert E1 <= E0 + 1e-6 * abs(E0)
            E0 = E1


def test_stoner_wohlfarth_switching_field():
    """Listing 2 sweep around the closed-form switching field (50 mT)."""
    g = _golden("stoner_wohlfarth_listing2.txt")
    mesh = synth.Mesh(int(g["nx"]), int(g["ny"]), int(g["nz"]), 2e-9, 2e-9, 2e-9)
    Ms0 = g["Ms"]
    step = g["step_mT"]
    mat = synth.Material(Ms=Ms0, A=g["A"], Ku=g["Ku"], u=tuple(g["axis"]), alpha=0.5, precession=0, demag=0)
    Ms = F.ms_array(mesh, mat)
    mT = 1e-3 / F.MU0
    sw_mT = g["Ku"] / Ms0 * 1e3                      # mu0 H_sw = Ku / Ms
    assert abs(sw_mT - 50.0) < 1e-9
    m = synth.tilt(synth.uniform_state(mesh, (-1, 0, 0)), 9, 1e-3)
    states = {}
    for i in (int(g["imin"]), 9, 11):
        mat.H = (i * step * mT, 0.0, 0.0)
        f = lambda y: F.rhs(mesh, mat, y, Ms, None, "fft")[0]
        # rtol 1e-8: with 2 nm cells the exchange modes make the step stability-limited
        # (h ~ 1e-12 s) and the controller's error noise (~ rtol * 2e12 /s) must stay
        # below the stopping threshold
        m, st = I.run(f, m, 1e-8, max_dmdt=1e6, max_steps=6000)
        assert st.last_maxdmdt < 1e6, (i, st.last_maxdmdt)
        states[i] = m[0].mean()
    assert states[9] < 0.0 < states[11]
