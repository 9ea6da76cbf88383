"""GPU parity of the extended terms against the FP64 oracle: bulk and D_2d DMI,
cell-based A and D, Zhang-Li and spin-orbit torques (the extended x-inverse
kernel), in the right-hand side, the energies, RK45 attempts and mixed
batches.

Tolerances as for the standard terms: FP64 1e-10 relative (max over cells),
FP32 1e-5 relative RMS.
"""
import numpy as np
import pytest

import synth
from oracle import demag as D
from oracle import fields as F
from oracle import integrate as I
from tests.gpu_util import make_ctx, max_rel, oracle_rhs, rms_rel

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


def _mat(mesh, kind, cells=False, stt=False, sot=False, seed=0, **kw):
    rng = np.random.default_rng(seed)
    base = dict(Ms=8e5, A=1.3e-11, D=3e-3, dmi=kind, Ku=4e5, u=(0.2, 0.3, 0.9), Kc=1e4, H=(1e4, -2e4, 3e4),
                alpha=0.3)
    if cells:
        base["A_cells"] = rng.uniform(0.5e-11, 2e-11, mesh.shape)
        # one sign: neighbours of opposite sign make the harmonic mean ill-conditioned
        base["D_cells"] = rng.uniform(1e-3, 4e-3, mesh.shape)
    if stt:
        base.update(u_stt=(60.0, -25.0, 10.0), beta=0.1)
    if sot:
        base.update(aJ=2e9, bJ=-7e8, p=(0.2, -0.5, 1.0))
    base.update(kw)
    return synth.Material(**base)


MESHES = [
    (7, 5, 1, 2e-9, 2.5e-9, 1.5e-9),     # film: one plane
    (9, 6, 3, 2e-9, 2e-9, 1e-9),         # cluster of 3 planes
    (5, 4, 9, 2e-9, 2e-9, 1e-9),         # separate y and z passes
    (33, 17, 2, 2e-9, 2e-9, 1e-9),       # ragged x and y tiles
]

CASES = [
    dict(kind=2),
    dict(kind=3),
    dict(kind=1, cells=True),
    dict(kind=2, cells=True, stt=True),
    dict(kind=3, sot=True),
    dict(kind=0, stt=True, sot=True),
    dict(kind=2, cells=True, stt=True, sot=True, precession=0),
]


@pytest.mark.parametrize("mesh", MESHES)
@pytest.mark.parametrize("case", range(len(CASES)))
def test_rhs_f64_matches_oracle(mesh, case):
    m = synth.Mesh(*mesh)
    sim = synth.Sim(m, _mat(m, seed=case, **CASES[case]), synth.random_state(3 + case, m))
    ctx = make_ctx("f64", [sim])
    dmdt, heff = ctx.rhs_host(sim.m0.ravel())
    ref_k, ref_H = oracle_rhs(sim, method="direct")
    assert max_rel(heff, ref_H) < TOL64
    assert max_rel(dmdt, ref_k) < TOL64


@pytest.mark.parametrize("case", [0, 1, 3, 6])
def test_rhs_f32_matches_oracle(case):
    m = synth.Mesh(24, 20, 3, 2e-9, 2e-9, 1e-9)
    sim = synth.Sim(m, _mat(m, seed=case, **CASES[case]), synth.random_state(8 + case, m))
    ctx = make_ctx("f32", [sim])
    dmdt, heff = ctx.rhs_host(sim.m0.ravel())
    ref_k, ref_H = oracle_rhs(sim, method="direct")
    assert rms_rel(heff, ref_H) < TOL32
    assert rms_rel(dmdt, ref_k) < TOL32


def test_masked_cells_with_extended_terms():
    m = synth.Mesh(9, 7, 3, 2e-9, 2e-9, 2e-9)
    Ms = np.full(m.shape, 8e5)
    Ms[1, 3, 4] = 0.0
    Ms[:, 0, :3] = 0.0
    Ms[2, 6, 8] = 4e5
    for case in (3, 6):
        sim = synth.Sim(m, _mat(m, seed=case, **CASES[case]), synth.random_state(5, m), Ms)
        ctx = make_ctx("f64", [sim])
        dmdt, heff = ctx.rhs_host(sim.m0.ravel())
        ref_k, ref_H = oracle_rhs(sim, method="direct")
        assert max_rel(heff, ref_H) < TOL64
        assert max_rel(dmdt, ref_k) < TOL64


@pytest.mark.parametrize("kind,cells", [(2, False), (3, True), (1, True)])
def test_energies_match_oracle(kind, cells):
    m = synth.Mesh(9, 6, 3, 2e-9, 2e-9, 1e-9)
    mat = _mat(m, kind, cells=cells, seed=4)
    sim = synth.Sim(m, mat, synth.random_state(9, m))
    ctx = make_ctx("f64", [sim])
    ctx.set_m(sim.m0.ravel())
    E = ctx.energy(0)
    Ms = F.ms_array(m, mat)
    ref = F.energies(m, mat, sim.m0, Ms, D.mesh_tensor(m), "direct")
    for term in ("exchange", "dmi", "total"):
        assert abs(E[term] - ref[term]) <= 1e-10 * max(abs(ref[term]), 1e-30), term


def test_mixed_batch_standard_and_extended():
    """One launch runs the extended kernel for the whole batch: the standard members
    still take their own path (interfacial DMI, uniform constants)."""
    m1 = synth.Mesh(12, 10, 1, 2e-9, 2e-9, 2e-9)
    m2 = synth.Mesh(9, 6, 3, 2e-9, 2e-9, 1e-9)
    sims = [synth.Sim(m1, _mat(m1, 1), synth.random_state(1, m1)),
            synth.Sim(m2, _mat(m2, 2, cells=True, stt=True, seed=2), synth.random_state(2, m2)),
            synth.Sim(m2, _mat(m2, 1, D=-2e-3), synth.random_state(3, m2)),
            synth.Sim(m1, _mat(m1, 3, sot=True, seed=4), synth.random_state(4, m1))]
    for prec in ("f64", "f32"):
        ctx = make_ctx(prec, sims)
        offs, _ = ctx.layout()
        dmdt, heff = ctx.rhs_host(np.concatenate([s.m0.ravel() for s in sims]))
        for i, s in enumerate(sims):
            n = 3 * s.mesh.ncells
            ref_k, ref_H = oracle_rhs(s, method="direct")
            gk, gH = dmdt[offs[i]:offs[i] + n], heff[offs[i]:offs[i] + n]
            if prec == "f64":
                assert max_rel(gH, ref_H) < TOL64 and max_rel(gk, ref_k) < TOL64, i
            else:
                assert rms_rel(gH, ref_H) < TOL32 and rms_rel(gk, ref_k) < TOL32, i


def test_rk45_attempts_with_spin_torques_match_oracle():
    """Zhang-Li and spin-orbit torques inside RK45: the GPU takes the oracle's steps."""
    m = synth.Mesh(16, 8, 2, 2e-9, 2e-9, 2e-9)
    mat = _mat(m, 2, cells=True, stt=True, sot=True, seed=7, alpha=0.2)
    sim = synth.Sim(m, mat, synth.random_state(11, m))
    ctx = make_ctx("f64", [sim])
    ctx.set_m(sim.m0.ravel())
    ctx.reset_time()
    ctx.rk45_setup(1e-6, t_end=1e-10)
    Ms = F.ms_array(m, mat)
    Nt = D.mesh_tensor(m)
    f = lambda y: F.rhs(m, mat, y, Ms, Nt, "direct")[0]
    st = I.Stepper(rtol=1e-6, t_end=1e-10)
    y = sim.m0.copy()
    for _ in range(10):
        y, _ = I.step(f, y, st)
    ctx.rk45_attempts(10)
    g = ctx.status(0)
    assert g["n_accepted"] == st.n_acc and g["n_rejected"] == st.n_rej
    assert abs(g["t"] - st.t) <= 1e-9 * st.t
    assert max_rel(ctx.get_m(0), y) < 1e-8


def test_spin_torque_switched_on_and_off_after_precompute():
    """mm_set_spin_torque after the graphs exist: the next attempts use the new torques
    (the graphs are rebuilt when the kernel variant changes)."""
    m = synth.Mesh(12, 10, 1, 2e-9, 2e-9, 2e-9)
    mat = _mat(m, 1)
    sim = synth.Sim(m, mat, synth.random_state(12, m))
    ctx = make_ctx("f64", [sim])
    Ms = F.ms_array(m, mat)
    Nt = D.mesh_tensor(m)
    for u, aJ in (((0.0, 0.0, 0.0), 0.0), ((80.0, 20.0, 0.0), 1e9), ((0.0, 0.0, 0.0), 0.0)):
        ctx.set_spin_torque(0, u, 0.05, aJ, 0.0, (0.0, 1.0, 0.0))
        mt = synth.Material(**{**mat.__dict__, "u_stt": u, "beta": 0.05, "aJ": aJ, "p": (0.0, 1.0, 0.0)})
        ctx.set_m(sim.m0.ravel())
        ctx.reset_time()
        ctx.rk45_setup(1e-6, t_end=5e-11)
        ctx.rk45_attempts(4)
        f = lambda y: F.rhs(m, mt, y, Ms, Nt, "direct")[0]
        st = I.Stepper(rtol=1e-6, t_end=5e-11)
        y = sim.m0.copy()
        for _ in range(4):
            y, _ = I.step(f, y, st)
        assert max_rel(ctx.get_m(0), y) < 1e-8, u


def test_rk4_cayley_with_bulk_dmi_and_refusal_with_torques():
    from oracle import cayley as CY
    from paper_2406_16064_gb300 import mm
    m = synth.Mesh(9, 6, 3, 2e-9, 2e-9, 1e-9)
    mat = _mat(m, 2, cells=True, seed=3)
    sim = synth.Sim(m, mat, synth.random_state(13, m))
    ctx = make_ctx("f64", [sim])
    ctx.set_m(sim.m0.ravel())
    ctx.rk4(2e-14, 5, True)
    Ms = F.ms_array(m, mat)
    Nt = D.mesh_tensor(m)
    ref = CY.run(m, mat, Ms, lambda y: F.h_eff(m, mat, y, Ms, Nt, "fft"), sim.m0.copy(), 2e-14, 5, True)
    assert np.abs(ctx.get_m(0) - ref.ravel()).max() < 1e-11
    ctx.set_spin_torque(0, (50.0, 0.0, 0.0), 0.1, 0.0, 0.0, (0.0, 0.0, 1.0))
    with pytest.raises(mm.MMError):
        ctx.rk4(2e-14, 1, True)
    ctx.rk4(2e-14, 1, False)                       # the projected scheme takes them


def test_wall_under_time_dependent_current_on_gpu():
    """The paper's head-to-head wall under u(t) = u0 exp(-b t) cos(w t) (Sec. "Domain-wall
    motion under currents"), FP64 on the GPU: fixed RK4 steps with projection, u set at
    each step's midpoint; centre and tilt follow dz/dt = (1 + alpha beta) u / (1 + alpha^2)
    and dphi/dt = (beta - alpha) u / ((1 + alpha^2) Delta) as in the oracle's test."""
    import math
    nx, dx = 200, 1e-9
    mesh = synth.Mesh(nx, 1, 1, dx, dx, dx)
    A, K, al, beta = 1.3e-11, 1e5, 0.1, 0.3
    Dw = math.sqrt(A / K)
    mat = synth.Material(Ms=8e5, A=A, Ku=K, u=(1, 0, 0), alpha=al, beta=beta, demag=0)
    u0, b, w = 100.0, 5e8, 2e9
    u = lambda t: u0 * math.exp(-b * t) * math.cos(w * t)
    Iu = lambda t: u0 * (math.exp(-b * t) * (w * math.sin(w * t) - b * math.cos(w * t)) + b) / (b * b + w * w)
    x = (np.arange(nx) + 0.5) * dx
    th = 2 * np.arctan(np.exp((x - 60e-9) / Dw))
    m0 = np.stack([np.cos(th), np.sin(th) * np.cos(0.4), np.sin(th) * np.sin(0.4)]).reshape(3, 1, 1, nx)
    ctx = make_ctx("f64", [synth.Sim(mesh, mat, m0)])
    ctx.set_m(m0.ravel())
    centre = lambda m: nx * dx - ((1 - m[0].ravel()) / 2).sum() * dx
    tilt = lambda m: math.atan2(m[2].sum(), m[1].sum())
    z0, p0 = centre(m0), tilt(m0)
    h, n = 8e-14, 5000
    dz, dp, ez, ep = [], [], [], []
    for i in range(n):
        ctx.set_spin_torque(0, (u((i + 0.5) * h), 0.0, 0.0), beta, 0.0, 0.0, (0.0, 0.0, 1.0))
        ctx.rk4(h, 1, False)
        if (i + 1) % 250 == 0:
            m = ctx.get_m(0).reshape(3, 1, 1, nx)
            t = (i + 1) * h
            dz.append(centre(m) - z0); ez.append((1 + al * beta) / (1 + al * al) * Iu(t))
            dp.append(tilt(m) - p0); ep.append((beta - al) / ((1 + al * al) * Dw) * Iu(t))
    dz, ez, dp, ep = map(np.array, (dz, ez, dp, ep))
    assert np.abs(dz - ez).max() < 0.01 * np.abs(ez).max()
    assert np.abs(dp - ep).max() < 0.02 * np.abs(ep).max()
