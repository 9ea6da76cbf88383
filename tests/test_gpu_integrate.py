"""GPU parity of the RK45 integrator, relaxation and NEB against the oracle / closed forms."""
import math

import numpy as np
import pytest

import synth
from oracle import demag as D
from oracle import fields as F
from oracle import integrate as I
from oracle import neb as NB
from tests.gpu_util import make_ctx, max_rel

pytestmark = pytest.mark.gpu


def _closed(alpha, gamma, Hz, t):
    gt = gamma / (1 + alpha ** 2)
    w = gt * Hz * t
    return np.array([math.cos(w) / math.cosh(alpha * w), math.sin(w) / math.cosh(alpha * w),
                     math.tanh(alpha * w)])


@pytest.mark.parametrize("precision,tol", [("f64", 2e-6), ("f32", 2e-4)])
def test_macrospin_closed_form_1ns(precision, tol):
    mesh = synth.Mesh(1, 1, 1, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, H=(0, 0, 1e5), alpha=0.5, gamma=2.21e5)
    m0 = np.array([1.0, 0, 0]).reshape(3, 1, 1, 1)
    ctx = make_ctx(precision, [synth.Sim(mesh, mat, m0)])
    ctx.set_m(m0.ravel())
    ctx.reset_time()
    ctx.relax(1e-6 if precision == "f64" else 1e-5, t_end=1e-9, max_steps=100000, sync_every=8)
    st = ctx.status(0)
    assert st["status"] == 1 and abs(st["t"] - 1e-9) < 1e-20
    m = ctx.get_m(0)
    assert np.abs(m - _closed(0.5, 2.21e5, 1e5, st["t"])).max() < tol


def test_film_relax_32_trajectory_matches_oracle():
    """32x32x1 film, FP64: the GPU and the oracle take the same accepted steps."""
    w = synth.film_relax_32()
    sim = w.sims[0]
    ctx = make_ctx("f64", [sim])
    ctx.set_m(sim.m0.ravel())
    ctx.reset_time()
    ctx.rk45_setup(w.rtol, t_end=w.t_end)
    Ms = F.ms_array(sim.mesh, sim.mat)
    Nt = D.mesh_tensor(sim.mesh)
    f = lambda y: F.rhs(sim.mesh, sim.mat, y, Ms, Nt, "direct")[0]
    st = I.Stepper(rtol=w.rtol, t_end=w.t_end)
    m = sim.m0.copy()
    for _ in range(12):
        m, _ = I.step(f, m, st)
    ctx.rk45_attempts(12)
    g = ctx.status(0)
    assert g["n_accepted"] == st.n_acc and g["n_rejected"] == st.n_rej
    assert abs(g["t"] - st.t) <= 1e-9 * st.t
    assert max_rel(ctx.get_m(0), m) < 1e-8


def test_film_relax_32_full_run_f64():
    """The whole 1 ns run: final state and time vs the oracle's."""
    w = synth.film_relax_32()
    sim = w.sims[0]
    ctx = make_ctx("f64", [sim])
    ctx.set_m(sim.m0.ravel())
    ctx.reset_time()
    ctx.relax(w.rtol, t_end=w.t_end, max_steps=200000, sync_every=64)
    g = ctx.status(0)
    assert g["status"] == 1
    Ms = F.ms_array(sim.mesh, sim.mat)
    Nt = D.mesh_tensor(sim.mesh)
    f = lambda y: F.rhs(sim.mesh, sim.mat, y, Ms, Nt, "direct")[0]
    m, st = I.run(f, sim.m0.copy(), w.rtol, t_end=w.t_end)
    mg = ctx.get_m(0).reshape(m.shape)
    Eg = F.energies(sim.mesh, sim.mat, mg, Ms, Nt, "direct")["total"]
    Eo = F.energies(sim.mesh, sim.mat, m, Ms, Nt, "direct")["total"]
    dev = np.abs(mg - m).max()
    # several relaxed states can be correct; equal energy marks an equivalent minimum
    assert dev < 1e-3 or abs(Eg - Eo) < 1e-6 * abs(Eo), (dev, Eg, Eo)


def test_norm_and_energy_decay_on_gpu():
    mesh = synth.Mesh(24, 16, 2, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, Ku=2e5, alpha=0.5, H=(1e4, 0, 0))
    sim = synth.Sim(mesh, mat, synth.random_state(2, mesh))
    ctx = make_ctx("f64", [sim])
    ctx.set_m(sim.m0.ravel())
    ctx.reset_time()
    ctx.rk45_setup(1e-6)
    E0 = ctx.energy(0)["total"]
    for _ in range(10):
        ctx.rk45_step()
        m = ctx.get_m(0).reshape(3, -1)
        assert np.abs(np.sqrt((m ** 2).sum(0)) - 1).max() < 1e-14
        E1 = ctx.energy(0)["total"]
        assert E1 <= E0 + 1e-6 * abs(E0)
        E0 = E1


def test_norm_and_energy_decay_on_gpu_f32():
    """FP32 states: the projection (float-float norm) leaves every |m| within two
    FP32 ulps of 1 (one rounding per component); the energy does not grow beyond
    the controller's tolerance."""
    mesh = synth.Mesh(24, 16, 2, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, Ku=2e5, alpha=0.5, H=(1e4, 0, 0))
    sim = synth.Sim(mesh, mat, synth.random_state(2, mesh))
    ctx = make_ctx("f32", [sim])
    ctx.set_m(sim.m0.ravel())
    ctx.reset_time()
    ctx.rk45_setup(1e-5)
    E0 = ctx.energy(0)["total"]
    for _ in range(10):
        ctx.rk45_step()
        m = ctx.get_m(0).reshape(3, -1)
        assert np.abs(np.sqrt((m ** 2).sum(0)) - 1).max() < 2 * 2.0 ** -23
        E1 = ctx.energy(0)["total"]
        assert E1 <= E0 + 1e-5 * abs(E0)
        E0 = E1


def test_stoner_wohlfarth_switching_on_gpu():
    mesh = synth.Mesh(4, 4, 4, 2e-9, 2e-9, 2e-9)
    Ms0, Ku = 1e6, 5e4
    mat = synth.Material(Ms=Ms0, A=1e-11, Ku=Ku, u=(1, 1, 0), alpha=0.5, precession=0, demag=0)
    ctx = make_ctx("f64", [synth.Sim(mesh, mat, synth.uniform_state(mesh))])
    m = synth.tilt(synth.uniform_state(mesh, (-1, 0, 0)), 9, 1e-3)
    ctx.set_m(m.ravel())
    mT = 1e-3 / F.MU0
    out = {}
    for i in (-20, 9, 11):
        ctx.set_field(0, (i * 5 * mT, 0.0, 0.0))
        ctx.relax(1e-8, max_dmdt=1e6, max_steps=20000, sync_every=16)
        assert ctx.status(0)["status"] == 2
        out[i] = ctx.get_m(0).reshape(3, -1)[0].mean()
    assert out[9] < 0.0 < out[11]


def test_uneven_batch_relax_matches_per_sim_oracle():
    """Several simulations of different sizes step together; each matches its own oracle run."""
    specs = [(8, 8, 1), (6, 4, 2), (12, 6, 1)]
    sims = []
    for i, (nx, ny, nz) in enumerate(specs):
        mesh = synth.Mesh(nx, ny, nz, 2e-9, 2e-9, 2e-9)
        mat = synth.Material(Ms=6e5 + 1e5 * i, A=1e-11, D=1e-3 * i, dmi=1, Ku=1e5, alpha=0.3 + 0.1 * i,
                             H=(0, 0, 2e4))
        sims.append(synth.Sim(mesh, mat, synth.random_state(20 + i, mesh)))
    ctx = make_ctx("f64", sims)
    ctx.set_m(np.concatenate([s.m0.ravel() for s in sims]))
    ctx.reset_time()
    ctx.rk45_setup(1e-6, t_end=2e-11)
    ctx.rk45_attempts(8)
    for i, s in enumerate(sims):
        Ms = F.ms_array(s.mesh, s.mat)
        Nt = D.mesh_tensor(s.mesh)
        f = lambda y: F.rhs(s.mesh, s.mat, y, Ms, Nt, "direct")[0]
        st = I.Stepper(rtol=1e-6, t_end=2e-11)
        m = s.m0.copy()
        for _ in range(8):
            if I.done_time(st):
                break
            m, _ = I.step(f, m, st)
        g = ctx.status(i)
        assert g["n_accepted"] == st.n_acc, i
        assert max_rel(ctx.get_m(i), m) < 1e-8


def test_field_sweep_uneven_batch_matches_oracle():
    """Listing-2 style sweep on an uneven batch: every simulation relaxes at each field
    (max |dm/dt| < 1e-2 rad/ns) and ends where the oracle's own sweep ends."""
    w = synth.uneven_batch(seed=7, count=3, precision="f64", choices=[(8, 8, 1), (6, 4, 2), (12, 6, 1)])
    ctx = make_ctx("f64", w.sims)
    ctx.set_m(np.concatenate([s.m0.ravel() for s in w.sims]))
    ctx.reset_time()
    offs, _ = ctx.layout()
    sweep = (-100.0, 0.0, 100.0)
    for H in sweep:
        for i in range(len(w.sims)):
            ctx.set_field(i, (0.0, 0.0, H * synth.MT))
        ctx.relax(1e-6, max_dmdt=w.max_dmdt, max_steps=50000, sync_every=32)
        for i in range(len(w.sims)):
            assert ctx.status(i)["status"] == 2
    mg = ctx.get_m(-1)
    for i, s in enumerate(w.sims):
        Ms = F.ms_array(s.mesh, s.mat)
        Nt = D.mesh_tensor(s.mesh)
        m = s.m0.copy()
        for H in sweep:
            mat = synth.Material(**{**s.mat.__dict__, "H": (0.0, 0.0, H * synth.MT)})
            f = lambda y, mat=mat: F.rhs(s.mesh, mat, y, Ms, Nt, "direct")[0]
            m, st = I.run(f, m, 1e-6, max_dmdt=w.max_dmdt, max_steps=50000)
            assert st.last_maxdmdt < w.max_dmdt
        n = 3 * s.mesh.ncells
        assert np.abs(mg[offs[i]:offs[i] + n] - m.ravel()).max() < 1e-3, i


def test_neb_single_cell_matches_closed_form_and_oracle():
    mesh = synth.Mesh(1, 1, 1, 3e-9, 3e-9, 3e-9)
    Ku, Ms0 = 5e5, 8e5
    H = 0.3 * 2 * Ku / (F.MU0 * Ms0)
    mat = synth.Material(Ms=Ms0, Ku=Ku, u=(0, 0, 1), H=(0, 0, H), alpha=0.5, precession=0, demag=0)
    n = 11
    chain = synth.geodesic_chain(synth.uniform_state(mesh, (0, 0, 1)), synth.uniform_state(mesh, (0, 0, -1)), n)
    for i in range(1, n - 1):
        chain[i] = synth.tilt(chain[i], 100 + i, 0.2)
    ctx = make_ctx("f64", [synth.Sim(mesh, mat, chain[i]) for i in range(n)])
    ctx.set_m(chain.ravel())
    ctx.neb_setup(0, n, 1e5)
    ctx.reset_time()
    E = ctx.neb_relax(1e-6, 600)
    mg = ctx.get_m(-1).reshape(chain.shape)
    c, Eo, st = NB.relax(mesh, mat, F.ms_array(mesh, mat), chain, 1e5, 1e-6, 600)
    V = 27e-27
    th = np.linspace(0, np.pi, n)
    expect = -Ku * V * np.cos(th) ** 2 - F.MU0 * Ms0 * V * H * np.cos(th)
    assert np.abs(E - expect).max() < 1e-3 * Ku * V
    assert np.array_equal(mg[0], chain[0]) and np.array_equal(mg[-1], chain[-1])
    assert np.abs(mg - c).max() < 1e-6
    assert np.abs(E - Eo).max() < 1e-9 * Ku * V


def test_neb_small_film_chain_matches_oracle():
    mesh = synth.Mesh(12, 12, 1, 1e-9, 1e-9, 0.5e-9)
    mat = synth.Material(Ms=5.8e5, A=1.5e-11, D=3e-3, dmi=1, Ku=8e5, alpha=0.5, precession=0)
    w = synth.neb_chain(n_images=6, n=12, radius=3e-9)
    chain = np.stack([s.m0 for s in w.sims])
    ctx = make_ctx("f64", [synth.Sim(mesh, mat, chain[i]) for i in range(6)])
    ctx.set_m(chain.ravel())
    ctx.neb_setup(0, 6, 1e5)
    ctx.reset_time()
    E = ctx.neb_relax(1e-5, 20)
    Ms = F.ms_array(mesh, mat)
    Nt = D.mesh_tensor(mesh)
    c, Eo, st = NB.relax(mesh, mat, Ms, chain, 1e5, 1e-5, 20, Nt, "direct")
    mg = ctx.get_m(-1).reshape(chain.shape)
    assert np.abs(mg - c).max() < 1e-6
    assert np.abs(E - Eo).max() < 1e-8 * np.abs(Eo).max()


def test_neb_small_film_chain_f32_matches_oracle():
    """FP32 chain (per-cell tangent, distance and force in FP32, sums in FP64)
    against the FP64 oracle over the first steps, before the two step-size
    sequences part: m within 1e-5, energies within 1e-5 relative (the FP32
    field bar)."""
    mesh = synth.Mesh(12, 12, 1, 1e-9, 1e-9, 0.5e-9)
    mat = synth.Material(Ms=5.8e5, A=1.5e-11, D=3e-3, dmi=1, Ku=8e5, alpha=0.5, precession=0)
    w = synth.neb_chain(n_images=6, n=12, radius=3e-9)
    chain = np.stack([s.m0 for s in w.sims])
    ctx = make_ctx("f32", [synth.Sim(mesh, mat, chain[i]) for i in range(6)])
    ctx.set_m(chain.ravel())
    ctx.neb_setup(0, 6, 1e5)
    ctx.reset_time()
    E = ctx.neb_relax(1e-5, 2)
    Ms = F.ms_array(mesh, mat)
    Nt = D.mesh_tensor(mesh)
    c, Eo, st = NB.relax(mesh, mat, Ms, chain, 1e5, 1e-5, 2, Nt, "direct")
    mg = ctx.get_m(-1).reshape(chain.shape)
    assert np.abs(mg - c).max() < 1e-5
    assert np.abs(E - Eo).max() < 1e-5 * np.abs(Eo).max()


def test_bounded_wait_times_out_cleanly():
    from paper_2406_16064_gb300 import mm
    mesh = synth.Mesh(2, 2, 1, 1e-9, 1e-9, 1e-9)
    ctx = make_ctx("f64", [synth.Sim(mesh, synth.Material(Ms=1e5), synth.uniform_state(mesh))])
    assert ctx.bounded_wait(100000) == mm.MM_ETIMEOUT
    # the context is still usable afterwards
    d, h = ctx.rhs_host(synth.uniform_state(mesh).ravel())
    assert np.isfinite(d).all()


def test_nan_input_reports_enan():
    from paper_2406_16064_gb300 import mm
    mesh = synth.Mesh(4, 4, 1, 1e-9, 1e-9, 1e-9)
    ctx = make_ctx("f64", [synth.Sim(mesh, synth.Material(Ms=5e5, A=1e-11), synth.uniform_state(mesh))])
    m = synth.random_state(3, mesh)
    m[0, 0, 1, 1] = np.nan
    ctx.set_m(m.ravel())
    ctx.reset_time()
    with pytest.raises(mm.MMError) as e:
        ctx.relax(1e-6, t_end=1e-12, max_steps=10, sync_every=1)
    assert e.value.code == mm.MM_ENAN


def test_profile_attempts_counts_every_kernel_kind():
    """Per-kind event timing: 7 x-forward and 7 x-inverse launches per attempt,
    one projection; in a NEB context also 7 NEB force launches."""
    mesh = synth.Mesh(12, 12, 1, 1e-9, 1e-9, 0.5e-9)
    mat = synth.Material(Ms=5.8e5, A=1.5e-11, D=3e-3, dmi=1, Ku=8e5, alpha=0.5, precession=0)
    w = synth.neb_chain(n_images=4, n=12, radius=3e-9)
    chain = np.stack([s.m0 for s in w.sims])
    for neb in (False, True):
        ctx = make_ctx("f32", [synth.Sim(mesh, mat, chain[i]) for i in range(4)])
        ctx.set_m(chain.ravel())
        if neb:
            ctx.neb_setup(0, 4, 1e5)
        ctx.reset_time()
        ctx.rk45_setup(1e-5, t_end=0.0, max_dmdt=0.0)
        prof = ctx.profile_attempts(2)
        assert prof["x_forward"][1] == 14 and prof["x_inverse_epilogue"][1] == 14
        assert prof["y_fused"][1] == 14 and prof["project"][1] == 2
        assert prof["neb"][1] == (14 if neb else 0)
        assert all(t > 0 for t, c in prof.values() if c)
