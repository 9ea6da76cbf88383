"""FP32 relaxed states against the FP64 oracle's relaxed states (max deviation 1e-3).

The FP32 form runs the fields, stages and the NEB force in FP32 (norms, error norms and
energies at FP64 accuracy); a relaxed state is a property of the energy landscape, so the
FP32 run must end within 1e-3 of the FP64 oracle's end state wherever the minimum is
unique (Sec. "LLG equation" with the relaxation of Listing 2; the nudged elastic band of
Sec. "Miscellaneous").
"""
import numpy as np
import pytest

import synth
from oracle import demag as D
from oracle import fields as F
from oracle import integrate as I
from oracle import neb as NB
from tests.gpu_util import make_ctx

pytestmark = pytest.mark.gpu


def test_field_sweep_uneven_batch_f32_matches_f64_oracle():
    """Listing-2 style sweep on an uneven FP32 batch (films of 1 and 2 planes, DMI and
    anisotropy drawn per simulation): at each field every simulation relaxes below
    1e-2 rad/ns, and the end state of the sweep is within 1e-3 of the FP64 oracle's.
    The FP32 run uses rtol = 1e-6: near equilibrium the controller holds the error of
    the stiff exchange modes at about rtol, which leaves |dm/dt| near rtol times their
    frequency (~2e12 /s with 2 nm cells), above the 1e7 rad/s threshold at 1e-5."""
    w = synth.uneven_batch(seed=7, count=3, precision="f32", choices=[(8, 8, 1), (6, 4, 2), (12, 6, 1)])
    ctx = make_ctx("f32", w.sims)
    ctx.set_m(np.concatenate([s.m0.ravel() for s in w.sims]))
    ctx.reset_time()
    offs, _ = ctx.layout()
    sweep = (-100.0, -20.0, 0.0, 40.0, 100.0)
    ends = []
    for H in sweep:
        for i in range(len(w.sims)):
            ctx.set_field(i, (0.0, 0.0, H * synth.MT))
        ctx.relax(1e-6, max_dmdt=w.max_dmdt, max_steps=50000, sync_every=32)
        for i in range(len(w.sims)):
            assert ctx.status(i)["status"] == 2
        ends.append(ctx.get_m(-1))
    for i, s in enumerate(w.sims):
        Ms = F.ms_array(s.mesh, s.mat)
        Nt = D.mesh_tensor(s.mesh)
        m = s.m0.copy()
        n = 3 * s.mesh.ncells
        for k, H in enumerate(sweep):
            mat = synth.Material(**{**s.mat.__dict__, "H": (0.0, 0.0, H * synth.MT)})
            f = lambda y, mat=mat: F.rhs(s.mesh, mat, y, Ms, Nt, "direct")[0]
            m, st = I.run(f, m, 1e-6, max_dmdt=w.max_dmdt, max_steps=50000)
            assert st.last_maxdmdt < w.max_dmdt
            assert np.abs(ends[k][offs[i]:offs[i] + n] - m.ravel()).max() < 1e-3, (i, H)


def test_neb_two_particle_chain_f32_relaxes_to_the_f64_oracle_chain():
    """Two particles (one 2x1x1 image with demag, uniaxial anisotropy and a field along the
    axis), 13 images between both up and both down: the FP32 chain relaxed on the GPU ends
    within 1e-3 of the FP64 oracle's relaxed chain, with the same image energies to 1e-4
    of the anisotropy barrier Ku V, and on the sequential path (the middle image has one
    particle reversed)."""
    mesh = synth.Mesh(2, 1, 1, 3e-9, 3e-9, 3e-9)
    Ku, Ms0, h = 5e5, 8e5, 0.3
    H = h * 2 * Ku / (F.MU0 * Ms0)
    mat = synth.Material(Ms=Ms0, Ku=Ku, u=(0, 0, 1), H=(0, 0, H), alpha=0.5, precession=0, demag=1)
    n = 13
    s = np.linspace(0, 2 * np.pi, n)
    chain = np.zeros((n, 3, 1, 1, 2))
    for i, si in enumerate(s):
        t1, t2 = min(si, np.pi), max(si - np.pi, 0.0)
        chain[i, :, 0, 0, 0] = [np.sin(t1) * np.cos(0.3), np.sin(t1) * np.sin(0.3), np.cos(t1)]
        chain[i, :, 0, 0, 1] = [np.sin(t2) * np.cos(1.1), np.sin(t2) * np.sin(1.1), np.cos(t2)]
        if 0 < i < n - 1:
            chain[i] = synth.tilt(chain[i], 200 + i, 0.15)
    ctx = make_ctx("f32", [synth.Sim(mesh, mat, chain[i]) for i in range(n)])
    ctx.set_m(chain.ravel())
    ctx.neb_setup(0, n, 1e5)
    ctx.reset_time()
    E = ctx.neb_relax(1e-5, 1600)
    mg = ctx.get_m(-1).reshape(chain.shape)
    Ms = F.ms_array(mesh, mat)
    c, Eo, st = NB.relax(mesh, mat, Ms, chain, 1e5, 1e-6, 1600, D.mesh_tensor(mesh), "direct")
    V = 27e-27
    assert np.abs(mg - c).max() < 1e-3
    assert np.abs(E - Eo).max() < 1e-4 * Ku * V
    mid = mg[(n - 1) // 2]
    assert abs(mid[2, 0, 0, 0] + 1) < 1e-3 and abs(mid[2, 0, 0, 1] - 1) < 1e-3
