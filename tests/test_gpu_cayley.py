"""GPU parity of the fixed-step RK4 integrators (mm_rk4): classical RK4 on the
Cayley-transform variable and RK4 on dm/dt with projection, against
oracle.cayley on the same seeded inputs, and the paper's macrospin comparison
(Sec. "Cayley transform") on the GPU."""
import math

import numpy as np
import pytest

import synth
from oracle import cayley as CY
from oracle import demag as D
from oracle import fields as F
from tests.gpu_util import make_ctx

pytestmark = pytest.mark.gpu


def _film(nx, ny, nz, seed, precession=1):
    mesh = synth.Mesh(nx, ny, nz, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, D=1e-3, dmi=1, Ku=5e5, u=(0, 0, 1), H=(5e4, 0, 2e4), alpha=0.3,
                         precession=precession, demag=1)
    return synth.Sim(mesh, mat, synth.random_state(seed, mesh))


def _oracle(sim, h, n, cayley, m0=None):
    Ms = F.ms_array(sim.mesh, sim.mat, sim.Ms_cells)
    Nt = D.mesh_tensor(sim.mesh)
    field = lambda y: F.h_eff(sim.mesh, sim.mat, y, Ms, Nt, "fft")
    m0 = sim.m0 if m0 is None else m0
    return CY.run(sim.mesh, sim.mat, Ms, field, m0.copy(), h, n, cayley)


# (12, 10, 1) runs the film path, (9, 7, 3) the cluster y/z path, (6, 5, 12)
# the column passes; precession off covers the damping-only f
@pytest.mark.parametrize("dims,precession", [((12, 10, 1), 1), ((9, 7, 3), 1), ((6, 5, 12), 1),
                                             ((12, 10, 1), 0)])
@pytest.mark.parametrize("cayley", [True, False])
def test_steps_match_the_oracle_f64(dims, precession, cayley):
    sim = _film(*dims, seed=11, precession=precession)
    ctx = make_ctx("f64", [sim])
    ctx.set_m(sim.m0.ravel())
    h, n = 2e-14, 6
    ctx.rk4(h, n, cayley)
    ref = _oracle(sim, h, n, cayley)
    m = ctx.get_m(0)
    assert np.abs(m - ref.ravel()).max() < 1e-11
    assert abs(ctx.status(0)["t"] - n * h) <= 1e-12 * n * h
    # one more call with another h captures again and continues from the new m
    ctx.rk4(h / 2, 2, cayley)
    ref = _oracle(sim, h / 2, 2, cayley, ref)
    assert np.abs(ctx.get_m(0) - ref.ravel()).max() < 1e-11


@pytest.mark.parametrize("cayley", [True, False])
def test_steps_match_the_oracle_f32(cayley):
    sim = _film(16, 12, 1, seed=5)
    ctx = make_ctx("f32", [sim])
    ctx.set_m(sim.m0.ravel())
    ctx.rk4(2e-14, 6, cayley)
    ref = _oracle(sim, 2e-14, 6, cayley)
    m = ctx.get_m(0)
    assert np.abs(m - ref.ravel()).max() < 2e-5
    nrm = np.sqrt((m.reshape(3, -1).astype(np.float64) ** 2).sum(0))
    assert np.abs(nrm - 1).max() < 5e-6        # a few FP32 roundings a step


def test_macrospin_cayley_beats_projection_on_gpu():
    """The macrospin of the paper's comparison (alpha = 0.05, H = 1e5 A/m along z,
    t = 1 ns): both GPU schemes equal the oracle's, and the Cayley error against
    the closed form is far below the projected scheme's."""
    mesh = synth.Mesh(1, 1, 1, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, H=(0.0, 0.0, 1e5), alpha=0.05, gamma=2.21e5, demag=0)
    sim = synth.Sim(mesh, mat, synth.uniform_state(mesh, (1.0, 0.0, 0.0)))
    gt = 2.21e5 / (1 + 0.05 ** 2)
    w = gt * 1e5 * 1e-9
    exact = np.array([math.cos(w) / math.cosh(0.05 * w), math.sin(w) / math.cosh(0.05 * w), math.tanh(0.05 * w)])
    err = {}
    for cay in (True, False):
        ctx = make_ctx("f64", [sim])
        ctx.set_m(sim.m0.ravel())
        ctx.rk4(1e-12, 1000, cay)
        m = ctx.get_m(0)
        ref = _oracle(sim, 1e-12, 1000, cay)
        assert np.abs(m - ref.ravel()).max() < 1e-12
        err[cay] = np.abs(m - exact).max()
    assert err[True] < err[False] / 5, err


def test_masked_cells_stay_fixed_on_gpu():
    mesh = synth.Mesh(6, 5, 1, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, Ku=2e5, H=(3e4, 0, 1e4), alpha=0.2, demag=1)
    Ms_cells = np.full(mesh.shape, 8e5)
    Ms_cells[0, 2, 3] = 0.0
    sim = synth.Sim(mesh, mat, synth.random_state(4, mesh), Ms_cells)
    for cay in (True, False):
        ctx = make_ctx("f64", [sim])
        ctx.set_m(sim.m0.ravel())
        ctx.rk4(5e-14, 8, cay)
        m = ctx.get_m(0).reshape(3, *mesh.shape)
        assert np.array_equal(m[:, 0, 2, 3], sim.m0[:, 0, 2, 3])
        assert np.abs(m - _oracle(sim, 5e-14, 8, cay)).max() < 1e-11


def test_uneven_batch_each_simulation_matches_its_oracle():
    sims = [_film(12, 10, 1, seed=3), _film(9, 7, 3, seed=4), _film(16, 6, 1, seed=5, precession=0)]
    ctx = make_ctx("f64", sims)
    ctx.set_m(np.concatenate([s.m0.ravel() for s in sims]))
    ctx.rk4(2e-14, 4, True)
    for i, s in enumerate(sims):
        assert np.abs(ctx.get_m(i) - _oracle(s, 2e-14, 4, True).ravel()).max() < 1e-11, i


def test_bad_arguments_are_rejected():
    from paper_2406_16064_gb300 import mm
    sim = _film(8, 8, 1, seed=1)
    ctx = make_ctx("f64", [sim])
    ctx.set_m(sim.m0.ravel())
    for h, n, c in ((0.0, 1, 1), (-1e-13, 1, 1), (float("inf"), 1, 0), (float("nan"), 1, 0), (1e-13, -1, 0),
                    (1e-13, 1, 2)):
        with pytest.raises(mm.MMError):
            ctx._check(ctx.L.mm_rk4(ctx.h, h, n, c))
    ctx.rk4(1e-13, 0, True)                       # zero steps: nothing moves
    assert np.array_equal(ctx.get_m(0), sim.m0.ravel())
