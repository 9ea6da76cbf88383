"""GPU: the scalar-potential demagnetising field (three forward transforms, one inverse;
Sec. "Magnetostatic energy") against the FP64 oracle's potential (oracle/potential.py):
exact face-charge potential of each cell at the cell centres, u one cell outside the
mesh, H = -grad u by central differences."""
import numpy as np
import pytest

import synth
from oracle import fields as F
from oracle import potential as P
from tests.gpu_util import make_ctx, max_rel, rms_rel

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (5, 3, 2), (16, 16, 1), (12, 10, 4), (8, 8, 8), (7, 1, 1), (1, 9, 3), (33, 17, 1)]


def _field(precision, sim):
    import torch
    ctx = make_ctx(precision, [sim])
    dt = torch.float32 if precision == "f32" else torch.float64
    m = torch.tensor(sim.m0.ravel(), dtype=dt, device="cuda")
    hd = torch.empty_like(m)
    ctx.demag_potential(m, hd, 0)
    torch.cuda.synchronize()
    return hd.double().cpu().numpy(), ctx


def _oracle(sim, method):
    Ms = F.ms_array(sim.mesh, sim.mat, sim.Ms_cells)
    return P.h_demag_potential(sim.mesh, Ms[None] * sim.m0, method)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_potential_field_matches_oracle(shape, precision):
    mesh = synth.Mesh(*shape, 2e-9, 2.5e-9, 1.5e-9)
    sim = synth.Sim(mesh, synth.Material(Ms=8e5), synth.random_state(11, mesh))
    H, _ = _field(precision, sim)
    ref = _oracle(sim, "direct" if mesh.ncells <= 512 else "fft")
    if precision == "f32":
        assert rms_rel(H, ref) < 1e-5
    else:
        assert max_rel(H, ref) < 1e-10


def test_potential_masked_cells_and_second_call():
    """Per-cell Ms (a disk) and a second call with another state: the kernel spectrum
    kept from the first call."""
    mesh = synth.Mesh(20, 14, 3, 2e-9, 2e-9, 3e-9)
    z, y, x = np.meshgrid(np.arange(3), np.arange(14), np.arange(20), indexing="ij")
    Ms_cells = np.where((x - 9.5) ** 2 + (y - 6.5) ** 2 <= 49, 6e5, 0.0)
    sim = synth.Sim(mesh, synth.Material(Ms=6e5), synth.random_state(3, mesh), Ms_cells)
    H, ctx = _field("f64", sim)
    assert max_rel(H, _oracle(sim, "fft")) < 1e-10
    import torch
    m2 = synth.random_state(4, mesh)
    mt = torch.tensor(m2.ravel(), dtype=torch.float64, device="cuda")
    hd = torch.empty_like(mt)
    ctx.demag_potential(mt, hd, 0)
    torch.cuda.synchronize()
    sim2 = synth.Sim(mesh, sim.mat, m2, Ms_cells)
    assert max_rel(hd.cpu().numpy(), _oracle(sim2, "fft")) < 1e-10


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_potential_uniform_cube_centre_and_film(precision):
    """Uniform M along z: the centre of a 16^3 cube is near -M/3 (second order in the
    cell size, as in the oracle's pin), and the whole field equals the oracle's."""
    mesh = synth.Mesh(16, 16, 16, 2e-9, 2e-9, 2e-9)
    sim = synth.Sim(mesh, synth.Material(Ms=1e6), synth.uniform_state(mesh, (0, 0, 1)))
    H, _ = _field(precision, sim)
    Hz = H.reshape(3, 16, 16, 16)[2]
    centre = Hz[7:9, 7:9, 7:9].mean() / 1e6
    assert abs(centre + 1.0 / 3.0) < 5e-3
    ref = _oracle(sim, "fft")
    assert (rms_rel(H, ref) < 1e-5) if precision == "f32" else (max_rel(H, ref) < 1e-10)


def test_potential_rejects_too_long_axes():
    from paper_2406_16064_gb300 import mm
    mesh = synth.Mesh(1100, 1, 1, 2e-9, 2e-9, 2e-9)
    with pytest.raises(mm.MMError) as e:
        _field("f32", synth.Sim(mesh, synth.Material(Ms=8e5), synth.random_state(1, mesh)))
    assert e.value.code == mm.MM_EINVAL


@pytest.mark.parametrize("seed", range(6))
def test_potential_random_meshes_match_oracle(seed):
    """Seeded random meshes of 1..24 cells per axis, random cell sizes, FP64 against
    the oracle's FFT potential (1e-10)."""
    rng = np.random.default_rng(300 + seed)
    shape = tuple(int(v) for v in rng.integers(1, 25, size=3))
    cells = tuple(float(v) for v in rng.uniform(1e-9, 4e-9, size=3))
    mesh = synth.Mesh(*shape, *cells)
    sim = synth.Sim(mesh, synth.Material(Ms=float(rng.uniform(4e5, 1.2e6))), synth.random_state(400 + seed, mesh))
    H, _ = _field("f64", sim)
    assert max_rel(H, _oracle(sim, "fft")) < 1e-10, shape
