"""GPU parity of the right-hand side, tensor and energies against the FP64 oracle.

Tolerances: FP64 fields 1e-10 relative (max over cells of |dH| / max |H|);
FP32 fields 1e-5 relative RMS (|dH|_2 / |H|_2).
"""
import numpy as np
import pytest

import synth
from oracle import demag as D
from oracle import fields as F
from oracle import newell as nw
from tests.gpu_util import make_ctx, max_rel, oracle_rhs, rms_rel

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


def _mat(**kw):
    base = dict(Ms=8e5, A=1.3e-11, D=3e-3, dmi=1, Ku=4e5, u=(0.2, 0.3, 0.9), Kc=1e4,
                H=(1e4, -2e4, 3e4), alpha=0.3)
    base.update(kw)
    return synth.Material(**base)


MESHES = [
    (1, 1, 1, 2e-9, 2e-9, 2e-9),
    (2, 1, 1, 2e-9, 3e-9, 1e-9),
    (3, 2, 1, 2e-9, 2e-9, 1e-9),
    (7, 5, 3, 2e-9, 2.5e-9, 1.5e-9),
    (1, 6, 4, 2e-9, 2e-9, 2e-9),
    (5, 1, 6, 1e-9, 2e-9, 3e-9),
    (32, 32, 1, 2.5e-9, 2.5e-9, 3e-9),
    (33, 17, 2, 2e-9, 2e-9, 1e-9),
    (9, 6, 5, 2e-9, 2e-9, 1e-9),       # cluster of 5 planes, padded z length 16
    (6, 5, 8, 2e-9, 2e-9, 1e-9),       # cluster of 8 planes
    (5, 4, 9, 2e-9, 2e-9, 1e-9),       # more planes than a cluster: separate y and z passes
    (70, 3, 1, 1e-9, 2e-9, 1e-9),      # several kx blocks with a ragged last block
]


@pytest.mark.parametrize("mesh", MESHES)
def test_newell_tensor_matches_oracle(mesh):
    m = synth.Mesh(*mesh)
    ctx = make_ctx("f64", [synth.Sim(m, _mat(), synth.random_state(1, m))])
    got = ctx.newell_tensor(0, m)
    ref = nw.mesh_tensor(*mesh)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("mesh", MESHES)
def test_rhs_f64_matches_oracle(mesh):
    m = synth.Mesh(*mesh)
    sim = synth.Sim(m, _mat(), synth.random_state(3, m))
    ctx = make_ctx("f64", [sim])
    dmdt, heff = ctx.rhs_host(sim.m0.ravel())
    ref_k, ref_H = oracle_rhs(sim, method="direct")
    assert max_rel(heff, ref_H) < TOL64
    assert max_rel(dmdt, ref_k) < TOL64


@pytest.mark.parametrize("mesh", MESHES[3:])
def test_rhs_f32_matches_oracle(mesh):
    m = synth.Mesh(*mesh)
    sim = synth.Sim(m, _mat(), synth.random_state(4, m))
    ctx = make_ctx("f32", [sim])
    dmdt, heff = ctx.rhs_host(sim.m0.ravel())
    ref_k, ref_H = oracle_rhs(sim, method="direct")
    assert rms_rel(heff, ref_H) < TOL32
    assert rms_rel(dmdt, ref_k) < TOL32


# Long rows: x tiles of one row whose shared memory limits an SM to 1-3 CTAs,
# so the x passes launch wider CTAs (512 / 1024 threads FP32, 512 FP64).
LONG_ROWS = [
    ("f32", (2048, 3, 1, 2e-9, 2e-9, 2e-9)),   # 2 CTAs per SM -> 512 threads
    ("f32", (4096, 2, 1, 2e-9, 2e-9, 2e-9)),   # 1 CTA per SM -> 1024 threads
    ("f32", (1500, 3, 2, 1e-9, 2e-9, 1e-9)),   # ragged row, two planes (cluster path)
    ("f64", (2048, 2, 1, 2e-9, 2e-9, 2e-9)),   # 1 CTA per SM -> 512 threads
    ("f64", (700, 3, 3, 2e-9, 1e-9, 1e-9)),    # 2 CTAs per SM -> 256 threads
]


@pytest.mark.parametrize("precision,mesh", LONG_ROWS)
def test_rhs_long_rows_wide_ctas(precision, mesh):
    m = synth.Mesh(*mesh)
    sim = synth.Sim(m, _mat(), synth.random_state(6, m))
    ctx = make_ctx(precision, [sim])
    dmdt, heff = ctx.rhs_host(sim.m0.ravel())
    ref_k, ref_H = oracle_rhs(sim, method="fft")
    if precision == "f64":
        assert max_rel(heff, ref_H) < TOL64
        assert max_rel(dmdt, ref_k) < TOL64
    else:
        assert rms_rel(heff, ref_H) < TOL32
        assert rms_rel(dmdt, ref_k) < TOL32


def test_rhs_masked_cells_and_terms_off():
    m = synth.Mesh(9, 7, 3, 2e-9, 2e-9, 2e-9)
    Ms = np.full(m.shape, 8e5)
    Ms[1, 3, 4] = 0.0
    Ms[:, 0, :3] = 0.0
    Ms[2, 6, 8] = 4e5
    sims = [synth.Sim(m, _mat(), synth.random_state(5, m), Ms),
            synth.Sim(m, _mat(demag=0, precession=0), synth.random_state(6, m)),
            synth.Sim(m, _mat(A=0.0, D=0.0, dmi=0, Ku=0.0, Kc=0.0), synth.random_state(7, m))]
    for sim in sims:
        ctx = make_ctx("f64", [sim])
        dmdt, heff = ctx.rhs_host(sim.m0.ravel())
        ref_k, ref_H = oracle_rhs(sim, method="direct")
        assert max_rel(heff, ref_H) < TOL64
        assert max_rel(dmdt, ref_k) < TOL64


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_uneven_batch_matches_oracle(precision):
    specs = [(16, 16, 1), (8, 4, 2), (24, 8, 1), (5, 7, 3), (16, 16, 1)]
    sims = []
    for i, (nx, ny, nz) in enumerate(specs):
        mesh = synth.Mesh(nx, ny, nz, 2e-9, 2e-9, 2e-9)
        mat = _mat(Ms=5e5 + 1e5 * i, A=1e-11 * (1 + i), D=1e-3 * i, Ku=1e5 * i, H=(0, 0, 1e4 * i))
        sims.append(synth.Sim(mesh, mat, synth.random_state(10 + i, mesh)))
    ctx = make_ctx(precision, sims)
    offs, total = ctx.layout()
    mall = np.concatenate([s.m0.ravel() for s in sims])
    dmdt, heff = ctx.rhs_host(mall)
    for i, s in enumerate(sims):
        n = 3 * s.mesh.ncells
        ref_k, ref_H = oracle_rhs(s, method="direct")
        gk, gH = dmdt[offs[i]:offs[i] + n], heff[offs[i]:offs[i] + n]
        if precision == "f64":
            assert max_rel(gH, ref_H) < TOL64 and max_rel(gk, ref_k) < TOL64
        else:
            assert rms_rel(gH, ref_H) < TOL32 and rms_rel(gk, ref_k) < TOL32
    # single-simulation evaluation of one member agrees with the batch
    d1, h1 = ctx.rhs_host(sims[3].m0.ravel(), sim=3)
    n = 3 * sims[3].mesh.ncells
    assert np.array_equal(d1, dmdt[offs[3]:offs[3] + n])


def test_rhs_device_buffers_torch():
    torch = pytest.importorskip("torch")
    m = synth.Mesh(20, 12, 2, 2e-9, 2e-9, 2e-9)
    sim = synth.Sim(m, _mat(), synth.random_state(8, m))
    ctx = make_ctx("f32", [sim])
    mt = torch.tensor(sim.m0.ravel(), dtype=torch.float32, device="cuda")
    kt = torch.empty_like(mt)
    ht = torch.empty_like(mt)
    ctx.rhs_device(mt, kt, ht)
    torch.cuda.synchronize()
    ref_k, ref_H = oracle_rhs(sim, method="direct")
    assert rms_rel(ht.cpu().numpy(), ref_H) < TOL32
    assert rms_rel(kt.cpu().numpy(), ref_k) < TOL32


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_energies_match_oracle(precision):
    m = synth.Mesh(12, 10, 3, 2e-9, 2e-9, 1e-9)
    sim = synth.Sim(m, _mat(), synth.random_state(9, m))
    ctx = make_ctx(precision, [sim])
    ctx.set_m(sim.m0.ravel())
    E = ctx.energy(0)
    ref = F.energies(m, sim.mat, sim.m0, F.ms_array(m, sim.mat), method="direct")
    scale = max(abs(v) for k, v in ref.items() if k != "total")
    tol = 1e-10 if precision == "f64" else 1e-5
    for k in ("exchange", "dmi", "uniaxial", "cubic", "zeeman", "demag", "total"):
        assert abs(E[k] - ref[k]) <= tol * scale, (k, E[k], ref[k])


def test_film_relax_32_rhs_at_full_size_f64():
    w = synth.film_relax_32()
    sim = w.sims[0]
    ctx = make_ctx("f64", [sim])
    dmdt, heff = ctx.rhs_host(sim.m0.ravel())
    ref_k, ref_H = oracle_rhs(sim, method="direct")
    assert max_rel(heff, ref_H) < TOL64 and max_rel(dmdt, ref_k) < TOL64


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_skyrmion_film_full_size(precision):
    """512x512x4 film (the benchmark workload): every cell vs the oracle's FFT convolution."""
    w = synth.skyrmion_film(precision=precision)
    sim = w.sims[0]
    ctx = make_ctx(precision, [sim])
    dmdt, heff = ctx.rhs_host(sim.m0.ravel())
    Ntab = D.mesh_tensor(sim.mesh)
    ref_k, ref_H = oracle_rhs(sim, method="fft", Ntab=Ntab)
    if precision == "f64":
        assert max_rel(heff, ref_H) < TOL64 and max_rel(dmdt, ref_k) < TOL64
    else:
        assert rms_rel(heff, ref_H) < TOL32 and rms_rel(dmdt, ref_k) < TOL32


def test_bulk_cube_full_size_properties_f32():
    """256^3 cube: uniform state mean demag field equals -N_box M (prism sum rule), and the
    local terms at sampled cells equal the oracle's, for the benchmark's launch shape."""
    n = 256
    mesh = synth.Mesh(n, n, n, 3e-9, 3e-9, 3e-9)
    mat = synth.Material(Ms=1.7e6, A=2.1e-11, Kc=-2.4e4, alpha=0.02)
    ctx = make_ctx("f32", [synth.Sim(mesh, mat, synth.uniform_state(mesh))])
    d = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    mu = synth.uniform_state(mesh, d)
    _, heff = ctx.rhs_host(mu.ravel())
    H = heff.reshape(3, -1)
    box = nw.as_matrix(nw.tensor_exact(0.0, 0.0, 0.0, n * 3e-9, n * 3e-9, n * 3e-9))
    Hc = -4.0 * mat.Kc / (F.MU0 * mat.Ms) * d ** 3        # cubic term, uniform
    expect = -box @ (d * mat.Ms) + Hc
    np.testing.assert_allclose(H.mean(axis=1), expect, rtol=0, atol=2e-5 * mat.Ms)
    # Voronoi state: local (non-demag) terms at sampled cells
    w = synth.bulk_cube()
    m0 = w.sims[0].m0
    mat_nod = synth.Material(**{**w.sims[0].mat.__dict__, "demag": 0})
    ctx2 = make_ctx("f32", [synth.Sim(mesh, mat_nod, m0)])
    _, h2 = ctx2.rhs_host(m0.ravel())
    h2 = h2.reshape((3,) + mesh.shape)
    rng = np.random.default_rng(0)
    for _ in range(64):
        z, y, x = rng.integers(0, n, 3)
        z0, y0, x0 = max(z - 1, 0), max(y - 1, 0), max(x - 1, 0)
        sub = m0[:, z0:z + 2, y0:y + 2, x0:x + 2]
        # oracle on the 3x3x3 neighbourhood; interior cell (or mesh edge) of the block
        sm = synth.Mesh(sub.shape[3], sub.shape[2], sub.shape[1], 3e-9, 3e-9, 3e-9)
        ref = F.h_eff(sm, mat_nod, sub, F.ms_array(sm, mat_nod))[:, z - z0, y - y0, x - x0]
        # the block's own boundary hides neighbours only where the mesh has none either
        np.testing.assert_allclose(h2[:, z, y, x], ref, rtol=0, atol=1e-5 * np.abs(ref).max() + 1e-3)


def test_newell_far_field_against_an_independent_quadrature():
    """The GPU's FP64 tensor at far offsets (its own Gauss-Legendre bands) against the
    cell-pair average integrated by Clenshaw-Curtis on each half-tent (1e-11)."""
    from tests.test_oracle_newell import _far_reference
    mesh = synth.Mesh(70, 9, 3, 2e-9, 2.5e-9, 1.5e-9)
    ctx = make_ctx("f64", [synth.Sim(mesh, synth.Material(Ms=8e5), synth.uniform_state(mesh))])
    t = ctx.newell_tensor(0, mesh)                     # [6][2nz-1][2ny-1][2nx-1]
    d = (mesh.dx, mesh.dy, mesh.dz)
    for (i, j, k) in ((8, 1, 0), (15, -4, 2), (33, 8, -2), (-69, 3, 1), (50, 0, 0)):
        got = t[:, k + mesh.nz - 1, j + mesh.ny - 1, i + mesh.nx - 1]
        ref = _far_reference(np.array([i * d[0], j * d[1], k * d[2]]), d)
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), (i, j, k)
