"""GPU parity at the full-size shapes of every workload, cell by cell against the FP64 oracle.

Each workload's full-size meshes select their own kernel variants and column lengths:

* the uneven batch's members 64x64x1, 128x64x2, 256x256x1 and 512x256x4 (cluster pass of
  2 and 4 planes with 128- and 512-point y columns -- the 512-point columns run with
  32-point register groups in FP32 -- and the single-plane y pass on 128- and 512-point
  columns), all in one batch as the benchmark launches them;
* the NEB chain's 32 images of 128x128x1 (256-point columns), as one batch;
* a 16x256x256 mesh: more planes than a cluster, so separate y passes and the z pass,
  both on 512-point columns, the column lengths of the 256^3 cube;
* the 256^3 cube itself at full size, through the superposition of a few point sources:
  with m = 0 except at a handful of cells, H_d at any cell is a short sum of Newell
  tensors (Eq. 8), which the oracle evaluates exactly at sampled cells.

Tolerances: FP64 fields 1e-10 relative (max over cells of |dH| / max |H|); FP32 fields
1e-5 relative RMS (|dH|_2 / |H|_2).
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


def _check(precision, got_k, got_H, ref_k, ref_H):
    if precision == "f64":
        assert max_rel(got_H, ref_H) < TOL64
        assert max_rel(got_k, ref_k) < TOL64
    else:
        assert rms_rel(got_H, ref_H) < TOL32
        assert rms_rel(got_k, ref_k) < TOL32


def _batch_members():
    """One simulation of each mesh of the uneven batch, materials drawn as the batch draws
    them, random states (so every spectral bin is populated), plus a second 512x256x4
    member with other constants sharing the first one's tensor."""
    w = synth.uneven_batch(seed=11, count=8, precision="f64")
    sims = []
    for k, dims in enumerate(synth.MESH_CHOICES + [(512, 256, 4)]):
        mesh = synth.Mesh(*dims, 2e-9, 2e-9, 2e-9)
        mat = synth.Material(**{**w.sims[k].mat.__dict__, "precession": 1, "H": (1e4, -2e4, 3e4)})
        sims.append(synth.Sim(mesh, mat, synth.random_state(40 + k, mesh)))
    return sims


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_uneven_batch_members_at_full_size(precision):
    sims = _batch_members()
    ctx = make_ctx(precision, sims)
    offs, _ = ctx.layout()
    dmdt, heff = ctx.rhs_host(np.concatenate([s.m0.ravel() for s in sims]))
    for i, s in enumerate(sims):
        n = 3 * s.mesh.ncells
        ref_k, ref_H = oracle_rhs(s, method="fft")
        _check(precision, dmdt[offs[i]:offs[i] + n], heff[offs[i]:offs[i] + n], ref_k, ref_H)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_neb_chain_images_at_full_size(precision):
    """All 32 images of the 128x128x1 chain evaluated in one batch; each image against the
    oracle (precession on here, so both torque terms are compared)."""
    w = synth.neb_chain(precision=precision)
    mat = synth.Material(**{**w.sims[0].mat.__dict__, "precession": 1, "H": (0.0, 0.0, 2e4)})
    sims = [synth.Sim(s.mesh, mat, s.m0) for s in w.sims]
    ctx = make_ctx(precision, sims)
    offs, _ = ctx.layout()
    dmdt, heff = ctx.rhs_host(np.concatenate([s.m0.ravel() for s in sims]))
    Nt = D.mesh_tensor(sims[0].mesh)
    for i in (0, 1, 7, 15, 16, 30):          # skyrmion end, the collapse region, near-uniform end
        s = sims[i]
        n = 3 * s.mesh.ncells
        ref_k, ref_H = oracle_rhs(s, method="fft", Ntab=Nt)
        _check(precision, dmdt[offs[i]:offs[i] + n], heff[offs[i]:offs[i] + n], ref_k, ref_H)
    # the last image is the uniform +z state: only the uniform-state field remains
    assert np.isfinite(heff).all()


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_many_planes_512_point_columns(precision):
    """16x256x256: y columns and z columns of 512 points each (the 256^3 cube's lengths),
    separate y forward, z (forward, product, inverse) and y inverse passes."""
    mesh = synth.Mesh(16, 256, 256, 3e-9, 3e-9, 3e-9)
    mat = synth.Material(Ms=1.7e6, A=2.1e-11, Kc=-2.4e4, alpha=0.02, H=(1e4, 0.0, -1e4))
    sim = synth.Sim(mesh, mat, synth.voronoi_domains(12, mesh, 16))
    ctx = make_ctx(precision, [sim])
    dmdt, heff = ctx.rhs_host(sim.m0.ravel())
    ref_k, ref_H = oracle_rhs(sim, method="fft")
    _check(precision, dmdt, heff, ref_k, ref_H)


def test_bulk_cube_point_sources_at_full_size_f32():
    """256^3 cube, FP32, the benchmark's launch shape (512-point y and z columns, 512^3
    padded grid).  m is zero except at six source cells, so the demag field is
    H_d(r) = -sum_s N(r - r_s) Ms m_s exactly (Eq. 8); the oracle evaluates that sum with
    its own Newell tensor at 200 sampled cells (next to the sources, across the cube,
    on its faces and corners).  Only demag is on, so H_eff = H_d."""
    n, d = 256, 3e-9
    mesh = synth.Mesh(n, n, n, d, d, d)
    Ms = 1.7e6
    mat = synth.Material(Ms=Ms, alpha=0.02)
    rng = np.random.default_rng(5)
    src = [(0, 0, 0), (255, 255, 255), (128, 64, 200), (3, 250, 17), (100, 101, 102), (255, 0, 128)]
    m = np.zeros((3,) + mesh.shape)
    dirs = synth.random_unit_vectors(77, len(src))
    for k, (z, y, x) in enumerate(src):
        m[:, z, y, x] = dirs[:, k]
    ctx = make_ctx("f32", [synth.Sim(mesh, mat, m)])
    _, heff = ctx.rhs_host(m.ravel())
    H = heff.reshape((3,) + mesh.shape)
    targets = set()
    for (z, y, x) in src:                      # the sources and their neighbours (largest fields)
        for dz, dy, dx in ((0, 0, 0), (1, 0, 0), (0, -1, 0), (0, 0, 1), (2, 2, 2)):
            t = (z + dz, y + dy, x + dx)
            if all(0 <= v < n for v in t):
                targets.add(t)
    for c in ((0, 0, 255), (255, 255, 0), (0, 255, 0), (127, 127, 127)):
        targets.add(c)
    while len(targets) < 200:
        targets.add(tuple(int(v) for v in rng.integers(0, n, 3)))
    targets = sorted(targets)
    ref = np.zeros((3, len(targets)))
    T = np.array(targets, dtype=float)
    for k, (z, y, x) in enumerate(src):
        N6 = nw.tensor((T[:, 2] - x) * d, (T[:, 1] - y) * d, (T[:, 0] - z) * d, d, d, d)
        Nm = nw.as_matrix(N6)                     # (3, 3, K)
        ref -= np.einsum("ijk,j->ik", Nm, Ms * dirs[:, k])
    got = np.array([H[:, z, y, x] for (z, y, x) in targets]).T
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    assert err < TOL32 * scale, (err, scale)
