"""mm_rhs_eval_static: the allocation-free right-hand side for callers that cannot call cudaMalloc.

Such a caller (for example a plugin that is only handed device buffers by its
host application) passes the state and the outputs; the library keeps every
intermediate in a static device array.  The result must equal the
context-based mm_rhs_eval on the same simulation, on two calls in a row (the
second call must not be disturbed by what the first left in the shared array).
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth
from tests.gpu_util import make_ctx, max_rel

pytestmark = pytest.mark.gpu


def _structs(mm, mesh, mat):
    m = mm.mm_mesh(mesh.nx, mesh.ny, mesh.nz, mesh.dx, mesh.dy, mesh.dz)
    t = mm.mm_material()
    t.Ms, t.A, t.D, t.dmi_kind = mat.Ms, mat.A, mat.D, int(mat.dmi)
    t.Ku, t.Kc = mat.Ku, mat.Kc
    for i in range(3):
        t.u[i] = float(mat.u[i])
        t.H[i] = float(mat.H[i])
    t.alpha, t.gamma = mat.alpha, mat.gamma
    t.precession, t.demag = int(mat.precession), int(mat.demag)
    return m, t


def _material(**kw):
    base = dict(Ms=8e5, A=1.3e-11, D=3e-3, dmi=1, Ku=4e5, u=(0.2, 0.3, 0.9), Kc=1e4,
                H=(1e4, -2e4, 3e4), alpha=0.3)
    base.update(kw)
    return synth.Material(**base)


def _check_against_context(torch, mm, precision, mesh, mat, seeds, free_fixed=False):
    """Call the static entry once per seed (calls in a row) and compare each result with
    the context's mm_rhs_eval on the same state.  free_fixed: the device's free memory
    must not change across a call after the first (kernels already loaded)."""
    dt = torch.float64 if precision == "f64" else torch.float32
    tol = 1e-10 if precision == "f64" else 1e-5
    ctx = make_ctx(precision, [synth.Sim(mesh, mat, synth.uniform_state(mesh))])
    L = mm.lib()
    cm, cmat = _structs(mm, mesh, mat)
    prec = mm.MM_F64 if precision == "f64" else mm.MM_F32
    for i, seed in enumerate(seeds):
        m = torch.tensor(synth.random_state(seed, mesh).ravel(), dtype=dt, device="cuda")
        k_ref, h_ref = torch.empty_like(m), torch.empty_like(m)
        ctx.rhs_device(m, k_ref, h_ref)
        torch.cuda.synchronize()
        k, h = torch.full_like(m, float("nan")), torch.full_like(m, float("nan"))
        free0 = torch.cuda.mem_get_info()[0]
        rc = L.mm_rhs_eval_static(ctypes.byref(cm), ctypes.byref(cmat), prec, ctypes.c_void_p(m.data_ptr()),
                                  ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(h.data_ptr()), None)
        assert rc == mm.MM_OK, L.mm_last_error(None)
        torch.cuda.synchronize()
        if free_fixed and i > 0:
            assert torch.cuda.mem_get_info()[0] == free0
        assert max_rel(h.cpu().numpy(), h_ref.cpu().numpy()) < tol
        assert max_rel(k.cpu().numpy(), k_ref.cpu().numpy()) < tol
    ctx.close()


@pytest.mark.parametrize("precision,mesh_dims", [("f64", (24, 20, 2)), ("f32", (33, 17, 1))])
def test_static_rhs_matches_context_rhs_twice(precision, mesh_dims):
    """Two calls in a row, different states; the second call allocates no device memory."""
    torch = pytest.importorskip("torch")
    from paper_2406_16064_gb300 import mm
    mesh = synth.Mesh(*mesh_dims, 2e-9, 2.5e-9, 1.5e-9)
    _check_against_context(torch, mm, precision, mesh, _material(), (11, 12), free_fixed=True)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_static_rhs_without_demag(precision):
    """Demag off: no tensor or spectrum is built; the local terms still match."""
    torch = pytest.importorskip("torch")
    from paper_2406_16064_gb300 import mm
    mesh = synth.Mesh(19, 11, 3, 2e-9, 2e-9, 1e-9)
    _check_against_context(torch, mm, precision, mesh, _material(demag=0), (21, 22))


def test_static_rhs_after_a_call_on_another_mesh():
    """A call on one mesh, a call on a larger mesh (another layout of the shared array),
    then the first mesh again: each matches the context result."""
    torch = pytest.importorskip("torch")
    from paper_2406_16064_gb300 import mm
    a = synth.Mesh(24, 20, 2, 2e-9, 2.5e-9, 1.5e-9)
    b = synth.Mesh(70, 45, 3, 2e-9, 2e-9, 1e-9)
    _check_against_context(torch, mm, "f64", a, _material(), (31,))
    _check_against_context(torch, mm, "f64", b, _material(), (32,))
    _check_against_context(torch, mm, "f64", a, _material(), (33,))


def test_static_rhs_rejects_meshes_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    from paper_2406_16064_gb300 import mm
    mesh = synth.Mesh(512, 512, 1, 2e-9, 2e-9, 2e-9)
    cm, cmat = _structs(mm, mesh, synth.Material(Ms=8e5, A=1e-11))
    L = mm.lib()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")   # the size check rejects before any use
    p = ctypes.c_void_p(buf.data_ptr())
    rc = L.mm_rhs_eval_static(ctypes.byref(cm), ctypes.byref(cmat), mm.MM_F64, p, p, None, None)
    assert rc == mm.MM_EINVAL
    assert b"32 MiB" in L.mm_last_error(None)


@pytest.mark.parametrize("kind", [2, 3])
def test_static_rhs_rejects_other_dmi_classes(kind):
    """Bulk and D_2d DMI run in the context path only; the static entry refuses them
    before touching the GPU."""
    torch = pytest.importorskip("torch")
    from paper_2406_16064_gb300 import mm
    mesh = synth.Mesh(8, 8, 1, 2e-9, 2e-9, 2e-9)
    cm, cmat = _structs(mm, mesh, synth.Material(Ms=8e5, A=1e-11, D=3e-3, dmi=kind))
    L = mm.lib()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    rc = L.mm_rhs_eval_static(ctypes.byref(cm), ctypes.byref(cmat), mm.MM_F64, p, p, None, None)
    assert rc == mm.MM_EINVAL
    assert b"DMI" in L.mm_last_error(None)
