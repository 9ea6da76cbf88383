"""GPU: the single-launch RK45 attempts of small single-plane meshes (one thread-block
cluster per simulation, all attempts of a call in one launch) against the FP64 oracle's
Dormand-Prince steps (Sec. "LLG equation") and against the pass kernels of the same
context."""
import numpy as np
import pytest

import synth
from oracle import demag as D
from oracle import fields as F
from oracle import integrate as I
from tests.gpu_util import make_ctx, max_rel

pytestmark = pytest.mark.gpu


def _ctx(precision, sims, passes=False):
    ctx = make_ctx(precision, sims)
    if passes:
        ctx.set_attempt_kernel(passes=True)
    ctx.set_m(np.concatenate([s.m0.ravel() for s in sims]))
    ctx.reset_time()
    return ctx


def _oracle_steps(sim, n, rtol, t_end=0.0, max_dmdt=0.0):
    Ms = F.ms_array(sim.mesh, sim.mat, sim.Ms_cells)
    Nt = D.mesh_tensor(sim.mesh)
    f = lambda y: F.rhs(sim.mesh, sim.mat, y, Ms, Nt, "direct")[0]
    st = I.Stepper(rtol=rtol, t_end=t_end)
    m = sim.m0.copy()
    for _ in range(n):
        if I.done_time(st):
            break
        m, status = I.step(f, m, st, max_dmdt)
        if status == 2:
            break
    return m, st


# ragged and tiny meshes, every local term, masked cells, precession off
CASES = [
    ((32, 32, 1), dict(Ms=8.6e5, A=1.3e-11, H=(8e3, 0, 0), alpha=0.5), None),
    ((13, 9, 1), dict(Ms=5.8e5, A=1.5e-11, D=3e-3, dmi=1, Ku=8e5, alpha=0.3), None),
    ((5, 31, 1), dict(Ms=8e5, A=1e-11, Kc=-2.4e4, H=(0, 2e4, 1e4), alpha=0.2), None),
    ((32, 1, 1), dict(Ms=8e5, A=1.3e-11, Ku=2e5, u=(1, 1, 0), alpha=0.5, precession=0), None),
    ((1, 1, 1), dict(Ms=8e5, H=(0, 0, 1e5), alpha=0.4), None),
    ((17, 20, 1), dict(Ms=6e5, A=1.2e-11, D=2e-3, dmi=1, Ku=3e5, alpha=0.25), "disk"),
]


def _sim(i, shape, kw, mask):
    mesh = synth.Mesh(*shape, 2e-9, 2.5e-9, 1.5e-9)
    mat = synth.Material(**kw)
    Ms_cells = None
    if mask == "disk":
        z, y, x = np.meshgrid(np.arange(shape[2]), np.arange(shape[1]), np.arange(shape[0]), indexing="ij")
        r2 = (x - shape[0] / 2 + 0.5) ** 2 + (y - shape[1] / 2 + 0.5) ** 2
        Ms_cells = np.where(r2 <= (min(shape[:2]) / 2) ** 2, mat.Ms, 0.0)
    return synth.Sim(mesh, mat, synth.random_state(40 + i, mesh), Ms_cells)


def test_single_launch_is_selected_only_where_it_applies():
    s32 = _sim(0, (32, 32, 1), CASES[0][1], None)
    ctx = _ctx("f64", [s32])
    one, nc = ctx.attempt_kernel()
    assert one and nc in (1, 2, 4, 8, 16)
    before = ctx.launches()
    ctx.rk45_setup(1e-6)
    ctx.rk45_attempts(5)
    assert ctx.launches() - before == 1          # five attempts, one launch
    before = ctx.launches()
    ctx.rk45_attempts(2500)
    assert ctx.launches() - before == 3          # at most 1024 attempts a launch
    assert _ctx("f64", [s32], passes=True).attempt_kernel() == (False, 0)
    for shape in ((33, 8, 1), (8, 33, 1), (8, 8, 2)):
        s = synth.Sim(synth.Mesh(*shape, 2e-9, 2e-9, 2e-9), synth.Material(Ms=8e5, A=1e-11),
                      synth.random_state(1, synth.Mesh(*shape, 2e-9, 2e-9, 2e-9)))
        assert make_ctx("f64", [s]).attempt_kernel() == (False, 0), shape
    s = _sim(1, (13, 9, 1), CASES[1][1], None)
    c = _ctx("f64", [s, s, s])
    c.neb_setup(0, 3, 1e5)
    assert c.attempt_kernel() == (False, 0)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("precision", ["f64", "f64_native"])
def test_single_launch_steps_match_oracle(case, precision):
    """Ten attempts from a random state: the same accepted and rejected steps as the
    oracle's Dormand-Prince run, t to 1e-9 and m to 1e-8 (FP64 contexts)."""
    shape, kw, mask = CASES[case]
    sim = _sim(case, shape, kw, mask)
    ctx = _ctx(precision, [sim])
    assert ctx.attempt_kernel()[0]
    ctx.rk45_setup(1e-6, t_end=0.0)
    ctx.rk45_attempts(10)
    m, st = _oracle_steps(sim, 10, 1e-6)
    g = ctx.status(0)
    assert g["n_accepted"] == st.n_acc and g["n_rejected"] == st.n_rej
    assert abs(g["t"] - st.t) <= 1e-9 * st.t
    assert max_rel(ctx.get_m(0), m) < 1e-8


@pytest.mark.parametrize("precision", ["f64", "f64_native", "f32"])
def test_single_launch_equals_the_pass_kernels(precision):
    """An uneven batch of small films in one launch (one cluster per simulation) against
    the same batch on the pass kernels: same steps and states (FP64 to 1e-10; FP32 over
    the first attempts, where both take the same step sizes, to 1e-5)."""
    sims = [_sim(i, *c) for i, c in enumerate(CASES)]
    n = 12 if precision != "f32" else 3
    rtol = 1e-6 if precision != "f32" else 1e-5
    out = []
    for passes in (False, True):
        ctx = _ctx(precision, sims, passes=passes)
        assert ctx.attempt_kernel()[0] == (not passes)
        ctx.rk45_setup(rtol)
        ctx.rk45_attempts(n)
        out.append((ctx.get_m(-1), [ctx.status(i) for i in range(len(sims))], ctx.layout()[0]))
    (ma, sa, offs), (mb, sb, _) = out
    for i, s in enumerate(sims):
        assert sa[i]["n_accepted"] == sb[i]["n_accepted"] and sa[i]["n_rejected"] == sb[i]["n_rejected"], i
        assert abs(sa[i]["t"] - sb[i]["t"]) <= (1e-9 if precision != "f32" else 1e-5) * sb[i]["t"], i
        k = 3 * s.mesh.ncells
        tol = 1e-10 if precision != "f32" else 1e-5
        assert max_rel(ma[offs[i]:offs[i] + k], mb[offs[i]:offs[i] + k]) < tol, i


def test_single_launch_f32_macro_steps_match_oracle():
    """FP32: the first attempts of the 32x32x1 film against the FP64 oracle (1e-5)."""
    sim = _sim(0, *CASES[0])
    ctx = _ctx("f32", [sim])
    assert ctx.attempt_kernel()[0]
    ctx.rk45_setup(1e-5)
    ctx.rk45_attempts(3)
    m, st = _oracle_steps(sim, 3, 1e-5)
    g = ctx.status(0)
    assert g["n_accepted"] == st.n_acc and g["n_rejected"] == st.n_rej
    assert max_rel(ctx.get_m(0), m) < 1e-5


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_single_launch_relaxes_to_the_oracle_state(precision):
    """Relaxation with precession off to max |dm/dt| < 1e9 rad/s: the single launch
    stops on the criterion and ends within 1e-3 of the FP64 oracle's relaxed state
    (or at the same energy: an equivalent minimum)."""
    kw = dict(Ms=5.8e5, A=1.5e-11, D=3e-3, dmi=1, Ku=8e5, alpha=0.5, precession=0)
    mesh = synth.Mesh(12, 10, 1, 1e-9, 1e-9, 0.5e-9)
    sim = synth.Sim(mesh, synth.Material(**kw), synth.random_state(5, mesh))
    ctx = _ctx(precision, [sim])
    assert ctx.attempt_kernel()[0]
    rtol = 1e-6 if precision == "f64" else 1e-5
    ctx.relax(rtol, max_dmdt=1e9, max_steps=200000, sync_every=256)
    assert ctx.status(0)["status"] == 2
    Ms = F.ms_array(mesh, sim.mat)
    Nt = D.mesh_tensor(mesh)
    f = lambda y: F.rhs(mesh, sim.mat, y, Ms, Nt, "direct")[0]
    m, st = I.run(f, sim.m0.copy(), 1e-6, max_dmdt=1e9, max_steps=200000)
    mg = ctx.get_m(0).reshape(m.shape)
    Eg = F.energies(mesh, sim.mat, mg, Ms, Nt, "direct")["total"]
    Eo = F.energies(mesh, sim.mat, m, Ms, Nt, "direct")["total"]
    dev = np.abs(mg - m).max()
    assert dev < 1e-3 or abs(Eg - Eo) < 1e-6 * abs(Eo), (dev, Eg, Eo)


def test_single_launch_t_end_clip_and_step():
    """t_end clipping lands exactly on t_end (status 1); rk45_step reports one accepted
    step per call on the single launch as on the passes."""
    sim = _sim(1, *CASES[1])
    for passes in (False, True):
        ctx = _ctx("f64", [sim], passes=passes)
        ctx.rk45_setup(1e-6, t_end=3e-13)
        acc, rej = ctx.rk45_step()
        assert acc == 1
        ctx.relax(1e-6, t_end=3e-13, max_steps=1000, sync_every=7)
        g = ctx.status(0)
        assert g["status"] == 1 and abs(g["t"] - 3e-13) < 1e-24
        if passes:
            assert g["n_accepted"] == ref["n_accepted"] and g["n_rejected"] == ref["n_rejected"]
            assert max_rel(ctx.get_m(0), mref) < 1e-10
        else:
            ref, mref = g, ctx.get_m(0)


def test_spin_torques_set_later_leave_the_single_launch():
    """Spin torques switched on after the single launch ran move the context to the pass
    kernels (the single launch has no torque terms); switched off, it returns."""
    sim = _sim(1, *CASES[1])
    ctx = _ctx("f64", [sim])
    ctx.rk45_setup(1e-6)
    ctx.rk45_attempts(1)
    assert ctx.attempt_kernel()[0]
    ctx.set_spin_torque(0, (50.0, 0.0, 0.0), 0.1, 0.0, 0.0, (0.0, 0.0, 1.0))
    assert ctx.attempt_kernel() == (False, 0)
    ctx.set_spin_torque(0, (0.0, 0.0, 0.0), 0.0, 0.0, 0.0, (0.0, 0.0, 1.0))
    assert ctx.attempt_kernel()[0]


@pytest.mark.parametrize("seed", range(40))
def test_single_launch_random_films_equal_the_pass_kernels(seed):
    """Seeded random films of 1..32 x 1..32 cells, random cell sizes, materials and term
    sets (DMI, anisotropies, field, precession, masked cells): five FP64 attempts on the
    single launch and on the pass kernels take the same steps and states (1e-10)."""
    rng = np.random.default_rng(1000 + seed)
    nx, ny = (int(v) for v in rng.integers(1, 33, size=2))
    mesh = synth.Mesh(nx, ny, 1, *(float(v) for v in rng.uniform(1e-9, 4e-9, size=3)))
    kw = dict(Ms=float(rng.uniform(4e5, 1.2e6)), A=float(rng.uniform(0.5e-11, 2e-11)) * (rng.random() < 0.9),
              alpha=float(rng.uniform(0.05, 0.6)), precession=int(rng.random() < 0.8),
              demag=int(rng.random() < 0.9))
    if rng.random() < 0.5:
        kw.update(D=float(rng.uniform(-4e-3, 4e-3)), dmi=1)
    if rng.random() < 0.5:
        u = rng.normal(size=3)
        kw.update(Ku=float(rng.uniform(-5e5, 1e6)), u=tuple(u / np.linalg.norm(u)))
    if rng.random() < 0.3:
        kw.update(Kc=float(rng.uniform(-5e4, 5e4)))
    if rng.random() < 0.6:
        kw.update(H=tuple(float(v) for v in rng.uniform(-1e5, 1e5, size=3)))
    mat = synth.Material(**kw)
    Ms_cells = None
    if rng.random() < 0.3:
        Ms_cells = np.where(rng.random((1, ny, nx)) < 0.8, mat.Ms, 0.0)
    sim = synth.Sim(mesh, mat, synth.random_state(2000 + seed, mesh), Ms_cells)
    out = []
    for passes in (False, True):
        ctx = _ctx("f64", [sim], passes=passes)
        assert ctx.attempt_kernel()[0] == (not passes)
        ctx.rk45_setup(1e-6)
        ctx.rk45_attempts(5)
        out.append((ctx.get_m(0), ctx.status(0)))
    (ma, sa), (mb, sb) = out
    assert sa["n_accepted"] == sb["n_accepted"] and sa["n_rejected"] == sb["n_rejected"], (nx, ny)
    assert abs(sa["t"] - sb["t"]) <= 1e-9 * max(sb["t"], 1e-30)
    assert max_rel(ma, mb) < 1e-10, (nx, ny)
