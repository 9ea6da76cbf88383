"""Checkpoint and resume of RK45 integration (mm_get_checkpoint / mm_set_checkpoint with
mm_get_m / mm_set_m): a run interrupted and resumed continues bit for bit like the
uninterrupted one, in the same context and in a new one built the same way.
(Collected after the other GPU files.)"""
import numpy as np
import pytest

import synth
from tests.gpu_util import make_ctx

pytestmark = pytest.mark.gpu


def _sims():
    m1 = synth.Mesh(24, 20, 1, 2e-9, 2e-9, 2e-9)
    m2 = synth.Mesh(9, 7, 3, 2e-9, 2e-9, 1e-9)
    mat = synth.Material(Ms=8e5, A=1.3e-11, D=2e-3, dmi=1, Ku=3e5, H=(2e4, 0, 1e4), alpha=0.2)
    return [synth.Sim(m1, mat, synth.random_state(21, m1)), synth.Sim(m2, mat, synth.random_state(22, m2))]


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_resume_is_bit_identical(precision):
    sims = _sims()
    m0 = np.concatenate([s.m0.ravel() for s in sims])
    ctx = make_ctx(precision, sims)
    ctx.set_m(m0)
    ctx.reset_time()
    ctx.rk45_setup(1e-6 if precision == "f64" else 1e-5, t_end=2e-11)
    ctx.rk45_attempts(9)
    ck = [ctx.checkpoint(i) for i in range(len(sims))]
    mk = ctx.get_m(-1)
    assert ck[0]["n_accepted"] + ck[0]["n_rejected"] == 9 and ck[0]["h"] > 0
    ctx.rk45_attempts(13)
    m_ref = ctx.get_m(-1)
    st_ref = [ctx.status(i) for i in range(len(sims))]
    # rewind the same context
    ctx.set_m(mk)
    for i, c in enumerate(ck):
        ctx.restore(i, c)
    assert ctx.checkpoint(0) == ck[0]
    ctx.rk45_attempts(13)
    assert np.array_equal(ctx.get_m(-1), m_ref)
    assert [ctx.status(i) for i in range(len(sims))] == st_ref
    # a new context with the same simulations
    ctx2 = make_ctx(precision, sims)
    ctx2.set_m(mk)
    for i, c in enumerate(ck):
        ctx2.restore(i, c)
    ctx2.rk45_attempts(13)
    assert np.array_equal(ctx2.get_m(-1), m_ref)
    assert [ctx2.status(i) for i in range(len(sims))] == st_ref


def test_invalid_checkpoints_are_refused():
    from paper_2406_16064_gb300 import mm
    sims = _sims()
    ctx = make_ctx("f64", sims)
    good = ctx.checkpoint(0)
    for bad in ({"rtol": 0.0}, {"h": -1e-13}, {"t": float("nan")}, {"status": 7}, {"n_accepted": -1}):
        with pytest.raises(mm.MMError):
            ctx.restore(0, {**good, **bad})
    ctx.restore(0, {**good, "rtol": 1e-6})
    assert ctx.checkpoint(0)["rtol"] == 1e-6
