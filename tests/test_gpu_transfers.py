"""GPU: host transfers of the state (mm_set_m / mm_get_m with host doubles).  In an FP32
context a page-locked host buffer crosses by DMA as FP64 and is converted on the device,
any other one is converted on the host: both round each value once, (float)x, and give
the same bits; FP64 contexts copy the doubles unchanged."""
import numpy as np
import pytest

import synth
from tests.gpu_util import make_ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_pinned_and_pageable_host_buffers_give_the_same_bits(precision):
    import torch
    sims = [synth.Sim(synth.Mesh(n, n, 1, 2e-9, 2e-9, 2e-9), synth.Material(Ms=8e5), None) for n in (7, 300)]
    ctx = make_ctx(precision, [synth.Sim(s.mesh, s.mat, synth.random_state(i, s.mesh)) for i, s in enumerate(sims)])
    total = ctx.layout()[1]
    rng = np.random.default_rng(5)
    m = rng.standard_normal(total)
    expect = m.astype(np.float32).astype(np.float64) if precision == "f32" else m
    ctx.set_m(m)                                        # pageable
    got_pageable = ctx.get_m(-1)
    pinned = torch.empty(total, dtype=torch.float64, pin_memory=True).numpy()
    pinned[:] = m
    ctx.set_m(np.zeros(total))
    ctx.set_m(pinned)                                   # page-locked
    out = torch.empty(total, dtype=torch.float64, pin_memory=True).numpy()
    got_pinned = ctx.get_m(-1, out=out)
    assert got_pinned is out
    assert np.array_equal(got_pageable, expect) and np.array_equal(got_pinned, expect)
    # one simulation's block through a page-locked buffer
    offs, _ = ctx.layout()
    n1 = 3 * sims[1].mesh.ncells
    out1 = torch.empty(n1, dtype=torch.float64, pin_memory=True).numpy()
    assert np.array_equal(ctx.get_m(1, out=out1), expect[offs[1]:offs[1] + n1])
