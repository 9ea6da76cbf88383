"""FP64 contexts: double-float transforms (MM_F64) against native FP64 arithmetic
(MM_F64_NATIVE) and the FP64 oracle.

An MM_F64 context keeps FP64 state and computes its FFTs, tensor product and z
convolution in double-float arithmetic (about 48 significant bits); its fields must
meet the FP64 bar against the oracle (1e-10 relative, max over cells) and agree with
the all-FP64 kernels to 1e-12.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import make_ctx, max_rel, oracle_rhs
from tests.test_gpu_rhs import MESHES, _mat

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mesh", MESHES)
def test_native_fp64_matches_oracle(mesh):
    m = synth.Mesh(*mesh)
    sim = synth.Sim(m, _mat(), synth.random_state(3, m))
    ctx = make_ctx("f64_native", [sim])
    dmdt, heff = ctx.rhs_host(sim.m0.ravel())
    ref_k, ref_H = oracle_rhs(sim, method="direct")
    assert max_rel(heff, ref_H) < 1e-10 and max_rel(dmdt, ref_k) < 1e-10


@pytest.mark.parametrize("dims", [(33, 17, 2), (9, 6, 5), (6, 5, 8), (5, 4, 9), (70, 3, 1), (64, 64, 1),
                                  (512, 512, 4)])
def test_double_float_agrees_with_native_fp64(dims):
    mesh = synth.Mesh(*dims, 2e-9, 2e-9, 1e-9)
    sim = synth.Sim(mesh, _mat(), synth.random_state(17, mesh))
    out = {}
    for prec in ("f64", "f64_native"):
        ctx = make_ctx(prec, [sim])
        out[prec] = ctx.rhs_host(sim.m0.ravel())
        ctx.close()
    (k_dd, h_dd), (k_64, h_64) = out["f64"], out["f64_native"]
    assert max_rel(h_dd, h_64) < 1e-12 and max_rel(k_dd, k_64) < 1e-12
