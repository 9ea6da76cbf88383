"""Helpers shared by the GPU parity tests (marshalling and error measures only)."""
import numpy as np

from oracle import demag as D
from oracle import fields as F


def make_ctx(precision, sims):
    from paper_2406_16064_gb300 import mm
    ctx = mm.Context(precision)
    for s in sims:
        ctx.add_sim(s.mesh, s.mat, s.Ms_cells)
    ctx.precompute()
    return ctx


def oracle_rhs(sim, m=None, method="auto", Ntab=None):
    Ms = F.ms_array(sim.mesh, sim.mat, sim.Ms_cells)
    m = sim.m0 if m is None else m
    return F.rhs(sim.mesh, sim.mat, m, Ms, Ntab, method)


def max_rel(a, b):
    """max over cells of |a - b| (3-vector norm) / max over cells of |b|."""
    a = np.asarray(a).reshape(3, -1)
    b = np.asarray(b).reshape(3, -1)
    return float(np.sqrt(((a - b) ** 2).sum(0)).max() / max(np.sqrt((b ** 2).sum(0)).max(), 1e-300))


def rms_rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.sqrt(((a - b) ** 2).sum()) / max(np.sqrt((b ** 2).sum()), 1e-300))
