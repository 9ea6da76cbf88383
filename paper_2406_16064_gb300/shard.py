"""Sharding of independent simulations across ranks (one GPU per rank).

The simulations of an uneven batch are independent units: each rank takes a
subset and advances it with its own context; nothing on the data path is
exchanged.  The partition balances the estimated cost of one right-hand side,
cells plus the padded FFT work, so ranks finish their attempts together.
A single simulation (or a NEB chain, whose images share one step size) is not
split: every rank runs a replica of it.
"""
from __future__ import annotations

import math


def _pad(n: int, min2: bool = False) -> int:
    if n <= 1:
        return 2 if min2 else 1
    p = 1
    while p < 2 * n - 1:
        p *= 2
    return p


def rhs_cost(nx: int, ny: int, nz: int) -> float:
    """Relative cost of one right-hand side: state traffic + padded FFT work."""
    px, py, pz = _pad(nx, True), _pad(ny), _pad(nz)
    n_fft = (px // 2 + 1) * py * pz
    return nx * ny * nz + n_fft * math.log2(max(2, px * py * pz)) / 8.0


def partition(costs, world: int):
    """Greedy longest-processing-time partition: list of index lists, one per rank.

    Deterministic: ties are broken by index, so every rank computes the same
    partition without communicating.
    """
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def shard_sims(meshes, rank: int, world: int):
    """Indices of the simulations rank `rank` owns; meshes are (nx, ny, nz)."""
    if world <= 1:
        return list(range(len(meshes)))
    return partition([rhs_cost(*m) for m in meshes], world)[rank]
