"""Work partitions across ranks (one GPU per rank) and the NEB chain's exchange.

Independent simulations: the simulations of an uneven batch are independent
units; each rank takes a subset and advances it with its own context, and
nothing on the data path is exchanged.  The partition balances the estimated
cost of one right-hand side, cells plus the padded FFT work, so ranks finish
their attempts together.

NEB chains (Sec. "Miscellaneous"): each rank owns a contiguous block of
images.  An image's tangent and spring force need its two neighbours, so
before every right-hand side a rank sends its first and last images (state
and energy) to the neighbouring ranks and receives theirs (one halo image on
each inner side); and the whole chain takes one step size, so the error norm
(and the stage-1 max |dm/dt|) is a maximum over all ranks.  `neb_blocks`,
`NebHalo` and `allreduce_max` are those three pieces; they move and reduce
data only.  A single simulation is not split: every rank runs a replica.
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


def neb_blocks(n_images: int, world: int):
    """Contiguous blocks [(first, end), ...] of the chain's images, one per rank, sizes
    differing by at most one (the first n_images % world ranks take one more)."""
    if world < 1 or n_images < world:
        raise ValueError("need at least one image per rank")
    base, extra = divmod(n_images, world)
    out, a = [], 0
    for r in range(world):
        b = a + base + (1 if r < extra else 0)
        out.append((a, b))
        a = b
    return out


class NebHalo:
    """Neighbour exchange of one rank's image block over torch.distributed (gloo on CPU,
    NCCL on GPUs): `exchange(first, last)` sends this rank's first image to the previous
    rank and its last image to the next one, and returns (left, right): the last image
    of the previous rank and the first image of the next rank, None at the chain's ends.
    Images are tensors of one shape and dtype on every rank (state, or state and energy
    packed together)."""

    def __init__(self, rank: int, world: int):
        self.rank, self.world = rank, world

    def exchange(self, first, last):
        import torch
        import torch.distributed as dist
        reqs = []
        left = right = None
        if self.rank > 0:
            left = torch.empty_like(first)
            reqs.append(dist.isend(first.contiguous(), self.rank - 1))
            reqs.append(dist.irecv(left, self.rank - 1))
        if self.rank < self.world - 1:
            right = torch.empty_like(last)
            reqs.append(dist.isend(last.contiguous(), self.rank + 1))
            reqs.append(dist.irecv(right, self.rank + 1))
        for req in reqs:
            req.wait()
        return left, right


def allreduce_max(x: float) -> float:
    """The maximum of x over all ranks (the chain's error norm, its max |dm/dt|)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
