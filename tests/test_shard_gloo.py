"""Multi-rank path on CPU: world_size-2 gloo ranks shard an uneven batch (no GPU)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from paper_2406_16064_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    w = synth.uneven_batch(seed=5, count=64)
    meshes = [(s.mesh.nx, s.mesh.ny, s.mesh.nz) for s in w.sims]
    mine = shard.shard_sims(meshes, rank, world)
    cost = sum(shard.rhs_cost(*meshes[i]) for i in mine)
    # gather every rank's ids and cost (bookkeeping only; nothing on the data path)
    ids = [None] * world
    dist.all_gather_object(ids, mine)
    costs = torch.tensor([cost], dtype=torch.float64)
    allc = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(allc, costs)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)   # stand-in for a timed region
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((ids, [c.item() for c in allc], t.item()))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_partition_the_batch(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    ids, costs, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(i for part in ids for i in part)
    assert flat == list(range(64))                       # disjoint cover
    assert max(costs) <= 1.15 * min(costs)                # balanced
    assert tmax == float(world)                           # max over ranks


def test_partition_is_deterministic_and_single_rank_takes_all():
    meshes = [(64, 64, 1), (512, 256, 4), (128, 64, 2), (256, 256, 1)] * 4
    assert shard.shard_sims(meshes, 0, 1) == list(range(16))
    a = [shard.shard_sims(meshes, r, 3) for r in range(3)]
    b = [shard.shard_sims(meshes, r, 3) for r in range(3)]
    assert a == b
    assert sorted(sum(a, [])) == list(range(16))
