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


# ------------------------------------------------------------------ NEB image blocks
def _neb_case():
    mesh = synth.Mesh(4, 3, 1, 2e-9, 2e-9, 1e-9)
    mat = synth.Material(Ms=5.8e5, A=1.5e-11, D=3e-3, dmi=1, Ku=8e5, alpha=0.5, precession=0)
    a = synth.uniform_state(mesh, (0, 0, 1))
    b = synth.tilt(synth.uniform_state(mesh, (0.2, 0.1, -1)), 3, 0.05)
    chain = synth.geodesic_chain(a, b, 7)
    for i in range(1, 6):
        chain[i] = synth.tilt(chain[i], 40 + i, 0.1)
    return mesh, mat, chain


def _neb_worker(rank, world, port, q, steps):
    """One rank of the split chain: owns a block of images, exchanges its boundary images'
    state and energy with its neighbours before every right-hand side, and reduces the
    step's maxima over all ranks; the per-image arithmetic is the oracle's."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    import torch
    from oracle import demag as D
    from oracle import fields as F
    from oracle import integrate as I
    from oracle import neb as NB
    mesh, mat, chain = _neb_case()
    n = chain.shape[0]
    Ms = F.ms_array(mesh, mat)
    Nt = D.mesh_tensor(mesh)
    a, b = shard.neb_blocks(n, world)[rank]
    halo = shard.NebHalo(rank, world)
    sent = []

    def f_split(c):                                   # c: (3, b - a, nz, ny, nx)
        own = np.ascontiguousarray(c.swapaxes(0, 1))
        HE = [NB.image_field_energy(mesh, mat, Ms, own[i], Nt, "direct") for i in range(b - a)]
        pack = lambda i: torch.from_numpy(np.concatenate([own[i].ravel(), [HE[i][1]]]))
        left, right = halo.exchange(pack(0), pack(b - a - 1))
        sent.append(1)
        ext = list(own)
        E = [e for _, e in HE]
        H = [h for h, _ in HE]
        if left is not None:
            ext.insert(0, left.numpy()[:-1].reshape(own[0].shape))
            E.insert(0, float(left[-1]))
            H.insert(0, np.zeros_like(H[0]))
        if right is not None:
            ext.append(right.numpy()[:-1].reshape(own[0].shape))
            E.append(float(right[-1]))
            H.append(np.zeros_like(H[0]))
        out = NB.chain_forces(mat, Ms, np.stack(ext), np.stack(H), np.array(E), 1e5)
        lo = 1 if left is not None else 0
        return np.ascontiguousarray(out[lo:lo + (b - a)].swapaxes(0, 1))

    st = I.Stepper(rtol=1e-5)
    c = np.ascontiguousarray(chain[a:b].swapaxes(0, 1))
    for _ in range(steps):
        c, _ = I.step(f_split, c, st, reduce=shard.allreduce_max)
        if a == 0:
            c[:, 0] = chain[0]
        if b == n:
            c[:, -1] = chain[-1]
    mine = np.ascontiguousarray(c.swapaxes(0, 1))
    got = [None] * world
    dist.all_gather_object(got, (a, b, mine, st.t, st.h, st.n_acc, st.n_rej, len(sent)))
    if rank == 0:
        q.put(got)
    dist.destroy_process_group()


def test_neb_image_blocks_split_equals_single_process_chain():
    """Two gloo ranks split a 7-image chain (4 + 3 images); after every stage's halo
    exchange and the shared step size, the chain equals the single-process oracle
    chain bit for bit, with the same accepted and rejected steps."""
    from oracle import demag as D
    from oracle import fields as F
    from oracle import neb as NB
    import numpy as np
    world, steps = 2, 6
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_neb_worker, args=(r, world, port, q, steps)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mesh, mat, chain = _neb_case()
    c, E, st = NB.relax(mesh, mat, F.ms_array(mesh, mat), chain, 1e5, 1e-5, steps, D.mesh_tensor(mesh), "direct")
    assert [(g[0], g[1]) for g in got] == shard.neb_blocks(chain.shape[0], world) == [(0, 4), (4, 7)]
    split = np.concatenate([g[2] for g in got])
    assert np.array_equal(split, c)
    for g in got:
        assert (g[3], g[4], g[5], g[6]) == (st.t, st.h, st.n_acc, st.n_rej)
        assert g[7] == 7 * steps                       # one exchange per right-hand side
    assert st.n_acc > 0


def test_neb_blocks_partition():
    assert shard.neb_blocks(32, 1) == [(0, 32)]
    assert shard.neb_blocks(32, 3) == [(0, 11), (11, 22), (22, 32)]
    blocks = shard.neb_blocks(7, 4)
    assert blocks[0][0] == 0 and blocks[-1][1] == 7 and all(b > a for a, b in blocks)
    assert all(blocks[i][1] == blocks[i + 1][0] for i in range(3))
    with pytest.raises(ValueError):
        shard.neb_blocks(2, 3)


# ------------------------------------------------------------------ batch results
def _batch_worker(rank, world, port, q):
    """One rank of a sharded batch: three RK45 steps of its own simulations (oracle
    arithmetic); every rank's results gathered on rank 0."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import demag as D
    from oracle import fields as F
    from oracle import integrate as I
    w = synth.uneven_batch(seed=9, count=6, precision="f64", choices=[(8, 8, 1), (6, 4, 2), (12, 6, 1)])
    meshes = [(s.mesh.nx, s.mesh.ny, s.mesh.nz) for s in w.sims]
    out = {}
    for i in shard.shard_sims(meshes, rank, world):
        s = w.sims[i]
        Ms = F.ms_array(s.mesh, s.mat)
        Nt = D.mesh_tensor(s.mesh)
        st = I.Stepper(rtol=1e-6)
        m = s.m0.copy()
        for _ in range(3):
            m, _ = I.step(lambda y: F.rhs(s.mesh, s.mat, y, Ms, Nt, "direct")[0], m, st)
        out[i] = (m, st.t, st.n_acc)
    got = [None] * world
    dist.all_gather_object(got, out)
    if rank == 0:
        q.put(got)
    dist.destroy_process_group()


def test_sharded_batch_results_equal_unsharded():
    from oracle import demag as D
    from oracle import fields as F
    from oracle import integrate as I
    import numpy as np
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    merged = {}
    for part in got:
        assert not (set(part) & set(merged))           # disjoint
        merged.update(part)
    w = synth.uneven_batch(seed=9, count=6, precision="f64", choices=[(8, 8, 1), (6, 4, 2), (12, 6, 1)])
    assert sorted(merged) == list(range(6))
    for i, s in enumerate(w.sims):
        Ms = F.ms_array(s.mesh, s.mat)
        Nt = D.mesh_tensor(s.mesh)
        st = I.Stepper(rtol=1e-6)
        m = s.m0.copy()
        for _ in range(3):
            m, _ = I.step(lambda y: F.rhs(s.mesh, s.mat, y, Ms, Nt, "direct")[0], m, st)
        assert np.array_equal(merged[i][0], m) and merged[i][1:] == (st.t, st.n_acc)
