"""Throughput of the LLG right-hand side inside adaptive RK45 on one GB300.

A step is one Dormand-Prince attempt over the whole workload: 7 right-hand
sides (RK prologue, zero-padded FFT demag with the fused tensor product,
exchange/DMI/anisotropy/Zeeman epilogue, LL torque), the FP64 error-norm
reduction, the step controller and the projection onto |m| = 1.  The metric
counts cell-updates: cells x right-hand sides / second.

Default workload: 512 x 512 x 4 thin film with interfacial DMI and
perpendicular anisotropy, ~200 reversed disks (FP32 path; the FP64 path is
measured on the same workload and reported beside it).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload film|film_relax_32|cube|cube128|neb|batch|sweep] [--driver rk45|sd|rk4-cayley|rk4-proj|...]

`--driver sd` times steepest-descent steps (one effective-field evaluation and
the Barzilai-Borwein update each) instead of RK45 attempts; `--driver
relax-compare` relaxes the workload from its start below --max-dmdt with RK45
and with steepest descent and reports both wall times.

`--driver rk4-cayley` / `--driver rk4-proj` time fixed classical RK4 steps
(four right-hand sides each) on the Cayley-transform variable or with
projection; `--driver cayley-error` runs the paper's macrospin comparison of the
two schemes (error against the closed form at 1 ns over a range of h).

`--ext` adds per-cell exchange and DMI constants and a Zhang-Li drift to the
workload, so the extended x-inverse variant runs (workload name `*_ext`).

`--driver cufft-compare` times the zero-padded demag convolution done with cuFFT
(torch.fft, three R2C + product + three C2R on the padded grid) against this
library's whole right-hand side on the workload's first simulation (a timed
comparison only; cuFFT is never on the product path).

`--workload sweep` times the N x N x 1 family of the paper's throughput
comparison (demag + exchange + Zeeman, N = 128 ... 4096, FP32) and reports each
N as RHS cell-updates/s and as Heun-equivalent cells/s (RHS rate / 2).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "LLG RHS cell-updates/s, FP32/batched vs FP64 plain, % HBM roofline, 1 GB300"
UNIT = "cell-updates/s"
L2_BYTES = 129e6


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ workloads
def workload_for(args, world=1):
    w = workload(args.workload, world)
    return synth.with_extended_terms(w) if getattr(args, "ext", False) else w


def workload(name, world=1):
    if name == "film":
        return synth.skyrmion_film(precision="f32")
    if name == "film_relax_32":
        return synth.film_relax_32()
    if name == "cube":
        return synth.bulk_cube()
    if name == "cube128":
        # the cube's recipe at 128^3 (spectrum 0.2 GB, above L2): a small case of its kernels for ncu
        return synth.bulk_cube(n=128)
    if name == "neb":
        return synth.neb_chain()
    if name == "batch":
        return synth.uneven_batch(count=64 * world)
    if name == "sweep":
        return synth.square_film(512)
    raise SystemExit(f"unknown workload {name}")


def cells(w):
    return sum(s.mesh.ncells for s in w.sims)


def pad(n, min2=False):
    if n <= 1:
        return 2 if min2 else 1
    p = 1
    while p < 2 * n - 1:
        p *= 2
    return p


def tensor_bytes(s, e):
    """Bytes of the stored demag tensor one right-hand side reads.  Films of 2..8 planes
    (cluster pass) convolve along z directly: xx, yy, zz, xy at dz = 0..nz-1 and xz, yz
    at dz = 1..nz-1 per (kx, ky >= 0) bin; other meshes: ncomp components at the kz <= Pz/2
    bins."""
    nx, ny, nz = s.mesh.nx, s.mesh.ny, s.mesh.nz
    Px, Py, Pz = pad(nx, True), pad(ny), pad(nz)
    Kx = Px // 2 + 1
    if Pz > 1 and Py > 1 and nz <= 8:
        return (4 * nz + 2 * (nz - 1)) * (Py // 2 + 1) * Kx * e
    ncomp = 6 if Pz > 1 else 4
    return ncomp * (Pz // 2 + 1) * (Py // 2 + 1) * Kx * e


def kernel_bytes(w, e, spectrum=True):
    """Compulsory bytes per attempt of each kernel kind: every stage vector, state, spectrum
    row and tensor value a kernel must read or write once (e = bytes of one real value).
    The x forward pass of stage s reads y_n and the s-1 earlier k's, writes y_s (s > 1) and
    the partial error vector (s = 7) and the x-transform rows; the column passes read and
    write the spectrum and read the tensor; the x inverse reads the spectrum rows and the
    stage state and writes k_s (and reads the partial error at s = 7); the projection reads
    y and writes m.  spectrum=False leaves out the demag spectrum written and read back
    between the passes (an intermediate of the implementation, not algorithmic traffic of
    the right-hand side): what remains are the state and stage vectors and the tensor."""
    out = {k: 0.0 for k in ("x_forward", "y_forward", "z_fused", "y_inverse", "y_fused",
                            "x_inverse_epilogue", "project", "yz_cluster")}
    sp = 1.0 if spectrum else 0.0
    for s in w.sims:
        n = s.mesh.ncells
        nx, ny, nz = s.mesh.nx, s.mesh.ny, s.mesh.nz
        Px, Py, Pz = pad(nx, True), pad(ny), pad(nz)
        Kx = Px // 2 + 1
        c = 2 * e                                    # one complex value
        spec_rows = 3 * nz * ny * Kx * c * sp        # x-transform rows (ny of Py)
        spec_full = 3 * nz * Py * Kx * c * sp        # all Py rows
        tens = tensor_bytes(s, e)
        demag = s.mat.demag
        for st in range(1, 8):
            out["x_forward"] += 3 * e * n * st + (3 * e * n if st > 1 else 0) + (3 * e * n if st == 7 else 0)
            if demag:
                out["x_forward"] += spec_rows
                if Pz > 1 and Py > 1 and nz <= 8:
                    out["yz_cluster"] += 2 * spec_rows + tens
                elif Pz > 1:
                    if Py > 1:
                        out["y_forward"] += spec_rows + spec_full
                        out["y_inverse"] += spec_full + spec_rows
                    out["z_fused"] += 2 * spec_full + tens
                elif Py > 1:
                    out["y_fused"] += 2 * spec_rows + tens
            out["x_inverse_epilogue"] += (spec_rows if demag else 0) + 6 * e * n + (3 * e * n if st == 7 else 0)
            if getattr(s.mat, "A_cells", None) is not None or getattr(s.mat, "D_cells", None) is not None:
                out["x_inverse_epilogue"] += 2 * e * n          # per-cell A and D
        out["project"] += 6 * e * n
    return out


def step_bytes_whole(w, e):
    """The whole-step algorithmic figure: 22.5 e + T bytes per cell-update (T = tensor bytes / cell)."""
    tot = 0.0
    for s in w.sims:
        nx, ny, nz = s.mesh.nx, s.mesh.ny, s.mesh.nz
        Px, Py, Pz = pad(nx, True), pad(ny), pad(nz)
        T = tensor_bytes(s, e) / s.mesh.ncells if s.mat.demag else 0.0
        tot += (22.5 * e + T) * s.mesh.ncells * 7
    return tot


# ------------------------------------------------------------------ ncu traffic
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.md")


# The sources that define (and instantiate) the kernels of the right-hand side
# and of the RK45 attempt, whose DRAM counters profiles/dram_traffic.md records.
KERNEL_SOURCES = ("control.cuh", "engine.cuh", "engine_f32.cu", "engine_f64.cu", "engine_impl.cuh",
                  "ext_terms.cuh", "mm_kernels.cuh", "passes.cuh", "plan.h")


def source_fingerprint():
    """Hash of the pass-kernel sources: DRAM counters taken on other sources are stale."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2406_16064_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        path = os.path.join(csrc, fn)
        if os.path.exists(path):
            with open(path, "rb") as f:
                h.update(fn.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kind, workload_name):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch of a kernel kind on a
    workload, from the committed ncu summary; None unless it was captured on the
    current kernel sources."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    fp = source_fingerprint()
    with open(TRAFFIC_FILE) as f:
        for line in f:
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) >= 5 and cells[0] == workload_name and cells[1] == kind and cells[3] == fp:
                try:
                    return float(cells[4])
                except ValueError:
                    return None
    return None


# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(self.index), "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, nme in enumerate(names):
                if len(r) > 5 + i and r[5 + i].strip().lower() == "active":
                    reasons.add(nme)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------------ oracle timing
def _oracle_worker(sim, n_warm, n_timed, budget_s, barrier, queue):
    """One host process of the oracle timing: W untimed right-hand sides of `sim`, then,
    after every process has reached the barrier, n_timed of them (or as many as fit
    budget_s when n_timed is None); reports (start, end, evaluations, cells)."""
    from oracle import demag as D
    from oracle import fields as F
    try:
        Nt = D.mesh_tensor(sim.mesh) if sim.mat.demag else None
        Ms = F.ms_array(sim.mesh, sim.mat, sim.Ms_cells)
        t0 = time.perf_counter()
        for _ in range(max(1, n_warm)):
            F.rhs(sim.mesh, sim.mat, sim.m0, Ms, Nt, "fft")
        one = (time.perf_counter() - t0) / max(1, n_warm)
        n = n_timed if n_timed is not None else int(max(1, budget_s // max(one, 1e-9)))
        barrier.wait()
        t0 = time.time()
        for _ in range(n):
            F.rhs(sim.mesh, sim.mat, sim.m0, Ms, Nt, "fft")
        queue.put((t0, time.time(), n, sim.mesh.ncells))
    except BaseException as e:  # noqa: BLE001 - reported to the parent, which raises
        barrier.abort()
        queue.put(("error", repr(e)))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_workers(sim, want=None):
    """Processes for the oracle timing: one per host core, fewer if the host's available
    memory cannot hold that many copies of the oracle's zero-padded FFT arrays (about
    27 padded grids of 8 bytes each per process)."""
    p = host_cores() if want is None else want
    grid = 1
    for n in (sim.mesh.nx, sim.mesh.ny, sim.mesh.nz):
        grid *= 2 * n if n > 1 else 1
    need = 27 * 8 * grid * 1.5 + 300e6
    try:
        with open("/proc/meminfo") as f:
            avail = next(int(l.split()[1]) * 1024 for l in f if l.startswith("MemAvailable"))
        p = min(p, max(1, int(avail * 0.8 // need)))
    except (OSError, StopIteration, ValueError):
        pass
    return max(1, p)


def oracle_pool_rate(sim, n_warm, n_timed=None, budget_s=12.0, workers=None):
    """The FP64 oracle, unchanged, in one process per host core (spawned, so it is safe
    after CUDA initialisation), each evaluating independent right-hand sides of `sim`
    concurrently.  Returns (cell-updates/s over all processes, processes, evaluations
    per process, seconds): the rate is all processes' cells x evaluations divided by the
    span from the first start to the last end, measured after a common barrier."""
    import multiprocessing as mp
    P = oracle_workers(sim, workers)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")          # one thread per process: the processes are the parallelism
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(P)
    q = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(sim, n_warm, n_timed, budget_s, barrier, q))
             for _ in range(P)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=900) for _ in range(P)]
    for pr in procs:
        pr.join()
    bad = [r for r in res if r[0] == "error"]
    if bad:
        raise RuntimeError(f"oracle worker failed: {bad[0][1]}")
    t0 = min(r[0] for r in res)
    t1 = max(r[1] for r in res)
    upd = sum(r[2] * r[3] for r in res)
    return upd / (t1 - t0), P, min(r[2] for r in res), t1 - t0


def oracle_rate(w, budget_s):
    """FP64 oracle right-hand sides of the workload's first simulation on the host cores."""
    s = w.sims[0]
    v, P, n, dt = oracle_pool_rate(s, 1, None, budget_s)
    return v, P, n, dt, s.mesh


# ------------------------------------------------------------------ main
REFERENCE_BUDGET_S = 90.0       # the whole --warmup W --steps K reference run


def reference_block(s, frac):
    """The first ny' x nx' columns of simulation s, all planes, with its state, Ms and
    material (a bounded sample of the workload): nx', ny' the powers of two at or below
    sqrt(frac) nx, sqrt(frac) ny (at least 8), so the zero-padded FFT grid, which sets the
    oracle's cost, shrinks with the block."""
    if frac >= 1.0:
        return s
    r = math.sqrt(frac)
    p2 = lambda v: 1 << max(3, int(math.floor(math.log2(max(v, 1.0)))))
    nx = min(s.mesh.nx, p2(r * s.mesh.nx))
    ny = min(s.mesh.ny, p2(r * s.mesh.ny))
    mesh = synth.Mesh(nx, ny, s.mesh.nz, s.mesh.dx, s.mesh.dy, s.mesh.dz)
    m0 = np.ascontiguousarray(s.m0[:, :, :ny, :nx])
    Ms = None if s.Ms_cells is None else np.ascontiguousarray(s.Ms_cells[:, :ny, :nx])
    return synth.Sim(mesh, s.mat, m0, Ms)


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores: W untimed and exactly K timed right-hand sides
    of the workload's first simulation, or of a block of it sized so the W + K steps
    take about REFERENCE_BUDGET_S seconds."""
    from oracle import demag as D
    from oracle import fields as F
    w = workload_for(args)
    line = {"impl": "reference", "metric": METRIC, "unit": UNIT, "n_gpus": world, "higher_is_better": True,
            "data": "synthetic", "dtype": "f64",
            "config": {"workload": w.name, "cells": cells(w), "path": "FP64 numpy oracle, host cores"}}
    if rank != 0:
        return None
    K, W = args.steps, args.warmup
    s0 = w.sims[0]
    Nt = D.mesh_tensor(s0.mesh) if s0.mat.demag else None
    Ms = F.ms_array(s0.mesh, s0.mat, s0.Ms_cells)
    t0 = time.perf_counter()
    F.rhs(s0.mesh, s0.mat, s0.m0, Ms, Nt, "fft")
    one = time.perf_counter() - t0
    del Nt
    # the processes run concurrently and share the memory bus: allow each step twice the
    # single-process time
    s = reference_block(s0, min(1.0, REFERENCE_BUDGET_S / max(2.0 * (K + W) * one, 1e-9)))
    value, P, _, dt = oracle_pool_rate(s, W, K)
    full = s0.mesh
    where = ("" if s is s0 else
             f" of a {s.mesh.nx}x{s.mesh.ny}x{s.mesh.nz} block of the {full.nx}x{full.ny}x{full.nz} mesh")
    line.update({"value": value, "steps": K, "warmup": W, "ms_per_step": 1e3 * dt / max(K, 1),
                 "scaling": "weak", "vs_baseline": None,
                 "cpu_baseline": {"value": value, "unit": UNIT, "cores": P, "kind": "oracle",
                                  "sample": f"per step, one right-hand side{where} in each of {P} processes "
                                            f"(FFT demag, numpy, one thread each, all running at once)"},
                 "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    return line


def timed_attempts(ctx, torch, stream, k):
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    ctx.rk45_attempts(k)
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end)


def setup_ctx(mm, w, precision, stream, rtol, tune=False, info=None):
    """A context with the workload's simulations, state and RK45 settings.  tune: give
    every mesh its autotuned tiles (cached per GPU, build, precision and mesh), recording
    the choices in `info`."""
    ctx = mm.Context(precision, stream=stream.cuda_stream)
    for s in w.sims:
        ctx.add_sim(s.mesh, s.mat, s.Ms_cells)
    if tune:
        import torch
        from paper_2406_16064_gb300 import tuning
        t0 = time.perf_counter()
        got = tuning.tune_context(ctx, [s.mesh for s in w.sims], torch.cuda.get_device_name(), reps=8)
        if info is not None:
            info["tuning"] = {k.split("|", 2)[2]: v for k, v in got.items()}
            info["tuning_seconds"] = time.perf_counter() - t0
    ctx.precompute()
    ctx.set_m(np.concatenate([s.m0.ravel() for s in w.sims]))
    if w.neb:
        ctx.neb_setup(0, len(w.sims), w.neb["k_spring"])
    ctx.reset_time()
    ctx.rk45_setup(rtol, t_end=0.0, max_dmdt=0.0)
    return ctx


SWEEP_N = (128, 256, 512, 1024, 2048, 4096)


def run_sweep(args, rank, world, dist):
    import torch
    from paper_2406_16064_gb300 import mm
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    prec = args.precision or "f32"
    rows = []
    launches = 0
    with Clocks(dev) as clk:
        for n in (tuple(int(v) for v in args.sweep_n.split(",")) if args.sweep_n else SWEEP_N):
            w = synth.square_film(n, precision=prec)
            ctx = setup_ctx(mm, w, prec, stream, w.rtol)
            k = int(max(10, min(args.steps, args.steps * (512 * 512) // (n * n))))
            ctx.rk45_attempts(args.warmup)
            n0 = ctx.launches()
            if dist:
                dist.barrier()
            ms = timed_attempts(ctx, torch, stream, k)
            torch.cuda.synchronize()
            t = torch.tensor([ms], dtype=torch.float64, device="cuda")
            if dist:
                dist.barrier()
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
            launches += ctx.launches() - n0
            rate = world * n * n * 7 * k / (float(t.item()) / 1e3)
            prof = ctx.profile_attempts(2)
            rows.append({"n": n, "value": rate, "heun_equivalent_cells_per_s": rate / 2,
                         "ms_per_step": float(t.item()) / k, "steps": k,
                         "kernels_ms_per_step": {kk: v[0] / 2 for kk, v in prof.items() if v[1]}})
            ctx.close()
            del ctx
    best = max(rows, key=lambda r: r["value"])
    line = {"metric": METRIC, "value": best["value"], "unit": UNIT, "n_gpus": world, "steps": best["steps"],
            "warmup": args.warmup, "ms_per_step": best["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": f"square_film_NxNx1_{prec}", "n_best": best["n"], "rhs_per_step": 7,
                       "terms": "demag + exchange + Zeeman",
                       "parallelism": "replicas" if world > 1 else "single"},
            "sweep": rows, "clocks": clk.summary(), "gpu_launches": launches}
    return line


def run_gpu(args, rank, world, dist):
    import torch
    from paper_2406_16064_gb300 import mm
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    w = workload_for(args, world)
    sharded = world > 1 and len(w.sims) > 1 and not w.neb
    if sharded:
        # independent simulations: each rank owns a cost-balanced share of the global batch
        from paper_2406_16064_gb300 import shard
        mine = shard.shard_sims([(s.mesh.nx, s.mesh.ny, s.mesh.nz) for s in w.sims], rank, world)
        w.sims = [w.sims[i] for i in mine]
    prec = args.precision or ("f64" if args.workload == "film_relax_32" else "f32")
    w.precision = prec
    e = 8 if prec == "f64" else 4
    ncell = cells(w)
    tinfo = {}
    ctx = setup_ctx(mm, w, prec, stream, w.rtol, tune=not args.no_autotune, info=tinfo)
    ctx.rk45_attempts(args.warmup)
    torch.cuda.synchronize()
    n0 = ctx.launches()
    if dist:
        dist.barrier()
    with Clocks(dev) as clk:
        ms = timed_attempts(ctx, torch, stream, args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = ctx.launches() - n0
    clocks = clk.summary()
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    ncell_job = world * ncell
    if sharded:
        c = torch.tensor([float(ncell)], dtype=torch.float64, device="cuda")
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        ncell_job = int(c.item())
    value = ncell_job * 7 * args.steps / (ms_max / 1e3)
    # per-kernel durations inside the same step (events on the launching stream)
    kb = kernel_bytes(w, e)
    kb_alg = kernel_bytes(w, e, spectrum=False)
    hbm, peak_kind = peaks()
    reps = max(1, min(5, args.steps))
    rows = {}
    dom, achieved, bytes_per_launch, avg_launch_ms = None, None, None, None
    single, ncl = ctx.attempt_kernel()
    prof = {} if single else ctx.profile_attempts(reps)
    for k, (tms, cnt) in prof.items():
        if cnt:
            rows[k] = {"ms_per_attempt": tms / reps, "launches": cnt,
                       "algorithmic_gbs": (kb_alg.get(k, 0.0) * reps) / (tms / 1e3) / 1e9
                       if kb_alg.get(k) and tms > 0 else None,
                       "with_spectrum_gbs": (kb.get(k, 0.0) * reps) / (tms / 1e3) / 1e9
                       if kb.get(k) and tms > 0 else None}
    step_ms = ms_max / args.steps
    step_bytes = step_bytes_whole(w, e)
    if single:
        # one launch runs every timed attempt (k_small_rk, one cluster per simulation):
        # its algorithmic bytes are the whole-step figure, kept in shared memory
        dom = "attempt_single_launch"
        per = min(args.steps, 1024)                 # the library issues at most 1024 attempts a launch
        nl = -(-args.steps // per)
        rows[dom] = {"ms_per_attempt": step_ms, "launches": nl, "attempts_per_launch": per,
                     "cluster_ctas_per_simulation": ncl}
        avg_launch_ms = ms_max / nl
        alg_per_launch = step_bytes * args.steps / nl
        spectrum_per_launch = 0.0
    else:
        dom = max((k for k in rows if kb.get(k)), key=lambda k: rows[k]["ms_per_attempt"])
        launches_dom = prof[dom][1] / reps
        avg_launch_ms = prof[dom][0] / prof[dom][1]
        alg_per_launch = kb_alg[dom] / launches_dom
        spectrum_per_launch = (kb[dom] - kb_alg[dom]) / launches_dom
    bytes_per_launch = alg_per_launch + spectrum_per_launch
    achieved = bytes_per_launch / (avg_launch_ms / 1e3) / 1e9
    achieved_alg = alg_per_launch / (avg_launch_ms / 1e3) / 1e9
    # end to end through the C ABI with host buffers: H2D of m, one attempt, D2H of m, each
    # step, from and to one page-locked host array of doubles (the public API's host form)
    ke = max(20, min(200, args.steps // 10))
    nstate = ctx.layout()[1]
    mhost = torch.empty(nstate, dtype=torch.float64, pin_memory=True).numpy()
    ctx.get_m(-1, out=mhost)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        ctx.set_m(mhost)
        ctx.rk45_attempts(1)
        ctx.get_m(-1, out=mhost)
    e2e_s = time.perf_counter() - t0
    e2e_value = (ncell_job / ncell) * ncell * 7 * ke / e2e_s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": {"workload": w.name, "cells": ncell, "rhs_per_step": 7, "rtol": w.rtol,
                   "parallelism": (f"sharded sims, {len(w.sims)} on rank 0" if sharded else
                                   "replicas" if world > 1 else "single"),
                   "l2": (f"single launch: the whole state ({int(step_bytes / 7 / 1e3)} kB per RHS) stays in "
                          f"the cluster's shared memory; one launch covers every timed attempt" if single else
                          f"inputs larger than L2: working set ~{int(step_bytes / 7 / 1e6)} MB per RHS "
                          f"(state, 7 stage vectors, spectrum, tensor) vs 129 MB L2")},
        "roofline": {"bound": "hbm", "kernel": "k_small_rk" if single else dom, "achieved": achieved, "peak": hbm,
                     "unit": "GB/s",
                     "frac": achieved / hbm if achieved else None, "peak_kind": f"of {peak_kind}",
                     "bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_launch_ms,
                     "bytes_meaning": ("the algorithmic bytes of every attempt of the launch (22.5 e + T per "
                                       "cell-update); the single launch keeps state, stage vectors and spectra "
                                       "in shared memory and moves only m and the tensor through DRAM" if single
                                       else "compulsory bytes of the launch: state, stage vectors and tensor (the "
                                       "algorithmic bytes) plus the demag spectrum it reads and writes between "
                                       "passes (implementation traffic), each given below"),
                     "algorithmic_bytes_per_launch": alg_per_launch,
                     "spectrum_bytes_per_launch": spectrum_per_launch,
                     "achieved_algorithmic": achieved_alg, "frac_algorithmic": achieved_alg / hbm,
                     "traffic": None if single else recorded_traffic(dom, w.name),
                     "source_fingerprint": source_fingerprint(),
                     "step_algorithmic_gbs": step_bytes / (step_ms / 1e3) / 1e9,
                     "step_frac": step_bytes / (step_ms / 1e3) / 1e9 / hbm},
        "kernels": rows,
        "autotune": tinfo or None,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * nstate,
                "d2h_bytes_per_step": 8 * nstate, "steps": ke,
                "host_buffer": "page-locked float64 (FP32 contexts convert on the device)"},
        "gpu_launches": launches,
    }
    ctx.close()
    # the FP64 plain path on the same workload, fewer steps
    if not args.no_f64 and prec == "f32":
        w64 = workload(args.workload, world)
        w64.sims = w.sims
        w64.precision = "f64"
        t64 = {}
        ctx64 = setup_ctx(mm, w64, "f64", stream, 1e-6, tune=not args.no_autotune, info=t64)
        ctx64.rk45_attempts(max(1, args.warmup // 4))
        k64 = max(3, min(args.steps, 100))
        ms64 = timed_attempts(ctx64, torch, stream, k64)
        v64 = (ncell_job / ncell) * ncell * 7 * k64 / (ms64 / 1e3)
        line["f64"] = {"value": v64, "ms_per_step": ms64 / k64, "steps": k64,
                       "step_algorithmic_gbs": step_bytes_whole(w, 8) / (ms64 / k64 / 1e3) / 1e9,
                       "step_frac": step_bytes_whole(w, 8) / (ms64 / k64 / 1e3) / 1e9 / hbm,
                       "autotune": t64 or None,
                       "transforms": "double-float (FP32 pairs); FP64 state, prologue, epilogue and reductions"}
        ctx64.close()
        # the same FP64 workload with native FP64 arithmetic in every kernel, for comparison
        ctxn = setup_ctx(mm, w64, "f64_native", stream, 1e-6)
        ctxn.rk45_attempts(1)
        kn = 3
        msn = timed_attempts(ctxn, torch, stream, kn)
        line["f64"]["native_fp64"] = {"value": (ncell_job / ncell) * ncell * 7 * kn / (msn / 1e3),
                                      "ms_per_step": msn / kn, "steps": kn}
        ctxn.close()
    if rank == 0 and not args.no_cpu:
        v, P, n, dt, mesh = oracle_rate(w, 12.0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": P, "kind": "oracle",
                                "sample": f"{P} processes at once, each {n}+ FP64 right-hand sides of the "
                                          f"{mesh.nx}x{mesh.ny}x{mesh.nz} mesh over {dt:.1f} s (numpy oracle, "
                                          f"FFT demag, one thread each; tensor setup excluded)"}
    return line


def run_sd(args, rank, world, dist):
    """Steepest-descent steps (one effective-field evaluation each) on the workload."""
    import torch
    from paper_2406_16064_gb300 import mm
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    w = workload(args.workload, world)
    if w.neb:
        raise SystemExit("--driver sd: the NEB workload has its own driver")
    prec = args.precision or ("f64" if args.workload == "film_relax_32" else "f32")
    ctx = mm.Context(prec, stream=stream.cuda_stream)
    for s in w.sims:
        ctx.add_sim(s.mesh, s.mat, s.Ms_cells)
    ctx.precompute()
    m0 = np.concatenate([s.m0.ravel() for s in w.sims])
    ctx.set_m(m0)
    ctx.minimize(0.0, max_steps=args.warmup, sync_every=args.warmup)
    ctx.set_m(m0)
    n0 = ctx.launches()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with Clocks(dev) as clk:
        start.record(stream)
        ctx.minimize(0.0, max_steps=args.steps, sync_every=args.steps)
        end.record(stream)
        end.synchronize()
    ms = start.elapsed_time(end)
    ncell = cells(w)
    line = {"metric": METRIC, "value": world * ncell * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": w.name, "cells": ncell, "driver": "steepest_descent (1 field evaluation a step)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "clocks": clk.summary(), "gpu_launches": ctx.launches() - n0}
    ctx.close()
    return line


def run_rk4(args, rank, world, dist, cayley):
    """Fixed RK4 steps (four right-hand sides each) on the workload, h = 1e-14 s."""
    import torch
    from paper_2406_16064_gb300 import mm
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    w = workload(args.workload, world)
    if w.neb:
        raise SystemExit("--driver rk4-*: the NEB workload has its own driver")
    prec = args.precision or ("f64" if args.workload == "film_relax_32" else "f32")
    ctx = mm.Context(prec, stream=stream.cuda_stream)
    for s in w.sims:
        ctx.add_sim(s.mesh, s.mat, s.Ms_cells)
    ctx.precompute()
    m0 = np.concatenate([s.m0.ravel() for s in w.sims])
    ctx.set_m(m0)
    h = 1e-14
    ctx.rk4(h, args.warmup, cayley)
    ctx.set_m(m0)
    if dist:
        dist.barrier()
    n0 = ctx.launches()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with Clocks(dev) as clk:
        start.record(stream)
        ctx.rk4(h, args.steps, cayley)
        end.record(stream)
        end.synchronize()
    ms = start.elapsed_time(end)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    m = ctx.get_m(0).reshape(3, -1)
    ncell = cells(w)
    line = {"metric": METRIC, "value": world * ncell * 4 * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": w.name, "cells": ncell, "h_s": h,
                       "driver": ("rk4 on the Cayley variable" if cayley else "rk4 with projection")
                       + " (4 right-hand sides a step)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "max_norm_error": float(np.abs(np.sqrt((m.astype(np.float64) ** 2).sum(0)) - 1).max()),
            "clocks": clk.summary(), "gpu_launches": ctx.launches() - n0}
    ctx.close()
    return line


def run_cayley_error(args, rank, world, dist):
    """The paper's macrospin comparison (Sec. "Cayley transform"): alpha = 0.05,
    H = 1e5 A/m along z, m(0) = x; max-norm error of m(1 ns) against the closed
    form for RK4 with projection and RK4 on the Cayley variable, FP64 on the GPU."""
    import torch
    import synth
    from paper_2406_16064_gb300 import mm
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    alpha, gamma, Hz, t_end = 0.05, 2.21e5, 1e5, 1e-9
    mesh = synth.Mesh(1, 1, 1, 2e-9, 2e-9, 2e-9)
    mat = synth.Material(Ms=8e5, H=(0.0, 0.0, Hz), alpha=alpha, gamma=gamma, demag=0)
    m0 = synth.uniform_state(mesh, (1.0, 0.0, 0.0))
    ph = gamma / (1 + alpha ** 2) * Hz * t_end
    exact = np.array([math.cos(ph) / math.cosh(alpha * ph), math.sin(ph) / math.cosh(alpha * ph),
                      math.tanh(alpha * ph)])
    rows = []
    for n in (250, 500, 1000, 2000, 4000, 8000):
        row = {"h_s": t_end / n, "steps": n}
        for name, cay in (("cayley", True), ("projection", False)):
            ctx = mm.Context("f64")
            ctx.add_sim(mesh, mat, None)
            ctx.precompute()
            ctx.set_m(m0.ravel())
            ctx.rk4(t_end / n, n, cay)
            row[name] = float(np.abs(ctx.get_m(0) - exact).max())
            ctx.close()
        rows.append(row)
    order = {k: math.log2(rows[0][k] / rows[1][k]) for k in ("cayley", "projection")}
    return {"metric": "macrospin max-norm error at 1 ns, RK4 with projection vs RK4 on the Cayley variable",
            "unit": "1", "higher_is_better": False, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "macrospin alpha=0.05 Hz=1e5 A/m t=1 ns"},
            "value": rows[2]["cayley"], "rows": rows, "order_coarsest": order}


def run_cufft_compare(args, rank, world, dist):
    """Timed comparison with cuFFT (through torch.fft), never on the product path: the
    zero-padded demag convolution of the workload's first simulation done the library
    way -- three 3-D R2C transforms of M on the padded grid, the symmetric tensor product
    per bin, three C2R transforms, crop -- against this library's whole right-hand side
    (mm_rhs_eval: its transforms skip the zero padding, the product is fused into the
    innermost transform, and the exchange / DMI / anisotropy / Zeeman / torque epilogue
    is included).  The cuFFT tensor spectrum is random (timing only)."""
    import torch
    from paper_2406_16064_gb300 import mm
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = workload(args.workload, world)
    prec = args.precision or "f32"
    s = w.sims[0]
    nx, ny, nz = s.mesh.nx, s.mesh.ny, s.mesh.nz
    P = (pad(nz), pad(ny), pad(nx, True))
    rdt = torch.float32 if prec == "f32" else torch.float64
    cdt = torch.complex64 if prec == "f32" else torch.complex128
    dev = "cuda"
    M = torch.tensor(s.m0 * s.mat.Ms, dtype=rdt, device=dev)
    g = torch.Generator(device=dev).manual_seed(0)
    Nk = torch.randn((6, P[0], P[1], P[2] // 2 + 1), dtype=cdt, device=dev, generator=g)

    def cufft_conv(fft_only=False):
        Mk = torch.fft.rfftn(M, s=P, dim=(1, 2, 3))
        if fft_only:
            Hk = Mk
        else:
            xx, yy, zz, xy, xz, yz = Nk
            Hk = torch.stack([xx * Mk[0] + xy * Mk[1] + xz * Mk[2],
                              xy * Mk[0] + yy * Mk[1] + yz * Mk[2],
                              xz * Mk[0] + yz * Mk[1] + zz * Mk[2]])
        return torch.fft.irfftn(Hk, s=P, dim=(1, 2, 3))[:, :nz, :ny, :nx].contiguous()

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st.record()
        for _ in range(reps):
            fn()
        en.record()
        en.synchronize()
        return st.elapsed_time(en) / reps

    reps = max(10, args.steps)
    t_conv = timed(cufft_conv, reps)
    t_fft = timed(lambda: cufft_conv(True), reps)
    del Nk
    torch.cuda.empty_cache()
    stream = torch.cuda.Stream()                 # a real stream: the context launches on it
    torch.cuda.set_stream(stream)
    ctx = mm.Context(prec, stream=stream.cuda_stream)
    ctx.add_sim(s.mesh, s.mat, s.Ms_cells)
    ctx.precompute()
    mt = torch.tensor(s.m0.ravel(), dtype=rdt, device=dev)
    kt, ht = torch.empty_like(mt), torch.empty_like(mt)
    n0 = ctx.launches()
    t_ours = timed(lambda: ctx.rhs_device(mt, kt, ht), reps)
    launches = ctx.launches() - n0
    ctx.close()
    return {"metric": "demag convolution time per evaluation: cuFFT (torch.fft) vs this library's whole RHS",
            "unit": "ms", "higher_is_better": False, "n_gpus": 1, "dtype": prec, "data": "synthetic",
            "config": {"workload": w.name, "mesh": [nx, ny, nz], "padded_grid_zyx": list(P)},
            "value": t_ours, "ours_rhs_ms": t_ours, "cufft_conv_ms": t_conv, "cufft_fft_only_ms": t_fft,
            "ours_vs_cufft_conv": t_conv / t_ours, "gpu_launches": launches}


def run_potential(args, rank, world, dist):
    """The demagnetising field through the magnetic scalar potential (mm_demag_potential:
    three forward transforms of M, one inverse of u, on a grid padded to 2^k >= 2n + 1)
    against the Newell right-hand side (mm_rhs_eval: three forward, tensor product,
    three inverse on 2^k >= 2n - 1, plus every local term and the torque) on the
    workload's first simulation; cell-updates/s of each."""
    import torch
    from paper_2406_16064_gb300 import mm
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = workload(args.workload, world)
    prec = args.precision or ("f64" if args.workload == "film_relax_32" else "f32")
    s = w.sims[0]
    rdt = torch.float32 if prec == "f32" else torch.float64
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = mm.Context(prec, stream=stream.cuda_stream)
    ctx.add_sim(s.mesh, s.mat, s.Ms_cells)
    ctx.precompute()
    mt = torch.tensor(s.m0.ravel(), dtype=rdt, device="cuda")
    a, b = torch.empty_like(mt), torch.empty_like(mt)
    ctx.demag_potential(mt, a, 0)               # first call: kernel spectrum (FP64)
    torch.cuda.synchronize()

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st.record(stream)
        for _ in range(reps):
            fn()
        en.record(stream)
        en.synchronize()
        return st.elapsed_time(en) / reps

    reps = max(10, args.steps)
    n0 = ctx.launches()
    t_pot = timed(lambda: ctx.demag_potential(mt, a, 0), reps)
    lp = (ctx.launches() - n0) / (reps + 3)
    t_newell = timed(lambda: ctx.rhs_device(mt, b, None), reps)
    n = s.mesh.ncells
    P = [1 << (2 * v).bit_length() for v in (s.mesh.nx, s.mesh.ny, s.mesh.nz)]
    ctx.close()
    return {"metric": "demag field evaluations, scalar potential vs Newell right-hand side", "unit": "cell-updates/s",
            "higher_is_better": True, "n_gpus": 1, "dtype": prec, "data": "synthetic",
            "config": {"workload": w.name, "cells": n, "potential_padded_grid_xyz": P},
            "value": n / (t_pot / 1e3), "potential_ms": t_pot, "potential_launches": lp,
            "newell_rhs_ms": t_newell, "newell_rhs_value": n / (t_newell / 1e3)}


def run_relax_compare(args, rank, world, dist):
    """Wall time to relax the workload from its start below --max-dmdt (rad/s): RK45
    (mm_relax, the workload's rtol) against steepest descent (mm_minimize)."""
    import torch
    from paper_2406_16064_gb300 import mm
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    w = workload(args.workload, world)
    prec = args.precision or ("f64" if args.workload == "film_relax_32" else "f32")
    ctx = mm.Context(prec)
    for s in w.sims:
        ctx.add_sim(s.mesh, s.mat, s.Ms_cells)
    ctx.precompute()
    m0 = np.concatenate([s.m0.ravel() for s in w.sims])
    out = {}
    for drv in ("rk45", "sd"):
        ctx.set_m(m0)
        ctx.reset_time()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if drv == "rk45":
            n = ctx.relax(w.rtol, t_end=0.0, max_dmdt=args.max_dmdt, max_steps=args.steps, sync_every=64)
            st = [ctx.status(i) for i in range(len(w.sims))]
            conv = all(x["status"] == 2 for x in st)
            rhs = 7 * n
        else:
            n, conv = ctx.minimize(args.max_dmdt, max_steps=args.steps, sync_every=16)
            rhs = n
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        E = sum(ctx.energy(i)["total"] for i in range(len(w.sims)))
        out[drv] = {"seconds": dt, "steps": n, "field_evaluations": rhs, "converged": bool(conv), "energy_J": E}
    ctx.close()
    return {"metric": "relaxation wall time below max|dm/dt|, RK45 vs steepest descent", "unit": "s",
            "higher_is_better": False, "n_gpus": world, "dtype": prec, "data": "synthetic",
            "config": {"workload": w.name, "cells": cells(w), "max_dmdt_rad_per_s": args.max_dmdt,
                       "rtol_rk45": w.rtol, "max_steps": args.steps},
            "value": out["sd"]["seconds"], "rk45": out["rk45"], "sd": out["sd"],
            "speedup": out["rk45"]["seconds"] / out["sd"]["seconds"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--workload", default="film")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--no-f64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--sweep-n", default=None, help="comma-separated N for --workload sweep")
    ap.add_argument("--driver", default="rk45",
                    help="rk45 (default), sd (steepest-descent steps), relax-compare, rk4-cayley, "
                         "rk4-proj, cayley-error, cufft-compare or potential")
    ap.add_argument("--max-dmdt", type=float, default=1e7, help="relax-compare threshold, rad/s")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the fixed tile rules instead of the autotuned (cached) tiles")
    ap.add_argument("--ext", action="store_true",
                    help="add per-cell A and D and a Zhang-Li drift to the workload (extended epilogue)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            dist.init_process_group("nccl")
        if args.driver == "sd":
            line = run_sd(args, rank, world, dist)
        elif args.driver in ("rk4-cayley", "rk4-proj"):
            line = run_rk4(args, rank, world, dist, args.driver == "rk4-cayley")
        elif args.driver == "cayley-error":
            line = run_cayley_error(args, rank, world, dist) if rank == 0 else None
        elif args.driver == "relax-compare":
            line = run_relax_compare(args, rank, world, dist) if rank == 0 else None
        elif args.driver == "cufft-compare":
            line = run_cufft_compare(args, rank, world, dist) if rank == 0 else None
        elif args.driver == "potential":
            line = run_potential(args, rank, world, dist) if rank == 0 else None
        else:
            line = (run_sweep if args.workload == "sweep" else run_gpu)(args, rank, world, dist)
        if dist:
            dist.destroy_process_group()
    if rank == 0 and line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
