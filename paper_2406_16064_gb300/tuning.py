"""Cache of autotuned tile shapes and schedules (host side).

`mm_autotune` times candidate tunings of one mesh on the GPU; this module
keeps its choices in a JSON file keyed by GPU name, library build, precision
and mesh, so a later context with the same meshes sets them (`mm_set_tuning`)
without timing again.  The cache file is `$MM_TUNE_CACHE`, else
`~/.cache/paper_2406_16064_gb300/tuning.json`.
"""
from __future__ import annotations

import hashlib
import json
import os

from . import mm

_BUILD = None


def build_id():
    """First 16 hex digits of sha256(libmm.so): choices from another build are stale."""
    global _BUILD
    if _BUILD is None:
        h = hashlib.sha256()
        with open(mm.LIB_PATH, "rb") as f:
            for chunk in iter(lambda: f.read(1 << 20), b""):
                h.update(chunk)
        _BUILD = h.hexdigest()[:16]
    return _BUILD


def cache_path():
    return os.environ.get("MM_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_2406_16064_gb300", "tuning.json")


def _dims(m):
    return (m.nx, m.ny, m.nz)


def batch_signature(meshes):
    """The batch's meshes and their counts: a mesh is tuned for the launches it shares."""
    count = {}
    for m in meshes:
        count[_dims(m)] = count.get(_dims(m), 0) + 1
    return ",".join(f"{a}x{b}x{c}*{n}" for (a, b, c), n in sorted(count.items()))


def key(gpu, precision, mesh, meshes=None):
    sig = batch_signature(meshes if meshes is not None else [mesh])
    return f"{gpu}|{build_id()}|{precision}|{mesh.nx}x{mesh.ny}x{mesh.nz}|{sig}"


def load(path=None):
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(entries, path=None):
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_context(ctx, meshes, gpu, reps=8, path=None, retune=False):
    """Give every simulation of ctx (not yet precomputed; meshes[i] is simulation i's
    mesh) the autotuned tiles of its mesh: from the cache when it has every mesh of
    this batch, else by mm_autotune, one mesh after the other (each timed inside a
    copy of the whole batch), then cached.  The CTA widths act on whole launches, so
    every mesh's entry carries the widths the last tuning chose.  Returns {mesh key:
    entry} with the tuning, its ms per attempt and the starting tuning's."""
    cache = load(path)
    firsts = {}
    for i, m in enumerate(meshes):
        firsts.setdefault(_dims(m), i)
    keys = {d: key(gpu, ctx.precision, meshes[i], meshes) for d, i in firsts.items()}
    if not retune and all(k in cache for k in keys.values()):
        for j, m in enumerate(meshes):
            ctx.set_tuning(j, cache[keys[_dims(m)]]["tuning"])
        return {k: dict(cache[k], cached=True) for k in keys.values()}
    out = {}
    for d, i in firsts.items():
        t, best, rule = ctx.autotune(i, reps)
        out[keys[d]] = {"tuning": t, "ms_per_attempt": best, "rule_ms_per_attempt": rule}
    widths = {k: t[k] for k in ("x_threads", "col_threads")}
    for k in out:
        out[k]["tuning"].update(widths)
        cache[k] = dict(out[k])
    save(cache, path)
    for j, m in enumerate(meshes):             # the same values as the tuning left them
        ctx.set_tuning(j, out[keys[_dims(m)]]["tuning"])
    return {k: dict(v, cached=False) for k, v in out.items()}
