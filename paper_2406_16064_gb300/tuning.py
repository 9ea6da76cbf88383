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


def key(gpu, precision, mesh):
    return f"{gpu}|{build_id()}|{precision}|{mesh.nx}x{mesh.ny}x{mesh.nz}"


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
    mesh) the autotuned tiles of its mesh: from the cache when it has them, else by
    mm_autotune (which sets them on every simulation with that mesh), then cached.
    Returns {mesh key: entry} with the tuning, its ms per attempt and the rule's."""
    cache = load(path)
    out, seen = {}, set()
    changed = False
    for i, m in enumerate(meshes):
        k = key(gpu, ctx.precision, m)
        if k in seen:
            continue
        seen.add(k)
        if k in cache and not retune:
            for j, mj in enumerate(meshes):
                if (mj.nx, mj.ny, mj.nz) == (m.nx, m.ny, m.nz):
                    ctx.set_tuning(j, cache[k]["tuning"])
            out[k] = dict(cache[k], cached=True)
            continue
        t, best, rule = ctx.autotune(i, reps)
        for j, mj in enumerate(meshes):   # same cells, other cell sizes: same tiles
            if (mj.nx, mj.ny, mj.nz) == (m.nx, m.ny, m.nz):
                ctx.set_tuning(j, t)
        cache[k] = {"tuning": t, "ms_per_attempt": best, "rule_ms_per_attempt": rule}
        out[k] = dict(cache[k], cached=False)
        changed = True
    if changed:
        save(cache, path)
    return out
