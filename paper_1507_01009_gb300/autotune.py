"""Autotuner for the walk's launch parameters.

For a given system (stars on the device, optional member offsets) it times
one tree build plus one tree walk through the C ABI for every combination of
walk group size G, leaf size n_leaf and interaction tile, and picks the
fastest. Results are cached in a JSON file keyed by GPU, total stars (power
of two bucket), member count (power of two bucket), theta and quadrupole
order, so a later run with a similar workload reuses the choice without
measuring.

Accuracy is set by theta (the opening test); G and n_leaf change which
cells a group opens and therefore the error slightly, never beyond the
opening-angle bound, so the tuner only minimises time.
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import rv

GRID_GROUP = (64, 32, 16)
GRID_LEAF = (8, 16, 32, 64)
GRID_TILE = (32, 64, 96, 128, 256)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
_LOCK = threading.Lock()


def bucket(n: int) -> int:
    """Power-of-two bucket of a positive count (0 for 0)."""
    return 0 if n <= 0 else int(math.ceil(math.log2(n)))


def cache_key(gpu: str, n: int, members: int, theta: float, quadrupole: bool) -> str:
    return f"{gpu}|n2^{bucket(n)}|m2^{bucket(members)}|theta{float(theta):.4f}|q{int(bool(quadrupole))}"


def candidates(groups=GRID_GROUP, leaves=GRID_LEAF, tiles=GRID_TILE):
    return [dict(group=g, n_leaf=l, tile=t) for g in groups for l in leaves for t in tiles]


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def measure(x, y, z, m, offsets, theta, eps_star, quadrupole, cfg, reps=3):
    """Median milliseconds of build and walk for one configuration."""
    import numpy as np
    import torch
    n = int(x.shape[0])
    ctx = rv.Context(n, theta=theta, eps_star=eps_star, quadrupole=quadrupole, **cfg)
    out = [torch.empty(n, dtype=torch.float32, device=x.device) for _ in range(4)]
    off = [0, n] if offsets is None else offsets

    def once():
        ctx.build_tree_members(off, x, y, z, m)
        ctx.tree_forces_members(out=out)

    once()
    torch.cuda.synchronize()
    tb, tw = [], []
    for _ in range(reps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        ctx.build_tree_members(off, x, y, z, m)
        e1.record()
        ctx.tree_forces_members(out=out)
        e2.record()
        e2.synchronize()
        tb.append(e0.elapsed_time(e1))
        tw.append(e1.elapsed_time(e2))
    ctx.sync_status()
    p2p, m2p = ctx.walk_stats()
    return {"build_ms": float(np.median(tb)), "walk_ms": float(np.median(tw)),
            "total_ms": float(np.median(tb) + np.median(tw)), "p2p_per_star": p2p / max(n, 1),
            "m2p_per_star": m2p / max(n, 1)}


def autotune(x, y, z, m, offsets=None, theta=0.5, eps_star=0.01, quadrupole=True, grid=None, reps=3,
             cache_path: str | None = DEFAULT_CACHE, force=False):
    """Fastest (group, n_leaf, tile) for this system. Returns
    {"config": {...}, "table": [...], "cached": bool}."""
    import torch
    n = int(x.shape[0])
    members = 1 if offsets is None else len(offsets) - 1
    key = cache_key(torch.cuda.get_device_name(x.device), n, members, theta, quadrupole)
    with _LOCK:
        cache = load_cache(cache_path) if cache_path else {}
        if not force and key in cache:
            return {"config": cache[key]["config"], "table": cache[key]["table"], "cached": True}
        table = []
        for cfg in (grid or candidates()):
            r = measure(x, y, z, m, offsets, theta, eps_star, quadrupole, cfg, reps)
            table.append({**cfg, **r})
        best = min(table, key=lambda r: r["total_ms"])
        cfg = {k: best[k] for k in ("group", "n_leaf", "tile")}
        if cache_path:
            cache[key] = {"config": cfg, "table": table}
            save_cache(cache, cache_path)
        return {"config": cfg, "table": table, "cached": False}
