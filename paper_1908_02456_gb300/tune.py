"""Autotuner for the kernels' launch-time knobs.

The one-orbital complex64 contraction streams the boundary tiles once per Horner
stage.  When the tiles are about the size of L2, keeping a leading part of them in
L2 (evict_last) lets the next stage read that part from L2 instead of HBM; how much
to keep depends on the grid and the device.  ``tune(ctx, ...)`` times short
``abc_run`` calls for a few candidate values on a copy of the caller's state, sets
the fastest on the context and caches the choice in a JSON file keyed by the
problem shape and the device name.  Tuning is set-up work: callers run it before
any timed region.
"""
from __future__ import annotations

import json
import os
from typing import Optional

from . import abc

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "tune_cache.json")


def _key(ctx: abc.Context, n_orb: int, device_name: str) -> str:
    return f"{device_name}|{ctx.shape}|h={ctx.h}|order={ctx.order}|prec={ctx.precision}|b={n_orb}"


def _load():
    try:
        return json.load(open(CACHE))
    except (OSError, ValueError):
        return {}


def _save(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, CACHE)


def candidates(n_tiles: int):
    """Candidate evict_last tile counts: none, fractions of the tile set, and all."""
    fr = [0.0, 0.3, 0.45, 0.55, 0.65, 0.75, 0.85, 1.0]
    return sorted({int(round(f * n_tiles)) for f in fr})


def tune(ctx: abc.Context, psi, aux, V, dt: float, steps: int = 40, repeats: int = 2,
         use_cache: bool = True, device_name: Optional[str] = None) -> dict:
    """Pick ABC_TUNE_L2_KEEP_TILES for this context; returns {"keep": k, "ms_per_step": t, ...}."""
    import torch
    n_orb = psi.shape[0]
    n_tiles = ctx.get_tuning(abc.TUNE_TILE_COUNT)
    if n_tiles == 0 or n_orb != 1:
        return {"keep": 0, "tuned": False, "reason": "no tiled contraction for this context"}
    name = device_name or torch.cuda.get_device_name()
    key = _key(ctx, n_orb, name)
    cache = _load() if use_cache else {}
    if key in cache:
        ctx.set_tuning(abc.TUNE_L2_KEEP_TILES, cache[key]["keep"])
        return dict(cache[key], cached=True)
    p, a = psi.clone(), (aux.clone() if aux is not None else None)
    results = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for keep in candidates(n_tiles):
        ctx.set_tuning(abc.TUNE_L2_KEEP_TILES, keep)
        ctx.run(p, a, V, dt, 3)                     # capture + warm
        best = float("inf")
        for _ in range(repeats):
            torch.cuda.synchronize()
            e0.record()
            ctx.run(p, a, V, dt, steps)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / steps)
        results[keep] = best
    keep = min(results, key=results.get)
    ctx.set_tuning(abc.TUNE_L2_KEEP_TILES, keep)
    out = {"keep": keep, "ms_per_step": results[keep], "tiles": n_tiles,
           "sweep": {str(k): round(v, 5) for k, v in sorted(results.items())}, "tuned": True}
    if use_cache:
        cache = _load()
        cache[key] = out
        _save(cache)
    return dict(out, cached=False)
