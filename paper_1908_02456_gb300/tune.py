"""Autotuner for the kernels' per-shape launch choices.

The fastest form of a time step depends on the grid, the orbital count, the
precision and the device, so the library exposes its choices as tuning knobs
(``abc_set_tuning``) and this module picks them by timing:

* the tensor-core GEMM's form (``TUNE_GEMM_TILE``: 96-column tiles with one CTA per
  SM, 64-column tiles with two, or the Karatsuba form with three real products) and its
  K split count (``TUNE_GEMM_SPLIT``: automatic, or 1, 2 splits per output tile);
* the interior stencil of an order-1 step: the four Horner stages fused in time
  (``TUNE_FUSED``) or stage by stage, and for the latter where the stencil runs
  beside the boundary chain (``TUNE_STENCIL``), how many planes each of its threads
  marches through (``TUNE_STENCIL_KZ``) and whether its planes are staged in shared
  memory by bulk copies (``TUNE_STENCIL_STAGED``);
* the order-1 back transform one, two or four orbitals per cell group
  (``TUNE_BACK_MULTI``), the four-orbital forward transform's reflection transform
  across lanes or in registers (``TUNE_FORWARD_RW``), whether it reads w on Gamma from
  the copy the previous stage's stencil wrote (``TUNE_GAMMA_COPY``), and, on the
  tensor-core path with a multiple of 32 orbitals, the node-major chain with both
  transforms one warp per cell and 32 orbitals (``TUNE_LANES``);
* for one complex64 orbital, the early start of the tiled contraction behind the
  forward transform (``TUNE_PDL``).

``tune(ctx, psi, aux, V, dt, ...)`` times short ``abc_run`` calls on a copy of the
caller's state, one knob group after the other (GEMM first, then the stencil form),
keeps the fastest setting on the context, and caches the choice in a JSON file keyed
by the device name and the problem shape.  Tuning is set-up work: callers run it
before any timed region.  Every setting computes the same step up to FP32 rounding.
"""
from __future__ import annotations

import json
import os
from typing import Optional

from . import abc

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "tune_cache.json")


def _key(ctx: abc.Context, n_orb: int, device_name: str, meanfield) -> str:
    return (f"{device_name}|{ctx.shape}|h={ctx.h}|order={ctx.order}|prec={ctx.precision}|fit={ctx.fit1}"
            f"|b={n_orb}|mf={meanfield is not None}")


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


def knob_groups(ctx: abc.Context, n_orb: int):
    """The candidate settings, as groups of {knob: value} dicts searched one group at a time."""
    groups = []
    tc = ctx.precision in (abc.C64_3XTF32, abc.C64_SPLIT_FP16) and n_orb >= 2 and ctx.order < 2 \
        and ctx.fit1 == abc.FIT1_LIMIT
    if tc:
        groups.append([{abc.TUNE_GEMM_TILE: t, abc.TUNE_GEMM_SPLIT: sp} for t in (0, 1, 2) for sp in (0, 1, 2)])
    if ctx.order == 1 and ctx.precision != abc.FP64:
        nx = ctx.shape[0]
        st = {abc.TUNE_STENCIL_STAGED: 0}
        stencil = [{abc.TUNE_FUSED: 0, abc.TUNE_STENCIL: m, abc.TUNE_STENCIL_KZ: 0, **st} for m in (0, 1, 2)]
        if nx % 2 == 0 and ctx.radius == 1 and n_orb >= 2:
            stencil += [{abc.TUNE_FUSED: 0, abc.TUNE_STENCIL: 0, abc.TUNE_STENCIL_KZ: kz, **st} for kz in (1, 2, 4, 8)]
            if nx <= 256:
                stencil.append({abc.TUNE_FUSED: 0, abc.TUNE_STENCIL: 0, abc.TUNE_STENCIL_KZ: 1,
                                abc.TUNE_STENCIL_STAGED: 1})
        if nx % 2 == 0 and min(ctx.shape) >= 8 and ctx.radius == 1:
            # abc_step and the adjoint still step stage by stage: the library's default form
            stencil.append({abc.TUNE_FUSED: 1, abc.TUNE_STENCIL: 0,
                            abc.TUNE_STENCIL_KZ: 1 if n_orb >= 2 else 0, **st})
        groups.append(stencil)
    if ctx.order == 1 and ctx.fit1 == abc.FIT1_LIMIT and n_orb >= 2 and n_orb % 2 == 0:
        groups.append([{abc.TUNE_BACK_MULTI: m} for m in ((0, 1, 2) if n_orb % 4 == 0 else (0, 2))])
    if n_orb >= 4 and n_orb % 4 == 0 and ctx.order < 2:
        lanes = tc and ctx.order == 1 and n_orb % 32 == 0
        ln = {abc.TUNE_LANES: 0} if lanes else {}
        if ctx.precision != abc.FP64 and ctx.radius == 1 and ctx.shape[0] % 2 == 0:
            fwd = [{abc.TUNE_FORWARD_RW: rw, abc.TUNE_GAMMA_COPY: gc, **ln} for gc in (0, 1) for rw in (0, 1)]
            if lanes:
                fwd += [{abc.TUNE_FORWARD_RW: 0, abc.TUNE_GAMMA_COPY: gc, abc.TUNE_LANES: ln}
                        for gc in (0, 1) for ln in (1, 2, 3, 4, 5)]
        else:
            fwd = [{abc.TUNE_FORWARD_RW: 0, **ln}, {abc.TUNE_FORWARD_RW: 1, **ln}]
            if lanes:
                fwd += [{abc.TUNE_FORWARD_RW: 0, abc.TUNE_LANES: ln} for ln in (1, 2, 3, 4, 5)]
        groups.append(fwd)
    if n_orb == 1 and ctx.precision != abc.FP64 and ctx.get_tuning(abc.TUNE_TILE_COUNT) > 0:
        groups.append([{abc.TUNE_PDL: 1}, {abc.TUNE_PDL: 0}])
    return groups


def _apply(ctx, setting):
    for k, v in setting.items():
        ctx.set_tuning(k, v)


def tune(ctx: abc.Context, psi, aux, V, dt: float, meanfield=None, steps: int = 8, repeats: int = 2,
         use_cache: bool = True, device_name: Optional[str] = None, fresh: Optional[dict] = None) -> dict:
    """Pick the knobs for this context and orbital count; returns the chosen setting,
    its step time and the sweep.  With `fresh` (a result of an uncached call) the
    result is only stored in the cache."""
    import torch
    n_orb = psi.shape[0]
    name = device_name or torch.cuda.get_device_name()
    key = _key(ctx, n_orb, name, meanfield)
    if fresh is not None:
        cache = _load()
        cache[key] = {k: v for k, v in fresh.items() if k != "cached"}
        _save(cache)
        return fresh
    if use_cache:
        cache = _load()
        if key in cache:
            setting = {int(k): v for k, v in cache[key]["setting"].items()}
            _apply(ctx, setting)
            return dict(cache[key], cached=True)
    p, a = psi.clone(), (aux.clone() if aux is not None else None)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def time_setting(setting):
        _apply(ctx, setting)
        ctx.run(p, a, V, dt, 2, meanfield=meanfield)        # capture + warm
        best = float("inf")
        for _ in range(repeats):
            torch.cuda.synchronize()
            e0.record()
            ctx.run(p, a, V, dt, steps, meanfield=meanfield)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / steps)
        return best

    chosen, sweep = {}, {}
    for group in knob_groups(ctx, n_orb):
        times = []
        for cand in group:
            setting = {**chosen, **cand}
            t = time_setting(setting)
            sweep[json.dumps({str(k): v for k, v in sorted(setting.items())})] = round(t, 5)
            times.append((t, cand))
        best = min(times, key=lambda x: x[0])
        chosen.update(best[1])
    _apply(ctx, chosen)
    ms = time_setting(chosen) if chosen else None
    out = {"setting": {str(k): v for k, v in sorted(chosen.items())}, "ms_per_step": ms, "sweep": sweep,
           "tuned": True}
    if use_cache:
        cache = _load()
        cache[key] = out
        _save(cache)
    return dict(out, cached=False)


def describe(setting: dict) -> dict:
    """Readable names of a setting returned by tune()."""
    names = {abc.TUNE_GEMM_TILE: "gemm_tile(0=96 cols x 1 CTA/SM, 1=64 cols x 2 CTAs/SM, 2=Karatsuba 64 cols)",
             abc.TUNE_GEMM_SPLIT: "gemm_split(0=auto)", abc.TUNE_FUSED: "fused_stencil",
             abc.TUNE_STENCIL: "stencil_placement(0=after contraction, 1=stage start, 2=serial)",
             abc.TUNE_STENCIL_BPS: "stencil_blocks_per_sm(0=one thread per pair)",
             abc.TUNE_STENCIL_KZ: "stencil_form(0=pair per thread, 1=capped registers, k>1=k planes)",
             abc.TUNE_BACK_MULTI: "back_transform_orbitals_per_group(0=1, 1=4, 2=2)", abc.TUNE_FORWARD_RW: "forward_transform_in_registers",
             abc.TUNE_GAMMA_COPY: "forward_reads_gamma_copy", abc.TUNE_STENCIL_STAGED: "stencil_planes_staged_by_bulk_copies",
             abc.TUNE_LANES: "node_major_chain(1=warp per cell, 2/3=cell split between 2 lanes, 4/5=between 4)", abc.TUNE_PDL: "pdl"}
    return {names.get(int(k), str(k)): v for k, v in setting.items()}
