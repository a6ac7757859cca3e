"""Autotuner for the batched advection launch.

The persistent batched kernel runs ``blocks_per_sm`` resident blocks per SM
(grid = #SM x blocks_per_sm).  The best value depends on the batch's mix of
dimensions, levels, CFL numbers and substeps, so it is measured: every
candidate is timed with CUDA events on the current stream and the fastest is
kept, optionally in a JSON cache keyed by the batch's signature.
"""
from __future__ import annotations

import json
import os

import torch

from .elm import Batch

CANDIDATES = (1, 2, 3, 4, 5, 6, 8)


def signature(meshes, n_sub) -> str:
    parts = [f"{meshes[0].precision}"] + sorted(f"{m.dim}:{m.level}:{m.macros.shape[0]}:{s}" for m, s in zip(meshes, n_sub))
    return "|".join(parts)


def tune_batch(meshes, T_old, T_new, dt, n_sub, candidates=CANDIDATES, reps: int = 5,
               cache_path: str | None = None) -> dict:
    """Returns {"blocks_per_sm": best, "ms": {candidate: median ms}}."""
    key = signature(meshes, n_sub)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    times = {}
    for bps in candidates:
        b = Batch(meshes, bps)
        b.advect(T_old, T_new, dt, n_sub)  # warm-up
        ev = []
        for _ in range(reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            b.advect(T_old, T_new, dt, n_sub)
            e.record()
            ev.append((s, e))
        torch.cuda.synchronize()
        ms = sorted(s.elapsed_time(e) for s, e in ev)
        times[bps] = ms[len(ms) // 2]
        del b
    best = min(times, key=times.get)
    result = {"blocks_per_sm": best, "ms": {str(k): v for k, v in times.items()}}
    if cache_path:
        cache[key] = result
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return result
