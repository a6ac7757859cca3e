"""Autotuner for the batched advection launch.

The persistent batched kernel has two launch-shape knobs: ``blocks_per_sm``
resident blocks per SM (grid = #SM x blocks_per_sm; 8 or more also selects
the kernel compiled for an 8-block register budget, fewer the 6-block one)
and ``chunks_per_item``, the tile a block takes per fetch from the shared
work list (that many consecutive 128-node chunks of one instance: larger
tiles mean fewer atomic fetches and block-wide barriers, smaller ones a
finer balance at the end of the launch).  The best shape depends on the
batch's mix of dimensions, levels, CFL numbers and substeps, so it is
measured: every candidate is timed with CUDA events on the current stream and
the fastest is kept, optionally in a JSON cache keyed by the batch's
signature.
"""
from __future__ import annotations

import json
import os

import torch

from .elm import Batch

BLOCKS_PER_SM = (2, 4, 6, 8)
CHUNKS_PER_ITEM = (1, 2, 4)


def signature(meshes, n_sub) -> str:
    parts = [f"{meshes[0].precision}"] + sorted(f"{m.dim}:{m.level}:{m.macros.shape[0]}:{s}" for m, s in zip(meshes, n_sub))
    return "|".join(parts)


def tune_batch(meshes, T_old, T_new, dt, n_sub, blocks_per_sm=BLOCKS_PER_SM, chunks_per_item=CHUNKS_PER_ITEM,
               reps: int = 5, cache_path: str | None = None) -> dict:
    """Returns {"blocks_per_sm": b, "chunks_per_item": c, "ms": {"b:c": median ms}}."""
    key = signature(meshes, n_sub)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    times = {}
    for bps in blocks_per_sm:
        for cpi in chunks_per_item:
            b = Batch(meshes, bps, cpi)
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
            times[(bps, cpi)] = ms[len(ms) // 2]
            del b
    best = min(times, key=times.get)
    result = {"blocks_per_sm": best[0], "chunks_per_item": best[1],
              "ms": {f"{k[0]}:{k[1]}": v for k, v in times.items()}}
    if cache_path:
        cache[key] = result
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return result
