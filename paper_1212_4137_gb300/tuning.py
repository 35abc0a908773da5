"""Tile shapes of the grouped contraction (k_gemm_grouped), chosen by measurement.

The grouped solve runs v = A^T y of all its problems, and the dense u = A x of their first sweep,
as one persistent tensor-core launch over 128 x N tiles with an S-stage load pipeline.  The best
(N, S) depends on how many starts the problems carry (N tiles of 64 waste less on 16 starts; 128
halves the P-operand traffic per flop on 256) and on the problems' sizes.  ``tune`` times every
shape the library builds on a group solve and returns the measurements; ``bench.py --tune`` runs it
on problem mixes drawn like the batching configuration, one per bucket of start counts, and writes
the table ``grouped_tiles.json`` beside this file (the measurements and the choice per bucket).
``choose`` reads that table; without it, or for a bucket it lacks, the library's default applies.
"""
from __future__ import annotations

import json
import os
import time

TILE_SHAPES = ((64, 2), (64, 3), (64, 4), (128, 2), (128, 3))
TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "grouped_tiles.json")


def bucket(r_max: int) -> str:
    """The bucket of a group by its largest start count."""
    for lim in (16, 64, 256):
        if r_max <= lim:
            return f"r<={lim}"
    return "r>256"


def tune(group, problems, reps: int = 2, shapes=TILE_SHAPES) -> dict:
    """Time spca_solve_group on `problems` (the argument of Group.solve) for each tile shape:
    {"N,S": best of `reps` wall-clock ms after one warm-up}, and the fastest shape."""
    import torch
    ms = {}
    for shape in shapes:
        group.solve(problems, tiles=shape)   # warm-up: captures the shape's graphs
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            group.solve(problems, tiles=shape)
            dt = 1e3 * (time.perf_counter() - t0)
            best = dt if best is None or dt < best else best
        ms[f"{shape[0]},{shape[1]}"] = round(best, 3)
    choice = min(ms, key=ms.get)
    return {"ms": ms, "choice": [int(t) for t in choice.split(",")]}


def load_table(path: str = TABLE) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def choose(r_max: int, table: dict | None = None):
    """The measured shape for a group whose largest start count is r_max, or None (the library's
    default)."""
    table = load_table() if table is None else table
    entry = table.get("buckets", {}).get(bucket(r_max))
    return tuple(entry["choice"]) if entry else None
