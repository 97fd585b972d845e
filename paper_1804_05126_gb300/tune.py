"""Autotuner for the batch team engine: picks the number of blocks per team by timing the real batch.

The team size trades per-request parallelism (large K: the heaviest requests finish sooner) against the
number of concurrently running requests (small K: more teams).  The best value depends on the mix of
sizes and stiffness, so it is measured: every candidate runs the batch once (after one warm-up run) with
CUDA events on the solver's stream, and the fastest is kept in a cache keyed by the batch's signature.
"""
from __future__ import annotations

import json
import os
import threading

import numpy as np

_cache: dict[str, int] = {}
_lock = threading.Lock()


def signature(items) -> str:
    """Batch class: operator kind, precision, count and size quartiles (log2 of N)."""
    kinds = sorted({it[0].desc["kind"] for it in items})
    precs = sorted({str(it[6]) for it in items})
    ns = np.array([it[0].n for it in items], dtype=np.float64)
    q = [int(round(np.log2(v))) for v in np.quantile(ns, [0.25, 0.5, 0.75, 1.0])]
    return json.dumps({"k": kinds, "p": precs, "n": len(items), "q": q}, sort_keys=True)


def tune_batch(solver, items, candidates=(1, 2, 4, 8, 16, 32, 64), cache_path: str | None = None):
    """Time the batch for each candidate team size; return (best, {k: ms}) and remember the best."""
    import torch

    key = signature(items)
    timings = {}
    stream = torch.cuda.current_stream()
    for k in candidates:
        solver.solve_batch(items, team_blocks=k)  # warm-up (workspace, code)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        solver.solve_batch(items, team_blocks=k)
        e1.record(stream)
        torch.cuda.synchronize()
        timings[k] = e0.elapsed_time(e1)
    best = min(timings, key=timings.get)
    with _lock:
        _cache[key] = best
        if cache_path:
            data = {}
            if os.path.exists(cache_path):
                with open(cache_path) as f:
                    data = json.load(f)
            data[key] = best
            with open(cache_path, "w") as f:
                json.dump(data, f, indent=1)
    return best, timings


def cached_team_blocks(items, cache_path: str | None = None) -> int | None:
    key = signature(items)
    with _lock:
        if key in _cache:
            return _cache[key]
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            return json.load(f).get(key)
    return None
