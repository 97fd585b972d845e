"""Autotuners of the engines' launch shapes, picked by timing the real work.

* Batch team engine: the number of blocks per team trades per-request parallelism (large K: the heaviest
  requests finish sooner) against the number of concurrently running requests (small K: more teams).
* Single solves on the grid engine: the tile shape of the 2D stencil step (the staged several-tiles path
  and the per-element one), the block size and the shared-memory extras.

The best value depends on the operator, its size and the precision, so it is measured: every candidate runs
the work after a warm-up run, timed with CUDA events on the solver's stream, and the fastest is kept in a
cache keyed by the work's signature.  Shape settings change results only through the order in which partial
sums are added.
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


# ---------------------------------------------------------------- single solves (grid engine launch shapes)
_solve_cache: dict[str, dict] = {}


def solve_signature(op, precision: str, p: int, m_o: int) -> str:
    """Solve class: operator kind and grid (or size), species, boundary, precision, p and m_o."""
    d = op.desc
    dims = [int(d["n"])] if d["kind"] == "csr" else [int(d.get(k, 1)) for k in ("nx", "ny", "nz")]
    return json.dumps({"k": d["kind"], "dims": dims, "ns": int(d.get("nspecies", 1)), "bc": str(d.get("bc", d.get("periodic"))),
                       "prec": precision, "p": p, "m_o": m_o}, sort_keys=True)


def solve_candidates(op, precision: str) -> list[dict]:
    """Launch shapes worth timing for this operator (configuration fields of kiops_config)."""
    kind = op.desc["kind"]
    if kind == "stencil2d":
        cands = [dict(tma=2 if precision == "fp64" else 1, tile_w=w, tile_h=h)
                 for (w, h) in ((32, 16), (64, 8), (16, 32), (128, 4))]
        cands.append(dict(tma=0, tile_w=0, tile_h=0))  # per-element several-tiles path / one-tile extras
        if precision == "fp64":
            cands += [dict(tma=0, tile_w=0, tile_h=0, block_threads=b) for b in (256, 512)]
        return cands
    return [dict(block_threads=b) for b in (0, 256, 512)] if precision == "fp64" else [dict(block_threads=0)]


def time_solve(solver, op, tau, b, tol, precision="fp64", m_init=10, m_o=2, reps=2) -> float:
    """Best of `reps` event-timed solves (ms) after one warm-up solve, on the solver's stream."""
    import torch

    solver.solve(op, tau, b, tol, m_init=m_init, m_o=m_o, precision=precision)
    stream = torch.cuda.current_stream()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        solver.solve(op, tau, b, tol, m_init=m_init, m_o=m_o, precision=precision)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_solve(solver, op, tau, b, tol, precision="fp64", m_init=10, m_o=2, candidates=None, reps=2,
               cache_path: str | None = None):
    """Time every candidate launch shape on this solve, keep the fastest on the solver and in the cache.
    Returns (best candidate, {candidate as json: ms})."""
    p = b.shape[0] - 1
    cands = candidates if candidates is not None else solve_candidates(op, precision)
    timings = {}
    base = {k: getattr(solver.cfg, k) for k in ("tma", "tile_w", "tile_h", "block_threads")}
    for cand in cands:
        solver.configure(**{**base, **cand})
        timings[json.dumps(cand, sort_keys=True)] = time_solve(solver, op, tau, b, tol, precision, m_init, m_o, reps)
    best = json.loads(min(timings, key=timings.get))
    solver.configure(**{**base, **best})
    key = solve_signature(op, precision, p, m_o)
    with _lock:
        _solve_cache[key] = best
        if cache_path:
            data = {}
            if os.path.exists(cache_path):
                with open(cache_path) as f:
                    data = json.load(f)
            data[key] = best
            with open(cache_path, "w") as f:
                json.dump(data, f, indent=1)
    return best, timings


def cached_solve_config(op, precision: str, p: int, m_o: int, cache_path: str | None = None) -> dict | None:
    key = solve_signature(op, precision, p, m_o)
    with _lock:
        if key in _solve_cache:
            return _solve_cache[key]
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            return json.load(f).get(key)
    return None
