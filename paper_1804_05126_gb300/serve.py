"""Serving loop: replay a timed request stream through the continuous-batching server and report
latency percentiles and throughput.

Requests are released at their arrival times (busy wait on a monotonic clock), submitted to the server
(which admits them against the HBM budget as slots and memory free up) and polled until done; latency is
completion time minus arrival time as seen by this host thread.
"""
from __future__ import annotations

import time

import numpy as np


def run_stream(solver, stream, precision_of=lambda P: P.precision, poll_slice_s: float = 0.0):
    """stream: list of (t_arrival_s, Problem).  Returns dict with per-request latency, results and stats."""
    import torch

    ops = [solver.operator(P.op) for _, P in stream]
    bs = [torch.as_tensor(P.b, device=solver.device) for _, P in stream]
    torch.cuda.synchronize()
    start = time.perf_counter()
    submitted = {}  # ticket -> index
    done_at = [None] * len(stream)
    stats = [None] * len(stream)
    ws = [None] * len(stream)
    nxt = 0
    while nxt < len(stream) or submitted:
        now = time.perf_counter() - start
        while nxt < len(stream) and stream[nxt][0] <= now:
            _, P = stream[nxt]
            t, w = solver.submit(ops[nxt], P.tau, bs[nxt], P.tol, P.m_init, P.m_o, precision_of(P))
            submitted[t] = nxt
            ws[nxt] = w
            nxt += 1
        for t in list(submitted):
            ok, st = solver.poll(t, poll_slice_s)
            if ok:
                i = submitted.pop(t)
                done_at[i] = time.perf_counter() - start
                stats[i] = st
    elapsed = time.perf_counter() - start
    lat = np.array([done_at[i] - stream[i][0] for i in range(len(stream))])
    return {"latency_s": lat, "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "elapsed_s": elapsed, "solves_per_s": len(stream) / elapsed, "w": ws, "stats": stats}
