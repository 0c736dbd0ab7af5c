"""CUDA-graph replay and launch-shape autotuning for the FP32 form.

``GraphSolve`` captures one rt_solve_columns of a fixed batch (memsets, the
Planck pre-kernel and the persistent solve kernel) into a CUDA graph and
replays it; the first solve runs outside capture so that the workspace and
the batch plan exist before capture.

``autotune`` times the persistent kernel's launch shapes (warps per CTA x
resident CTAs per SM) on the actual batch with CUDA events and keeps the
fastest.  Work units are 32 systems of one column whatever the shape and
each column is summed in unit order, so every candidate must give the same
bits; a candidate that does not is rejected (stability check).  Results are
cached per batch signature.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

from . import rt
from .solver import DeviceBatch, Solver

DEFAULT_CANDIDATES = [(b, c) for b in (64, 128, 192, 256) for c in (0, 2, 4)]


class GraphSolve:
    """One batch, one handle, one captured graph."""

    def __init__(self, solver: Solver, batch: DeviceBatch, stream: torch.cuda.Stream | None = None):
        self.solver, self.batch = solver, batch
        self.stream = stream or torch.cuda.Stream()
        with torch.cuda.stream(self.stream):
            solver.solve(batch, self.stream)          # plan + workspace outside capture
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            solver.solve(batch, self.stream)

    def replay(self):
        # replay() launches on the current stream; keep it on the capture stream
        with torch.cuda.stream(self.stream):
            self.graph.replay()


def signature(batch: DeviceBatch, cfg: dict) -> str:
    h = hashlib.sha1()
    h.update(batch.n_layers.tobytes())
    h.update(batch.n_bins.tobytes())
    h.update(str(batch.n_g).encode())
    h.update(json.dumps(cfg, sort_keys=True, default=str).encode())
    return h.hexdigest()[:16]


def _time(solver: Solver, batch: DeviceBatch, stream, reps: int) -> float:
    with torch.cuda.stream(stream):
        solver.solve(batch, stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            solver.solve(batch, stream)
        e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(batch: DeviceBatch, g_weights, candidates=None, reps: int = 5,
             cache_path: str | None = None, **cfg) -> dict:
    """Return {'block_threads', 'ctas_per_sm', 'ms', 'table', 'stable'}."""
    candidates = candidates or DEFAULT_CANDIDATES
    key = signature(batch, cfg)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    stream = torch.cuda.Stream()
    ref = None
    table, best = [], None
    for block, ctas in candidates:
        s = Solver(g_weights, precision=rt.RT_FP32_FORM, block_threads=block, ctas_per_sm=ctas, **cfg)
        try:
            ms = _time(s, batch, stream, reps)
            out = s.outputs(batch, stream)
            stream.synchronize()
            net = out["F_net"].cpu().numpy()
        finally:
            s.close()
        stable = True
        if ref is None:
            ref = net
        else:
            stable = bool(np.array_equal(net, ref))
        table.append(dict(block_threads=block, ctas_per_sm=ctas, ms=ms, stable=stable))
        if stable and (best is None or ms < best["ms"]):
            best = dict(block_threads=block, ctas_per_sm=ctas, ms=ms)
    res = dict(best, table=table, stable=all(t["stable"] for t in table))
    if cache_path:
        cache[key] = res
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return res
