"""CUDA-graph replay and launch-shape autotuning for the FP32 form.

``GraphSolve`` captures one rt_solve_columns of a fixed batch (memsets, the
Planck pre-kernel and the persistent solve kernel) into a CUDA graph and
replays it; the first solve runs outside capture so that the workspace and
the batch plan exist before capture.

``autotune`` times the persistent kernel's variants on the actual batch with
CUDA events and keeps the fastest: warps per CTA, resident CTAs per SM,
systems per lane (one, or two on the paired FP32 instructions), where
the Planck values come from (the pre-kernel's table staged in shared memory
or read directly, or evaluated in the solve kernel) and the staging depth
(levels of elimination scratch the back-substitution has in flight through
its shared-memory ring: more hides more L2 latency, but costs resident CTAs
when tall columns already fill shared memory).  Work units are 32 x (systems per lane) systems of one column
whatever the shape, and each column is summed in unit order, so candidates
with the same systems per lane must give the same bits; one that does not
is rejected (stability check).  Across systems per lane only the rounding
order differs, and the results must agree to 1e-5 of the largest flux.
Results are cached per batch signature.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

from . import rt
from .solver import DeviceBatch, Solver

KNOBS = ("block_threads", "ctas_per_sm", "systems_per_lane", "planck_staging", "staging_depth")


# Above about this many layers a unit's staged Planck column, not the
# register file, limits the resident warps: the direct staging mode (B read
# from the pre-kernel's table, nothing staged) becomes a candidate.
TALL_COLUMN_LAYERS = 230


def default_candidates(n_g: int, max_layers: int = 0) -> list[dict]:
    staging = ((rt.RT_STAGE_SHARED, rt.RT_STAGE_DIRECT, rt.RT_STAGE_INLINE) if n_g < 8
               else (rt.RT_STAGE_SHARED, rt.RT_STAGE_DIRECT) if max_layers > TALL_COLUMN_LAYERS
               else (rt.RT_STAGE_SHARED,))
    # staging depths 2 and 3 for the (faster) two systems per lane; one
    # system per lane at the default depth
    return [dict(block_threads=b, ctas_per_sm=c, systems_per_lane=n, planck_staging=st, staging_depth=d)
            for n in (1, 2) for st in staging for b in (128, 256) for c in (0, 2)
            for d in ((2, 3) if n == 2 else (2,))]


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
    """Return the fastest stable candidate's knobs (``KNOBS``) and 'ms', with
    'table' (every candidate) and 'stable'.  ``candidates`` are dicts of
    ``KNOBS`` (missing ones take the library defaults)."""
    candidates = candidates or default_candidates(batch.n_g, int(np.max(batch.n_layers)))
    key = signature(batch, dict(cfg, candidates=candidates))
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    stream = torch.cuda.Stream()
    ref = {}                       # first result per systems-per-lane
    table, best = [], None
    for cand in candidates:
        knobs = {k: cand[k] for k in KNOBS if k in cand}
        s = Solver(g_weights, precision=rt.RT_FP32_FORM, **knobs, **cfg)
        try:
            ms = _time(s, batch, stream, reps)
            out = s.outputs(batch, stream)
            stream.synchronize()
            net = out["F_net"].cpu().numpy()
        finally:
            s.close()
        spl = knobs.get("systems_per_lane", 0)
        if spl not in ref:
            ref[spl] = net
            first = next(iter(ref.values()))
            scale = max(float(np.abs(first).max()), 1e-30)
            stable = bool(np.max(np.abs(net - first)) <= 1e-5 * scale)
        else:
            stable = bool(np.array_equal(net, ref[spl]))
        table.append(dict(knobs, ms=ms, stable=stable))
        if stable and (best is None or ms < best["ms"]):
            best = dict(knobs, ms=ms)
    res = dict(best, table=table, stable=all(t["stable"] for t in table))
    if cache_path:
        cache[key] = res
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return res
