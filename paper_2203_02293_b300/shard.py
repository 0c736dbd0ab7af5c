"""Column sharding across ranks (one GPU per rank).

Every (column, bin, g) system is independent and the only coupling is the
sum over a column's own systems, so a batch splits by column with no
exchange on the data path.  ``partition`` cuts the columns into contiguous
blocks of nearly equal cost (layers x bins); each rank solves its block and
owns the matching slice of the outputs.  Collectives are used only to time
(max over ranks) and, optionally, to gather results for checking.
"""
from __future__ import annotations

import numpy as np


def partition(n_layers, n_bins, world: int) -> list[tuple[int, int]]:
    """Contiguous [start, stop) column ranges, one per rank, balanced by cost."""
    cost = np.asarray(n_layers, np.int64) * np.asarray(n_bins, np.int64)
    n = cost.size
    if world < 1:
        raise ValueError("world must be >= 1")
    cum = np.concatenate([[0], np.cumsum(cost)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        cuts.append(int(np.clip(np.searchsorted(cum, target, side="left"), cuts[-1], n)))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """Largest value of x over all ranks (the step time of a synchronous job)."""
    if dist is None or not dist.is_initialized():
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
