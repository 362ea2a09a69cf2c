"""One process per GPU, each clustering its own events.

Events are independent (CLUE clusters each event, and each layer of it, on its
own: Sec. 2), so ranks share no data: there is no collective on the data path.
Two ways to give ranks their work:

* weak scaling (the benchmark's mode): every rank clusters a full batch of its
  own, drawn with rank-specific seeds, so per-GPU work is fixed as ranks grow;
* strong scaling: one global list of events split across ranks, balanced by
  hit count (greedy: largest event to the least-loaded rank).

Only the measurement crosses ranks: a barrier before and after the timed
region, the maximum of the ranks' times and the sum of their hits.
"""
from __future__ import annotations

import numpy as np


def weak_seeds(rank: int, size_seed: int = 0, first_event_seed: int = 1000):
    """Seeds of rank `rank`'s own batch (rank 0 keeps the single-GPU seeds)."""
    return size_seed + rank, first_event_seed + 100_000 * rank


def strong_split(sizes, world: int, rank: int):
    """Indices of the events rank `rank` clusters, from a global size list.
    Every event goes to exactly one rank; loads differ by at most one event."""
    sizes = np.asarray(sizes, np.int64)
    load = np.zeros(world, np.int64)
    owner = np.empty(sizes.size, np.int64)
    for i in np.argsort(-sizes, kind="stable"):
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += sizes[i]
    return np.nonzero(owner == rank)[0]


def reduce_timing(ms_local: float, hits_local: int, dist=None):
    """(max ms over ranks, total hits over ranks); identity without `dist`."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms_local), int(hits_local)
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64)
    h = torch.tensor([int(hits_local)], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(h, op=dist.ReduceOp.SUM)
    return float(t.item()), int(h.item())
