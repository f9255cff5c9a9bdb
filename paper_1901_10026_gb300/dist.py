"""Sharding one graph's global count across ranks.

The global count is a sum over edges (Sec. "Global Typed Graphlet Counts";
Sec. "Parallelization": each worker holds the graph and counts its own
edges), so every rank forms undivided per-configuration sums of its share and
the ranks add them; the division by |E(H)| happens once, after the sum.  The
only exchange is that one sum-reduce of a histogram of ``tg_global_len(L, k)``
entries.  On the GPU a rank's share is ``tg_count_shard(g, k, rank, world)``
(a cost-balanced slice of the per-edge pass plus its share of the whole-graph
4-cycle and 4-clique enumerations); the contiguous edge ranges below are the
same decomposition for per-edge counters (``tg_count_range``) and for the CPU
tests.

Host logic only (no counting here); the device work is the library's.
"""
from __future__ import annotations

import numpy as np


def edge_costs(n: int, eu: np.ndarray, ev: np.ndarray) -> np.ndarray:
    """Work estimate per canonical edge: endpoint degrees plus a constant."""
    deg = np.bincount(np.concatenate([eu, ev]), minlength=n).astype(np.float64)
    return deg[eu] + deg[ev] + 64.0


def shard_ranges(costs: np.ndarray, world: int):
    """Split [0, M) into `world` contiguous ranges of roughly equal cost."""
    M = int(costs.shape[0])
    if world <= 1 or M == 0:
        return [(0, M)] + [(M, M)] * max(0, world - 1)
    cum = np.cumsum(costs)
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(cum, total * r / world, side="left")) + 1)
    cuts.append(M)
    cuts = np.maximum.accumulate(np.clip(np.array(cuts), 0, M))
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


def allreduce_sums(sums, group=None):
    """Sum per-rank undivided histograms in place (torch tensor, int64 view)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    return sums
