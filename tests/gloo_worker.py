"""Rank body for the world-size-2 gloo tests (spawned; importable by name).

Each rank plays one GPU of a sharded global count: it takes its cost-balanced
contiguous edge range, forms that range's undivided per-configuration sums
(here from the oracle's per-edge graphlet rows, since the CPU has no device),
joins the one sum-reduce, and finalizes.  Everything but the per-edge rows is
the host logic the multi-GPU path runs.
"""
from __future__ import annotations

import os

import numpy as np


def undivided_sums(rows, eu, ev, types, L):
    """Sum per-edge graphlet rows into the global histogram layout, undivided."""
    from tests.layout import colex_index, global_blocks, pairs

    blocks, total = global_blocks(L, 4)
    off = {h: o for h, _, o in blocks}
    idx = {s: colex_index(L, s) for s in (2, 3, 4)}
    P = pairs(L)
    out = np.zeros(total, np.uint64)
    for row, a, b in zip(rows, eu, ev):
        ti, tj = int(types[a]), int(types[b])
        out[off[0] + idx[2][tuple(sorted((ti, tj)))]] += np.uint64(1)
        for t in range(L):
            for h, base in ((1, 0), (2, L)):
                v = row[base + t]
                if v:
                    out[off[h] + idx[3][tuple(sorted((ti, tj, t)))]] += v
        for h in range(3, 9):
            base = 2 * L + (h - 3) * len(P)
            for p, (t, u) in enumerate(P):
                v = row[base + p]
                if v:
                    out[off[h] + idx[4][tuple(sorted((ti, tj, t, u)))]] += v
    return out


def rank_main(rank, world, port, graph_seed, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist

    import oracle
    import paper_1901_10026_gb300 as tg
    from paper_1901_10026_gb300 import dist as tgdist
    from paper_1901_10026_gb300 import synth

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        G = synth.er_1000(seed=graph_seed)
        og = oracle.OracleGraph.from_edges(G)
        eu, ev = og.edges()
        ranges = tgdist.shard_ranges(tgdist.edge_costs(G.n, eu, ev), world)
        a, b = ranges[rank]
        rows = og.per_edge(k=4, level="graphlet", edges=np.arange(a, b))
        sums = undivided_sums(rows, eu[a:b], ev[a:b], G.types, G.L)
        t = torch.from_numpy(sums.view(np.int64).copy())
        tgdist.allreduce_sums(t)
        final = tg.tg_global_finalize(G.L, 4, t.numpy().view(np.uint64))
        want = og.global_counts(k=4)
        results.put((rank, a, b, bool(np.array_equal(final, want)), int(sums.sum() > 0)))
    finally:
        dist.destroy_process_group()
