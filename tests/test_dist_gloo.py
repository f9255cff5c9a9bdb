"""The sharded (N > 1) path on CPU: world-size-2 gloo ranks, cost-balanced
edge ranges, one sum-reduce of undivided sums, finalize = the oracle's global
counts.  No GPU; the per-range sums come from the oracle."""
import multiprocessing as mp
import socket

import numpy as np
import pytest

from paper_1901_10026_gb300 import dist as tgdist


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_ranges_partition_the_edges():
    g = np.random.default_rng(7)
    for M, world in ((0, 2), (1, 2), (5, 4), (1000, 2), (1000, 3), (12345, 8)):
        costs = g.pareto(1.1, size=M) + 1.0
        rr = tgdist.shard_ranges(costs, world)
        assert len(rr) == world and rr[0][0] == 0 and rr[-1][1] == M
        assert all(a <= b for a, b in rr)
        assert all(rr[i][1] == rr[i + 1][0] for i in range(world - 1))  # contiguous, disjoint
        if M >= world:
            share = [costs[a:b].sum() for a, b in rr]
            # each rank within one edge's cost of an equal share
            assert max(share) <= costs.sum() / world + costs.max() + 1e-9


def test_edge_costs_follow_degrees():
    eu = np.array([0, 0, 0, 1], np.int32)
    ev = np.array([1, 2, 3, 2], np.int32)
    c = tgdist.edge_costs(4, eu, ev)
    assert c.tolist() == [3 + 2 + 64.0, 3 + 2 + 64.0, 3 + 1 + 64.0, 2 + 2 + 64.0]


@pytest.mark.parametrize("graph_seed", [3, 11])
def test_two_gloo_ranks_reproduce_the_global_count(oracle_mod, graph_seed):
    ctx = mp.get_context("spawn")
    results = ctx.Queue()
    port = _free_port()
    from tests.gloo_worker import rank_main
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, graph_seed, results)) for r in range(2)]
    for p in procs:
        p.start()
    got = [results.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    (r0, a0, b0, ok0, nz0), (r1, a1, b1, ok1, nz1) = got
    assert (r0, r1) == (0, 1) and a0 == 0 and b0 == a1 and b1 > a1  # two non-empty shards
    assert ok0 and ok1 and nz0 and nz1
