"""Batched counting against per-graph counts and the oracle, bit-exact: the
single persistent launch, the union of each type-count group through the
whole-graph path, and the tuner's choice between them."""
import numpy as np
import pytest

import oracle
import paper_1901_10026_gb300 as tg
from paper_1901_10026_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10026_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.init()


def _batch_graphs(count, seed):
    """Small graphs from the batched workload's laws, scaled down in n."""
    out = []
    for it in synth.batch_spec(count, seed=seed):
        it.n = max(2, it.n // 8)
        if it.family == "cl":
            it.avg_degree = min(it.avg_degree, (it.n - 1) / 2.0)
        out.append(synth.batch_graph(it, seed=seed))
    # degenerate members: empty graph, single edge, L = 16
    out.append(synth.TypedEdgeList(5, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(5, np.uint8), 2))
    out.append(synth.TypedEdgeList(2, np.array([0], np.int32), np.array([1], np.int32), np.array([0, 1], np.uint8), 2))
    out.append(synth.tiny_random(60, 0.2, 16, synth.rng(880)))
    return out


def _dev(n):
    import torch
    return torch.zeros(n, dtype=torch.int64, device="cuda:0")


@pytest.mark.parametrize("path", ["auto", "union", "persistent"])
@pytest.mark.parametrize("mode", [tg.TG_BATCH_GLOBAL, tg.TG_BATCH_PER_EDGE_GRAPHLET, tg.TG_BATCH_PER_EDGE_ORBIT])
def test_batch_matches_oracle(mode, path):
    Gs = _batch_graphs(40, 3)
    graphs = [tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L) for G in Gs]
    if mode == tg.TG_BATCH_GLOBAL:
        outs = [_dev(tg.tg_global_len(G.L, 4)) for G in Gs]
    else:
        level = tg.TG_ORBIT if mode == tg.TG_BATCH_PER_EDGE_ORBIT else tg.TG_GRAPHLET
        outs = [_dev(max(1, g.M * tg.tg_slots(G.L, 4, level))) for G, g in zip(Gs, graphs)]
    plan = tg.Batch(graphs, 4, mode, outs, path=path)
    if path == "auto":
        plan.tune()
    elif path == "persistent":
        assert plan.tune() != 0  # the union path is not built
    for rep in range(2):  # persistent path: the first run captures the CUDA graph, the second replays it
        for o in outs:
            o.zero_()
        plan.run()
        for G, g, o in zip(Gs, graphs, outs):
            got = o.cpu().numpy().view(np.uint64)
            og = oracle.OracleGraph.from_edges(G)
            if mode == tg.TG_BATCH_GLOBAL:
                assert np.array_equal(got, og.global_counts(k=4)), G.name
            else:
                lv = "orbit" if mode == tg.TG_BATCH_PER_EDGE_ORBIT else "graphlet"
                want = og.per_edge(k=4, level=lv)
                assert np.array_equal(got[: want.size].reshape(want.shape), want), G.name
    plan.close()


@pytest.mark.parametrize("cta", [256, 0])
def test_one_shot_batch_equals_single_graph_counts(cta):
    Gs = _batch_graphs(25, 4)
    graphs = [tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L) for G in Gs]
    outs = [_dev(tg.tg_global_len(G.L, 3)) for G in Gs]
    tg.tg_count_batch(graphs, 3, tg.TG_BATCH_GLOBAL, outs, cta_threads=cta)
    for g, o, G in zip(graphs, outs, Gs):
        assert np.array_equal(o.cpu().numpy().view(np.uint64), tg.tg_count_global(g, 3)), G.name


@pytest.mark.parametrize("k", [3, 4])
def test_union_path_k3_and_medium_graphs(k):
    # several graphs per type count, some large enough for the CTA kernels
    Gs = [synth.cl_sweep(4000, 24000, L, seed=s) for L in (2, 3) for s in (1, 2)] + \
         [synth.er_avg_degree(3000, 12.0, 2, seed=3)]
    graphs = [tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L) for G in Gs]
    outs = [_dev(max(1, g.M * tg.tg_slots(G.L, k, tg.TG_GRAPHLET))) for G, g in zip(Gs, graphs)]
    plan = tg.Batch(graphs, k, tg.TG_BATCH_PER_EDGE_GRAPHLET, outs, path="union")
    plan.run()
    for G, g, o in zip(Gs, graphs, outs):
        want = tg.tg_count_per_edge(g, k, tg.TG_GRAPHLET)
        assert np.array_equal(o.cpu().numpy().view(np.uint64).reshape(want.shape), want), G.name
    plan.close()


def test_batch_rejects_host_outputs():
    G = synth.er_1000(seed=1)
    g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    with pytest.raises(tg.TGError):
        tg.Batch([g], 4, tg.TG_BATCH_GLOBAL, [np.zeros(tg.tg_global_len(G.L, 4), np.uint64)])
