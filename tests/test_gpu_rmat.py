"""R-MAT graphs and the 16-bit counter boundary of the 4-cycle waves, through
the C ABI against the oracles, bit-exact in uint64 (tolerance 0).

* R-MAT scale 16, edge factor 16, (a, b, c, d) = (0.57, 0.19, 0.19, 0.05),
  L = 8 uniform types (the R-MAT-23 recipe at 1/128 of the size): the whole
  global histogram against the second oracle, and per-edge orbit rows of a
  sample (random edges, the costliest edges, both ends of the edge order)
  against the paper-method oracle, for the default per-edge pass and for the
  fused per-edge kernel and for the per-edge pass in batches of work units.
* K_{2,b} for b = 2^16 - 1 and 2^16: every 4-cycle has the same highest-ranked
  node (a hub of degree b) and the other hub as its far end, so that far end
  collects b middles in one counter: 2^16 - 1 is the largest count the 16-bit
  halves hold (anchors of degree below 2^16), 2^16 takes the 32-bit counters.
  Checked against the closed form of the typed complete bipartite graph and
  against the second oracle, at L = 1 (all middles of one type) and L = 3.
"""
from collections import Counter
from math import comb, prod

import numpy as np
import pytest

import oracle
import paper_1901_10026_gb300 as tg
from oracle import o2
from paper_1901_10026_gb300 import synth
from tests import layout

pytestmark = pytest.mark.gpu

EDGE_PASSES = {"auto": dict(edge_pass=tg.TG_EDGE_PASS_AUTO),
               "fused": dict(edge_pass=tg.TG_EDGE_PASS_FUSED),
               "batched": dict(edge_batch=50000)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10026_gb300 import build
    build.build()
    oracle.build()
    o2.build()
    torch.cuda.init()
    yield
    tg.tg_set_tune(reset=True)


@pytest.fixture(scope="module")
def rmat16():
    G = synth.rmat_23(scale=16)
    return G, o2.global_counts_of(G, 4), oracle.OracleGraph.from_edges(G)


@pytest.fixture(params=list(EDGE_PASSES))
def edge_pass(request):
    tg.tg_set_tune(kernel=tg.TG_KERNEL_CYCLES, **EDGE_PASSES[request.param])
    yield request.param
    tg.tg_set_tune(reset=True)


def test_rmat16_global_equals_independent_oracle(rmat16, edge_pass):
    G, want, _ = rmat16
    g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    got = tg.tg_count_global(g, 4)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (edge_pass, bad[:5], got[bad[:5]], want[bad[:5]])
    assert np.count_nonzero(got) == got.shape[0]  # every typed configuration occurs at L = 8
    got3 = tg.tg_count_global(g, 3)
    assert np.array_equal(got3, want[: got3.shape[0]])


def test_rmat16_sampled_orbit_rows(rmat16, edge_pass):
    import torch
    G, _, og = rmat16
    g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    assert g.M == og.M
    rows = torch.zeros((g.M, tg.tg_slots(G.L, 4, tg.TG_ORBIT)), dtype=torch.int64, device="cuda")
    tg.tg_count_per_edge(g, 4, tg.TG_ORBIT, rows)
    torch.cuda.synchronize()
    u, v = og.edges()
    gu, gv = tg.tg_edge_list(g)
    assert np.array_equal(u, gu) and np.array_equal(v, gv)
    deg = np.bincount(np.concatenate([u, v]), minlength=G.n)
    cost = deg[u].astype(np.int64) + deg[v]
    pick = synth.rng(931, 0).choice(g.M, 300, replace=False)
    sample = np.unique(np.concatenate([pick, np.argsort(cost)[-12:], [0, 1, g.M - 2, g.M - 1]]))
    want = og.per_edge(k=4, level="orbit", edges=sample)
    got = rows[torch.from_numpy(sample).to("cuda")].cpu().numpy().view(np.uint64)
    bad = np.argwhere(got != want)
    assert bad.shape[0] == 0, (edge_pass, sample[bad[0][0]], bad[:5])


def _k2b(b, L, seed):
    types = synth.uniform_types(b + 2, L, synth.rng(932, b, L, seed))
    src = np.repeat(np.array([0, 1], np.int32), b)
    dst = np.tile(np.arange(2, b + 2, dtype=np.int32), 2)
    return synth.TypedEdgeList(b + 2, src, dst, types, L, f"K2,{b}-L{L}")


def _k2b_closed_form(G):
    """Typed induced counts of K_{2,b}: edges hub-leaf, 3-paths (hub, two
    leaves) and (leaf, both hubs), 4-stars (hub, three leaves), 4-cycles (both
    hubs, two leaves); nothing else."""
    L = G.L
    hubs = Counter(int(t) for t in G.types[:2])
    leaves = Counter(int(t) for t in G.types[2:])

    def choose(counts, m):
        need = Counter(m)
        return prod(comb(counts.get(t, 0), c) for t, c in need.items())

    want = Counter()
    for h in layout.multisets(L, 1):
        for lf in layout.multisets(L, 1):
            want[(0, tuple(sorted(h + lf)))] += choose(hubs, h) * choose(leaves, lf)
        for m2 in layout.multisets(L, 2):
            want[(1, tuple(sorted(h + m2)))] += choose(hubs, h) * choose(leaves, m2)
        for m3 in layout.multisets(L, 3):
            want[(4, tuple(sorted(h + m3)))] += choose(hubs, h) * choose(leaves, m3)
    for lf in layout.multisets(L, 1):
        want[(1, tuple(sorted(lf + tuple(sorted(hubs.elements())))))] += choose(leaves, lf)
    for m2 in layout.multisets(L, 2):
        want[(5, tuple(sorted(m2 + tuple(sorted(hubs.elements())))))] += choose(leaves, m2)
    return {k: v for k, v in want.items() if v}


@pytest.mark.parametrize("b", [(1 << 16) - 1, 1 << 16])
@pytest.mark.parametrize("L", [1, 3])
def test_complete_bipartite_16bit_boundary(b, L):
    G = _k2b(b, L, 0)
    tg.tg_set_tune(reset=True)
    g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    assert g.max_degree == b
    got = tg.tg_count_global(g, 4)
    assert layout.decode_global(got, L, 4) == _k2b_closed_form(G)
    assert np.array_equal(got, o2.global_counts_of(G, 4))
    # the count that sits at the boundary: all b middles of the 4-cycles at one far end
    h5 = sum(c for (h, _), c in layout.decode_global(got, L, 4).items() if h == 5)
    assert h5 == comb(b, 2)
