"""Sparse per-edge output through the C ABI against the oracle's dense rows:
for every edge, the (graphlet or orbit, type multiset) -> count pairs decoded
from (offsets, ids, counts) must be exactly the nonzero slots of the
oracle's row, keyed by the same motif and the sorted types of all its nodes
(the edge's two endpoint types plus the slot's one or two).  Bit-exact."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1901_10026_gb300 as tg
from paper_1901_10026_gb300 import synth
from tests import layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10026_gb300 import build
    build.build()
    oracle.build()


def _dense_dict(row, L, k, level, ti, tj):
    P = layout.pairs(L)
    out = {}
    for t in range(L):
        for m, base in ((1, 0), (2, L)):
            if row[base + t]:
                out[(m, tuple(sorted((ti, tj, t))))] = int(row[base + t])
    if k == 4:
        nblk = 10 if level == tg.TG_ORBIT else 6
        for b in range(nblk):
            for p, (t, u) in enumerate(P):
                v = row[2 * L + b * len(P) + p]
                if v:
                    out[(3 + b, tuple(sorted((ti, tj, t, u))))] = int(v)
    return out


def _check(G, k, level):
    g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    og = oracle.OracleGraph.from_edges(G)
    want = og.per_edge(k=k, level="orbit" if level == tg.TG_ORBIT else "graphlet")
    u, v = og.edges()
    offsets, ids, counts = tg.tg_count_per_edge_sparse(g, k, level)
    assert offsets.shape[0] == g.M + 1 and offsets[0] == 0
    assert np.all(np.diff(offsets) >= 0) and offsets[-1] == ids.shape[0]
    assert ids.shape[0] == np.count_nonzero(want)
    lookup = {}
    for e in range(g.M):
        ti, tj = int(G.types[u[e]]), int(G.types[v[e]])
        got = {}
        for q in range(offsets[e], offsets[e + 1]):
            sid = int(ids[q])
            if sid not in lookup:
                lookup[sid] = tg.tg_sparse_id(G.L, k, level, sid)
            got[lookup[sid]] = int(counts[q])
        assert got == _dense_dict(want[e], G.L, k, level, ti, tj), (G.name, e)
    return g


@pytest.mark.parametrize("k,level", [(3, tg.TG_GRAPHLET), (4, tg.TG_GRAPHLET), (4, tg.TG_ORBIT)])
def test_sparse_rows_equal_the_oracle(k, level):
    _check(synth.er_1000(seed=7), k, level)
    r = synth.rng(960)
    for c in range(6):
        G = synth.tiny_random(int(r.integers(2, 40)), float(r.uniform(0.1, 0.9)), int(r.integers(1, 6)),
                              synth.rng(961, c))
        G.name = f"tiny-{c}"
        _check(G, k, level)


def test_sparse_chung_lu_and_capacity():
    r = synth.rng(962)
    u, v = synth.chung_lu_exact(20000, 120000, 2.1, r)
    G = synth.TypedEdgeList(20000, u, v, synth.zipf_types(20000, 5, 1.2, r), 5, "cl-20k")
    g = _check(G, 4, tg.TG_GRAPHLET)
    offsets = np.zeros(g.M + 1, np.int64)
    nnz = ctypes.c_int64(0)
    ids = np.zeros(8, np.uint32)
    counts = np.zeros(8, np.uint64)
    rc = tg.lib().tg_count_per_edge_sparse(g.handle, 4, tg.TG_GRAPHLET, tg._ptr(offsets), tg._ptr(ids),
                                           tg._ptr(counts), 8, ctypes.byref(nnz), None)
    assert rc == tg.TG_EOVERFLOW and nnz.value == offsets[-1] > 8
