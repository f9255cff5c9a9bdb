"""Oracle against closed forms on graph families whose typed counts are known.

Each expected value is a product of binomials over the node-type counts,
derived from the definitions (induced, connected, type multiset), not from the
oracle.
"""
import itertools
from collections import Counter
from math import comb, prod

import numpy as np
import pytest

from paper_1901_10026_gb300 import synth
from tests import layout


def _typed_choose(counts, m):
    """Number of ways to pick a sub-multiset m (tuple) from nodes with type counts."""
    need = Counter(m)
    return prod(comb(counts.get(t, 0), c) for t, c in need.items())


def _graph(n, edges, types, L):
    e = np.array(edges, np.int32).reshape(-1, 2)
    return synth.TypedEdgeList(n, e[:, 0].copy(), e[:, 1].copy(), np.array(types, np.uint8), L)


@pytest.fixture(params=["o1", "o2"])
def which(request):
    """The global counts under test: the paper-method oracle (o1) or the
    independent non-induced-inversion oracle (o2).  Per-edge checks use o1."""
    return request.param


def _global(oracle_mod, G, which="o1"):
    og = oracle_mod.OracleGraph.from_edges(G)
    if which == "o2":
        from oracle import o2
        vec = o2.global_counts(G.n, G.src, G.dst, G.types, G.L, 4)
    else:
        vec = og.global_counts(k=4)
    return layout.decode_global(vec, G.L, 4), og


@pytest.mark.parametrize("n,L,seed", [(4, 1, 0), (6, 2, 1), (8, 3, 2), (9, 4, 3), (7, 3, 4)])
def test_typed_clique(oracle_mod, which, n, L, seed):
    types = synth.uniform_types(n, L, synth.rng(910, seed))
    G = _graph(n, list(itertools.combinations(range(n), 2)), types, L)
    got, og = _global(oracle_mod, G, which)
    cnt = Counter(int(t) for t in types)
    want = {}
    for size, h in ((2, 0), (3, 2), (4, 8)):
        for m in layout.multisets(L, size):
            c = _typed_choose(cnt, m)
            if c:
                want[(h, m)] = c
    assert got == want
    # per edge: g12(t,t') = pairs of the remaining n-2 nodes, g2(t) = remaining nodes
    rows = og.per_edge(k=4, level="orbit")
    u, v = og.edges()
    for e in range(og.M):
        rest = Counter(cnt)
        rest[int(types[u[e]])] -= 1
        rest[int(types[v[e]])] -= 1
        d = layout.decode_orbit_row(rows[e], L)
        w = {}
        for t in range(L):
            if rest.get(t, 0):
                w[(2, (t,))] = rest[t]
        for (t, tt) in layout.pairs(L):
            c = comb(rest.get(t, 0), 2) if t == tt else rest.get(t, 0) * rest.get(tt, 0)
            if c:
                w[(12, (t, tt))] = c
        assert d == w


@pytest.mark.parametrize("s,L,seed", [(3, 1, 0), (6, 2, 1), (9, 3, 2), (12, 4, 3)])
def test_typed_star(oracle_mod, which, s, L, seed):
    types = synth.uniform_types(s + 1, L, synth.rng(911, seed))
    G = _graph(s + 1, [(0, x) for x in range(1, s + 1)], types, L)
    got, og = _global(oracle_mod, G, which)
    c0 = int(types[0])
    leaves = Counter(int(t) for t in types[1:])
    want = {}
    for m in layout.multisets(L, 1):
        c = _typed_choose(leaves, m)
        if c:
            want[(0, tuple(sorted((c0,) + m)))] = c
    for m in layout.multisets(L, 2):
        c = _typed_choose(leaves, m)
        if c:
            want[(1, tuple(sorted((c0,) + m)))] = c
    for m in layout.multisets(L, 3):
        c = _typed_choose(leaves, m)
        if c:
            want[(4, tuple(sorted((c0,) + m)))] = c
    assert got == want
    # per edge (centre, leaf): g1 = other leaves, g5 = pairs of other leaves
    rows = og.per_edge(k=4, level="orbit")
    u, v = og.edges()
    for e in range(og.M):
        leaf = int(v[e])
        rest = Counter(leaves)
        rest[int(types[leaf])] -= 1
        w = {}
        for t in range(L):
            if rest.get(t, 0):
                w[(1, (t,))] = rest[t]
        for (t, tt) in layout.pairs(L):
            c = comb(rest.get(t, 0), 2) if t == tt else rest.get(t, 0) * rest.get(tt, 0)
            if c:
                w[(5, (t, tt))] = c
        assert layout.decode_orbit_row(rows[e], L) == w


def _windows(types, n, size, cyclic):
    out = Counter()
    last = n if cyclic else n - size + 1
    for s in range(last):
        out[tuple(sorted(int(types[(s + q) % n]) for q in range(size)))] += 1
    return out


@pytest.mark.parametrize("n,L,seed", [(5, 2, 0), (7, 3, 1), (12, 4, 2), (30, 3, 3)])
def test_typed_cycle(oracle_mod, which, n, L, seed):
    types = synth.uniform_types(n, L, synth.rng(912, seed))
    G = _graph(n, [(x, (x + 1) % n) for x in range(n)], types, L)
    got, og = _global(oracle_mod, G, which)
    want = {}
    for size, h in ((2, 0), (3, 1), (4, 3)):
        for m, c in _windows(types, n, size, True).items():
            want[(h, m)] = c
    assert got == want
    # every edge: 2 wedges (g1), end edge of two 4-paths (g3), centre of one (g4)
    rows = og.per_edge(k=4, level="orbit")
    for e in range(og.M):
        d = layout.decode_orbit_row(rows[e], L)
        assert sum(c for (o, _), c in d.items() if o == 1) == 2
        assert sum(c for (o, _), c in d.items() if o == 3) == 2
        assert sum(c for (o, _), c in d.items() if o == 4) == 1
        assert all(o in (1, 3, 4) for (o, _) in d)


def test_four_cycle(oracle_mod, which):
    types = [0, 1, 0, 1]
    G = _graph(4, [(0, 1), (1, 2), (2, 3), (3, 0)], types, 2)
    got, _ = _global(oracle_mod, G, which)
    assert got == {(0, (0, 1)): 4, (1, (0, 0, 1)): 2, (1, (0, 1, 1)): 2, (5, (0, 0, 1, 1)): 1}


@pytest.mark.parametrize("n,L,seed", [(4, 1, 0), (9, 2, 1), (25, 3, 2)])
def test_typed_path(oracle_mod, which, n, L, seed):
    types = synth.uniform_types(n, L, synth.rng(913, seed))
    G = _graph(n, [(x, x + 1) for x in range(n - 1)], types, L)
    got, _ = _global(oracle_mod, G, which)
    want = {}
    for size, h in ((2, 0), (3, 1), (4, 3)):
        for m, c in _windows(types, n, size, False).items():
            want[(h, m)] = c
    assert got == want


@pytest.mark.parametrize("a,b,L,seed", [(2, 2, 1, 0), (3, 4, 2, 1), (5, 6, 3, 2), (4, 7, 4, 3)])
def test_typed_complete_bipartite(oracle_mod, which, a, b, L, seed):
    types = synth.uniform_types(a + b, L, synth.rng(914, seed))
    A = Counter(int(t) for t in types[:a])
    B = Counter(int(t) for t in types[a:])
    G = _graph(a + b, [(x, a + y) for x in range(a) for y in range(b)], types, L)
    got, _ = _global(oracle_mod, G, which)
    want = Counter()
    # edges: one node per side
    for ma in layout.multisets(L, 1):
        for mb in layout.multisets(L, 1):
            want[(0, tuple(sorted(ma + mb)))] += _typed_choose(A, ma) * _typed_choose(B, mb)
    # 3-paths: centre on one side, two leaves on the other; no triangles
    for one, two in ((A, B), (B, A)):
        for m1 in layout.multisets(L, 1):
            for m2 in layout.multisets(L, 2):
                want[(1, tuple(sorted(m1 + m2)))] += _typed_choose(one, m1) * _typed_choose(two, m2)
            for m3 in layout.multisets(L, 3):
                want[(4, tuple(sorted(m1 + m3)))] += _typed_choose(one, m1) * _typed_choose(two, m3)
    # 4-cycles: two nodes from each side
    for m2a in layout.multisets(L, 2):
        for m2b in layout.multisets(L, 2):
            want[(5, tuple(sorted(m2a + m2b)))] += _typed_choose(A, m2a) * _typed_choose(B, m2b)
    want = {k: v for k, v in want.items() if v}
    assert got == want
