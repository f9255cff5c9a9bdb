"""Oracle invariants: untyped = sum over types (Prop. 1), L = 1, degree identity,
relabel and type-permutation equivariance."""
import numpy as np
import pytest

from oracle import brute
from paper_1901_10026_gb300 import synth
from tests import layout


def _sum_by_graphlet(dec):
    out = {}
    for (h, _m), c in dec.items():
        out[h] = out.get(h, 0) + c
    return out


@pytest.mark.parametrize("seed", range(6))
def test_untyped_equals_sum_over_types(oracle_mod, seed):
    g = synth.rng(930, seed)
    G = synth.tiny_random(int(g.integers(20, 60)), float(g.uniform(0.1, 0.4)), 4, g)
    og = oracle_mod.OracleGraph.from_edges(G)
    typed = _sum_by_graphlet(layout.decode_global(og.global_counts(), 4))
    og1 = oracle_mod.OracleGraph(G.n, G.src, G.dst, np.zeros(G.n, np.uint8), 1)
    untyped = _sum_by_graphlet(layout.decode_global(og1.global_counts(), 1))
    assert typed == untyped
    # per edge as well (Prop. 1 is stated per edge)
    rt = og.per_edge(level="orbit")
    r1 = og1.per_edge(level="orbit")
    P = 10
    for e in range(og.M):
        a = layout.decode_orbit_row(rt[e], 4)
        b = layout.decode_orbit_row(r1[e], 1)
        sa = {}
        for (o, _k), c in a.items():
            sa[o] = sa.get(o, 0) + c
        assert sa == {o: c for (o, _k), c in b.items()}


def test_L1_equals_untyped_brute_force(oracle_mod):
    for seed in range(10):
        G = synth.tiny_random(10, 0.5, 1, synth.rng(931, seed))
        og = oracle_mod.OracleGraph.from_edges(G)
        got = layout.decode_global(og.global_counts(), 1)
        assert got == brute.global_graphlets(G.n, G.src, G.dst, G.types)


@pytest.mark.parametrize("seed", range(4))
def test_degree_identity(oracle_mod, seed):
    """d_i + d_j = 2|T_ij| + |S_i| + |S_j| + 2 (each degree also counts the edge)."""
    G = synth.tiny_random(50, 0.2, 3, synth.rng(932, seed))
    og = oracle_mod.OracleGraph.from_edges(G)
    rows = og.per_edge(k=3)
    u, v = og.edges()
    deg = np.bincount(np.concatenate([u, v]), minlength=G.n)
    L = G.L
    for e in range(og.M):
        S = int(rows[e, :L].sum())
        T = int(rows[e, L:2 * L].sum())
        assert deg[u[e]] + deg[v[e]] == 2 * T + S + 2


@pytest.mark.parametrize("seed", range(3))
def test_relabel_and_type_permutation(oracle_mod, seed):
    g = synth.rng(933, seed)
    G = synth.tiny_random(40, 0.25, 4, g)
    og = oracle_mod.OracleGraph.from_edges(G)
    base_rows = og.per_edge(level="orbit")
    u, v = og.edges()
    base_glob = layout.decode_global(og.global_counts(), 4)
    perm = g.permutation(G.n).astype(np.int32)       # node relabel old -> new
    tperm = g.permutation(4).astype(np.uint8)        # type relabel
    new_types = np.empty(G.n, np.uint8)
    new_types[perm] = tperm[G.types]
    G2 = synth.TypedEdgeList(G.n, perm[G.src], perm[G.dst], new_types, 4)
    og2 = oracle_mod.OracleGraph.from_edges(G2)
    rows2 = og2.per_edge(level="orbit")
    u2, v2 = og2.edges()
    index2 = {(int(a), int(b)): e for e, (a, b) in enumerate(zip(u2, v2))}
    for e in range(og.M):
        a, b = int(perm[u[e]]), int(perm[v[e]])
        e2 = index2[(min(a, b), max(a, b))]
        d1 = layout.decode_orbit_row(base_rows[e], 4)
        d2 = layout.decode_orbit_row(rows2[e2], 4)
        mapped = {(o, tuple(sorted(int(tperm[t]) for t in key))): c for (o, key), c in d1.items()}
        assert mapped == d2
    glob2 = layout.decode_global(og2.global_counts(), 4)
    mapped = {(h, tuple(sorted(int(tperm[t]) for t in m))): c for (h, m), c in base_glob.items()}
    assert mapped == glob2


def test_edge_cases(oracle_mod):
    # no edges at all; isolated nodes; a single edge; loops and duplicates only
    for n, src, dst in ((5, [], []), (1, [0], [0]), (2, [0, 1, 1], [1, 0, 1]), (3, [2], [0])):
        G = synth.TypedEdgeList(n, np.array(src, np.int32), np.array(dst, np.int32),
                                np.zeros(n, np.uint8), 2)
        og = oracle_mod.OracleGraph.from_edges(G)
        glob = og.global_counts()
        assert glob[1:].sum() == 0
        assert glob[0] == og.M
        assert og.per_edge().sum() == 0
    with pytest.raises(ValueError):
        oracle_mod.OracleGraph(3, np.array([0], np.int32), np.array([3], np.int32), np.zeros(3, np.uint8), 2)
    with pytest.raises(ValueError):
        oracle_mod.OracleGraph(3, np.array([0], np.int32), np.array([1], np.int32), np.array([0, 2, 0], np.uint8), 2)
