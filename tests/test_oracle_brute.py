"""Oracle (paper's Alg. 1-3 + closed forms) against brute force of the definitions."""
import numpy as np
import pytest

from oracle import brute
from paper_1901_10026_gb300 import synth
from tests import layout


def _cases(count, seed):
    g = synth.rng(900, seed)
    for c in range(count):
        n = int(g.integers(2, 12))
        L = int(g.integers(1, 5))
        dens = float(g.uniform(0.1, 0.9))
        yield synth.tiny_random(n, dens, L, synth.rng(901, seed, c))


@pytest.mark.parametrize("seed", [0, 1])
def test_per_edge_orbits_match_brute_force(oracle_mod, seed):
    for G in _cases(120, seed):
        og = oracle_mod.OracleGraph.from_edges(G)
        rows = og.per_edge(k=4, level="orbit")
        u, v = og.edges()
        edges, bf = brute.per_edge_orbits(G.n, G.src, G.dst, G.types)
        assert [(int(a), int(b)) for a, b in zip(u, v)] == edges
        for e, (a, b) in enumerate(edges):
            got = layout.decode_orbit_row(rows[e], G.L)
            want = {(o, key): c for (o, key), c in bf[(a, b)].items()}
            assert got == want, (G.n, G.L, (a, b))


@pytest.mark.parametrize("seed", [2])
def test_per_edge_graphlets_are_orbit_sums(oracle_mod, seed):
    """Sec. "From Typed Orbits to Graphlets": h-rows equal the orbit sums."""
    for G in _cases(60, seed):
        og = oracle_mod.OracleGraph.from_edges(G)
        orb = og.per_edge(k=4, level="orbit")
        grl = og.per_edge(k=4, level="graphlet")
        for e in range(og.M):
            o = layout.decode_orbit_row(orb[e], G.L)
            h = {}
            for (g, key), c in o.items():
                hk = (layout.ORBIT_TO_GRAPHLET[g], key)
                h[hk] = h.get(hk, 0) + c
            assert layout.decode_graphlet_row(grl[e], G.L) == h


@pytest.mark.parametrize("seed", [3, 4])
def test_global_matches_brute_force(oracle_mod, seed):
    for G in _cases(80, seed):
        og = oracle_mod.OracleGraph.from_edges(G)
        got = layout.decode_global(og.global_counts(k=4), G.L, 4)
        want = brute.global_graphlets(G.n, G.src, G.dst, G.types)
        assert got == want


def test_k3_rows_are_prefix(oracle_mod):
    for G in _cases(20, 5):
        og = oracle_mod.OracleGraph.from_edges(G)
        r3 = og.per_edge(k=3)
        r4 = og.per_edge(k=4)
        assert r3.shape[1] == 2 * G.L
        assert np.array_equal(r3, r4[:, : 2 * G.L])
        g3 = og.global_counts(k=3)
        g4 = og.global_counts(k=4)
        assert np.array_equal(g3, g4[: g3.shape[0]])


def test_sampled_edges_equal_full_rows(oracle_mod):
    G = synth.tiny_random(11, 0.6, 3, synth.rng(902))
    og = oracle_mod.OracleGraph.from_edges(G)
    full = og.per_edge(k=4, level="orbit")
    pick = np.array([og.M - 1, 0, og.M // 2], np.int64)
    assert np.array_equal(og.per_edge(k=4, level="orbit", edges=pick), full[pick])
