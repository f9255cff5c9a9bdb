"""Pins of the directed typed 3-node oracle (Sec. "Directed Typed Graphlets"):
the relabelling-search oracle against the dyad-census brute force on random
tiny digraphs (loops, repeated and reciprocal arcs included), closed forms of
tournaments, bidirected cliques, directed cycles and stars, and the sums over
direction classes against the undirected 3-node counts of the second oracle."""
from math import comb

import numpy as np
import pytest

from oracle import brute_dir, o2, odir
from paper_1901_10026_gb300 import synth

N3 = lambda L: comb(L + 2, 3)
PATHS = [0, 1, 2, 3, 4, 7]
TRIANGLES = [5, 6, 8, 9, 10, 11, 12]


def _G(n, arcs, L=1, types=None):
    arcs = np.array(arcs, np.int32).reshape(-1, 2)
    t = np.zeros(n, np.uint8) if types is None else np.asarray(types, np.uint8)
    return synth.TypedEdgeList(n, arcs[:, 0].copy(), arcs[:, 1].copy(), t, L)


def _by_class(glob, L):
    return np.asarray(glob, np.int64).reshape(13, N3(L)).sum(axis=1)


@pytest.mark.parametrize("seed", range(60))
def test_oracle_equals_brute_force(seed):
    r = np.random.default_rng(seed)
    n = int(r.integers(3, 13))
    L = int(r.integers(1, 4))
    m = int(r.integers(0, 3 * n))
    src = r.integers(0, n, m).astype(np.int32)
    dst = r.integers(0, n, m).astype(np.int32)
    G = synth.TypedEdgeList(n, src, dst, r.integers(0, L, n).astype(np.uint8), L)
    rows, glob = odir.counts_of(G)
    und, brows, bglob = brute_dir.counts(n, src, dst, G.types, L)
    assert rows.shape == (len(und), 13 * L)
    assert np.array_equal(rows, np.array(brows, np.uint64).reshape(len(und), 13 * L))
    assert np.array_equal(glob, np.array(bglob, np.uint64))


def test_every_class_is_met():
    r = np.random.default_rng(7)
    seen = np.zeros(13, np.int64)
    for _ in range(40):
        G = synth.er_directed(9, 20, 0.4, 1, seed=int(r.integers(1 << 30)))
        seen += _by_class(odir.counts_of(G, rows=False)[1], 1)
    assert np.all(seen > 0)


@pytest.mark.parametrize("n", [3, 4, 7])
def test_closed_forms(n):
    C3 = comb(n, 3)
    tour = [(a, b) for a in range(n) for b in range(a + 1, n)]
    want = np.zeros(13, np.int64)
    want[5] = C3  # transitive tournament: every triad is 030T
    assert np.array_equal(_by_class(odir.counts_of(_G(n, tour))[1], 1), want)
    bid = tour + [(b, a) for a, b in tour]
    want = np.zeros(13, np.int64)
    want[12] = C3  # bidirected clique: 300
    assert np.array_equal(_by_class(odir.counts_of(_G(n, bid))[1], 1), want)
    star_out = [(0, v) for v in range(1, n)]
    want = np.zeros(13, np.int64)
    want[0] = comb(n - 1, 2)  # 021D
    assert np.array_equal(_by_class(odir.counts_of(_G(n, star_out))[1], 1), want)
    star_in = [(v, 0) for v in range(1, n)]
    want = np.zeros(13, np.int64)
    want[1] = comb(n - 1, 2)  # 021U
    assert np.array_equal(_by_class(odir.counts_of(_G(n, star_in))[1], 1), want)
    star_mut = star_out + star_in
    want = np.zeros(13, np.int64)
    want[7] = comb(n - 1, 2)  # 201
    assert np.array_equal(_by_class(odir.counts_of(_G(n, star_mut))[1], 1), want)
    cyc = [(v, (v + 1) % n) for v in range(n)]
    want = np.zeros(13, np.int64)
    if n == 3:
        want[6] = 1  # 030C
    else:
        want[2] = n  # 021C
    assert np.array_equal(_by_class(odir.counts_of(_G(n, cyc))[1], 1), want)


def test_typed_closed_form_tournament():
    # transitive tournament with types: the 030T count of a multiset is the
    # number of node triples with those types
    n, L = 9, 3
    types = np.array([0, 1, 2, 0, 1, 2, 0, 0, 1], np.uint8)
    tour = [(a, b) for a in range(n) for b in range(a + 1, n)]
    glob = odir.counts_of(_G(n, tour, L, types), rows=False)[1].reshape(13, N3(L))
    import itertools
    want = np.zeros(N3(L), np.int64)
    for tri in itertools.combinations(range(n), 3):
        a, b, c = sorted(int(types[v]) for v in tri)
        want[a + (b + 1) * b // 2 + (c + 2) * (c + 1) * c // 6] += 1
    assert np.array_equal(glob[5], want)
    assert glob.sum() == want.sum()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_direction_sums_equal_undirected_counts(seed):
    G = synth.er_directed(400, 2400, 0.3, 3, seed=seed)
    rows, glob = odir.counts_of(G)
    h = o2.global_counts_of(G, 3)  # [edges][3-paths][triangles] of the underlying graph
    L, n3 = G.L, N3(G.L)
    P = L * (L + 1) // 2
    g = glob.reshape(13, n3).astype(np.int64)
    assert np.array_equal(g[PATHS].sum(axis=0), h[P:P + n3].astype(np.int64))
    assert np.array_equal(g[TRIANGLES].sum(axis=0), h[P + n3:P + 2 * n3].astype(np.int64))
    assert rows.shape[0] == int(h[:P].sum())
