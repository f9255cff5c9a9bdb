"""Pins of the directed typed 4-node oracle (Sec. "Directed Typed Graphlets",
199 classes of connected 4-node digraphs): against the brute force over all
node quadruples of tiny digraphs (loops, repeated and reciprocal arcs
included), closed forms of tournaments, bidirected cliques, directed cycles
and stars, and the sums over the classes of each undirected shape against
the undirected oracles (global counts of O2, per-edge rows of O1)."""
from math import comb

import numpy as np
import pytest

import oracle
from oracle import brute_dir, o2, odir
from paper_1901_10026_gb300 import synth

N4 = lambda L: comb(L + 3, 4)


def _G(n, arcs, L=1, types=None):
    arcs = np.array(arcs, np.int32).reshape(-1, 2)
    t = np.zeros(n, np.uint8) if types is None else np.asarray(types, np.uint8)
    return synth.TypedEdgeList(n, arcs[:, 0].copy(), arcs[:, 1].copy(), t, L)


def _canon(arcs4):
    """Class index of a digraph on positions 0..3 given as arcs."""
    code = 0
    for a, b in arcs4:
        code |= 1 << (4 * a + b)
    codes, _ = odir.classes4()
    return int(np.flatnonzero(codes == brute_dir._canon4(code))[0])


def _shape(code):
    """h3..h8 index (0..5) of the underlying undirected graph of a class code."""
    pairs = [(a, b) for a in range(4) for b in range(a + 1, 4)
             if (code >> (4 * a + b)) & 1 or (code >> (4 * b + a)) & 1]
    deg = sorted(sum(1 for p in pairs if v in p) for v in range(4))
    m = len(pairs)
    if m == 3:
        return 1 if deg == [1, 1, 1, 3] else 0
    if m == 4:
        return 2 if deg == [2, 2, 2, 2] else 3
    return 4 if m == 5 else 5


def test_class_table():
    codes, edges = odir.classes4()
    assert len(codes) == 199 and list(codes) == brute_dir.class_table4()
    assert sorted(set(edges.tolist())) == [3, 4, 5, 6]
    shapes = np.bincount([_shape(int(c)) for c in codes], minlength=6)
    # directed versions of path, star, cycle, tailed triangle, chordal cycle, clique
    assert shapes.sum() == 199 and np.all(shapes > 0)


@pytest.mark.parametrize("seed", range(25))
def test_oracle_equals_brute_force(seed):
    r = np.random.default_rng(400 + seed)
    n = int(r.integers(4, 10))
    L = int(r.integers(1, 3))
    m = int(r.integers(0, 3 * n))
    src = r.integers(0, n, m).astype(np.int32)
    dst = r.integers(0, n, m).astype(np.int32)
    G = synth.TypedEdgeList(n, src, dst, r.integers(0, L, n).astype(np.uint8), L)
    rows, glob = odir.counts4_of(G)
    und, brows, bglob = brute_dir.counts4(n, src, dst, G.types, L)
    P = L * (L + 1) // 2
    assert np.array_equal(rows, np.array(brows, np.uint64).reshape(len(und), 199 * P))
    assert np.array_equal(glob, np.array(bglob, np.uint64))


@pytest.mark.parametrize("n", [4, 6, 8])
def test_closed_forms(n):
    def by_class(G):
        return odir.counts4_of(G, rows=False)[1].reshape(199, N4(1)).sum(axis=1)

    tour = [(a, b) for a in range(n) for b in range(a + 1, n)]
    want = np.zeros(199, np.int64)
    want[_canon([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])] = comb(n, 4)
    assert np.array_equal(by_class(_G(n, tour)), want)
    bid = tour + [(b, a) for a, b in tour]
    want = np.zeros(199, np.int64)
    want[_canon([(a, b) for a in range(4) for b in range(4) if a != b])] = comb(n, 4)
    assert np.array_equal(by_class(_G(n, bid)), want)
    out_star = [(0, v) for v in range(1, n)]
    want = np.zeros(199, np.int64)
    want[_canon([(0, 1), (0, 2), (0, 3)])] = comb(n - 1, 3)
    assert np.array_equal(by_class(_G(n, out_star)), want)
    in_star = [(v, 0) for v in range(1, n)]
    want = np.zeros(199, np.int64)
    want[_canon([(1, 0), (2, 0), (3, 0)])] = comb(n - 1, 3)
    assert np.array_equal(by_class(_G(n, in_star)), want)
    cyc = [(v, (v + 1) % n) for v in range(n)]
    want = np.zeros(199, np.int64)
    if n == 4:
        want[_canon([(0, 1), (1, 2), (2, 3), (3, 0)])] = 1
    else:
        want[_canon([(0, 1), (1, 2), (2, 3)])] = n
    assert np.array_equal(by_class(_G(n, cyc)), want)


@pytest.mark.parametrize("seed", [1, 2])
def test_shape_sums_equal_undirected_counts(seed):
    G = synth.er_directed(150, 900, 0.3, 2, seed=seed)
    rows, glob = odir.counts4_of(G)
    L = G.L
    P, n3, n4 = L * (L + 1) // 2, comb(L + 2, 3), N4(L)
    codes, _ = odir.classes4()
    shape = np.array([_shape(int(c)) for c in codes])
    g = glob.reshape(199, n4).astype(np.int64)
    h = o2.global_counts_of(G, 4).astype(np.int64)
    off4 = P + 2 * n3
    for s in range(6):
        assert np.array_equal(g[shape == s].sum(axis=0), h[off4 + s * n4: off4 + (s + 1) * n4]), s
    # per edge: the classes of one shape add up to the undirected graphlet row
    og = oracle.OracleGraph.from_edges(G)
    urows = og.per_edge(k=4, level="graphlet").astype(np.int64)
    d = rows.reshape(rows.shape[0], 199, P).astype(np.int64)
    for s in range(6):
        assert np.array_equal(d[:, shape == s, :].sum(axis=1), urows[:, 2 * L + s * P: 2 * L + (s + 1) * P]), s
