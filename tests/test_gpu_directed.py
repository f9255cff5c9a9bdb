"""Directed typed 3-node graphlets through the C ABI against the directed
oracle (Sec. "Directed Typed Graphlets"), bit-exact: per-edge rows and global
counts on random tiny digraphs (loops, repeated and reciprocal arcs), a
directed Erdos-Renyi graph, directed R-MAT scale 14 with L = 8 (arcs as
drawn), stars and cliques; the sums over direction classes equal the
undirected 3-node counts of the same graph; errors."""
from math import comb

import numpy as np
import pytest

import paper_1901_10026_gb300 as tg
from oracle import odir
from paper_1901_10026_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10026_gb300 import build
    build.build()
    odir.build()


def _check(G):
    g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L, directed=True)
    want_rows, want = odir.counts_of(G)
    assert g.M == want_rows.shape[0]
    got = tg.tg_count_directed_global(g)
    assert np.array_equal(got, want), G.name
    rows = tg.tg_count_directed_per_edge(g)
    bad = np.argwhere(rows != want_rows)
    assert bad.shape[0] == 0, (G.name, bad[:5])
    return g, got


@pytest.mark.parametrize("seed", range(25))
def test_tiny_random_digraphs(seed):
    r = np.random.default_rng(1000 + seed)
    n = int(r.integers(2, 40))
    L = int(r.integers(1, 5))
    m = int(r.integers(0, 4 * n))
    G = synth.TypedEdgeList(n, r.integers(0, n, m).astype(np.int32), r.integers(0, n, m).astype(np.int32),
                            r.integers(0, L, n).astype(np.uint8), L, f"tiny{seed}")
    _check(G)


def test_directed_er_and_undirected_sums():
    G = synth.er_directed(3000, 30000, 0.25, 3, seed=5)
    g, got = _check(G)
    L = G.L
    n3 = comb(L + 2, 3)
    und = tg.tg_count_global(g, 3)
    P = L * (L + 1) // 2
    gg = got.reshape(13, n3).astype(np.int64)
    assert np.array_equal(gg[[0, 1, 2, 3, 4, 7]].sum(0), und[P:P + n3].astype(np.int64))
    assert np.array_equal(gg[[5, 6, 8, 9, 10, 11, 12]].sum(0), und[P + n3:].astype(np.int64))


def test_directed_rmat14():
    G = synth.rmat_23(scale=14)
    _check(G)


@pytest.mark.parametrize("L", [1, 16])
def test_type_count_extremes(L):
    # L = 1 (untyped census) and the largest L (the widest shared histogram)
    _check(synth.er_directed(600, 5000, 0.3, L, seed=11 + L))


@pytest.mark.parametrize("n", [3, 50, 300])
def test_stars_and_cliques(n):
    star = [(0, v) for v in range(1, n)] + [(v, 0) for v in range(1, n, 3)]
    a = np.array(star, np.int32)
    _check(synth.TypedEdgeList(n, a[:, 0].copy(), a[:, 1].copy(), (np.arange(n) % 2).astype(np.uint8), 2,
                               f"star{n}"))
    k = min(n, 60)
    cl = [(x, y) for x in range(k) for y in range(k) if x != y and (x + 2 * y) % 3]
    a = np.array(cl, np.int32)
    _check(synth.TypedEdgeList(k, a[:, 0].copy(), a[:, 1].copy(), (np.arange(k) % 3).astype(np.uint8), 3,
                               f"clique{k}"))


def test_device_io_and_errors():
    import torch
    G = synth.er_directed(500, 3000, 0.3, 2, seed=9)
    dev = torch.device("cuda", 0)
    g = tg.tg_build_csr(G.n, torch.from_numpy(G.src).to(dev), torch.from_numpy(G.dst).to(dev),
                        torch.from_numpy(G.types).to(dev), G.L, directed=True)
    want_rows, want = odir.counts_of(G)
    out = torch.zeros(tg.tg_dir_global_len(G.L), dtype=torch.int64, device=dev)
    tg.tg_count_directed_global(g, out)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), want)
    rows = torch.zeros((g.M, tg.tg_dir_slots(G.L)), dtype=torch.int64, device=dev)
    tg.tg_count_directed_per_edge(g, rows)
    assert np.array_equal(rows.cpu().numpy().view(np.uint64), want_rows)
    und = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    with pytest.raises(tg.TGError):
        tg.tg_count_directed_global(und)
    empty = tg.tg_build_csr(4, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(4, np.uint8), 1,
                            directed=True)
    assert not tg.tg_count_directed_global(empty).any()
