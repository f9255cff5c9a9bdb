"""Directed typed 4-node graphlets through the C ABI against the directed
4-node oracle, bit-exact: per-edge rows and global counts on random tiny
digraphs (loops, repeated and reciprocal arcs), a directed Erdos-Renyi graph
and directed R-MAT scale 8; the sums over the classes of each undirected
shape equal the library's undirected 4-node counts; errors."""
from math import comb

import numpy as np
import pytest

import paper_1901_10026_gb300 as tg
from oracle import brute_dir, odir
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
    want_rows, want = odir.counts4_of(G)
    assert g.M == want_rows.shape[0]
    got = tg.tg_count_directed4_global(g)
    assert np.array_equal(got, want), G.name
    rows = tg.tg_count_directed4_per_edge(g)
    bad = np.argwhere(rows != want_rows)
    assert bad.shape[0] == 0, (G.name, bad[:5])
    return g, got


@pytest.mark.parametrize("seed", range(12))
def test_tiny_random_digraphs(seed):
    r = np.random.default_rng(2000 + seed)
    n = int(r.integers(4, 30))
    L = int(r.integers(1, 4))
    m = int(r.integers(0, 4 * n))
    G = synth.TypedEdgeList(n, r.integers(0, n, m).astype(np.int32), r.integers(0, n, m).astype(np.int32),
                            r.integers(0, L, n).astype(np.uint8), L, f"tiny{seed}")
    _check(G)


def test_directed_er_and_shape_sums():
    G = synth.er_directed(400, 2400, 0.3, 2, seed=8)
    g, got = _check(G)
    L = G.L
    P, n3, n4 = L * (L + 1) // 2, comb(L + 2, 3), comb(L + 3, 4)
    codes = brute_dir.class_table4()

    def shape(code):
        pairs = [(a, b) for a in range(4) for b in range(a + 1, 4)
                 if (code >> (4 * a + b)) & 1 or (code >> (4 * b + a)) & 1]
        deg = sorted(sum(1 for q in pairs if v in q) for v in range(4))
        m = len(pairs)
        if m == 3:
            return 1 if deg == [1, 1, 1, 3] else 0
        if m == 4:
            return 2 if deg == [2, 2, 2, 2] else 3
        return 4 if m == 5 else 5

    sh = np.array([shape(c) for c in codes])
    und = tg.tg_count_global(g, 4).astype(np.int64)
    gg = got.reshape(199, n4).astype(np.int64)
    off4 = P + 2 * n3
    for s in range(6):
        assert np.array_equal(gg[sh == s].sum(0), und[off4 + s * n4: off4 + (s + 1) * n4]), s


def test_directed_rmat8():
    G = synth.rmat_23(scale=8)
    G = synth.TypedEdgeList(G.n, G.src, G.dst, (np.arange(G.n) % 3).astype(np.uint8), 3, "rmat8-L3")
    _check(G)


def test_device_output_and_errors():
    import torch
    G = synth.er_directed(200, 1200, 0.3, 2, seed=12)
    g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L, directed=True)
    _, want = odir.counts4_of(G, rows=False)
    out = torch.zeros(tg.tg_dir4_global_len(G.L), dtype=torch.int64, device="cuda:0")
    tg.tg_count_directed4_global(g, out)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), want)
    und = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    with pytest.raises(tg.TGError):
        tg.tg_count_directed4_global(und)
