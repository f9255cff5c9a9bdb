"""The seeded generators of the synthetic workloads (no GPU): sizes and laws
the recipes state, determinism, and the type permutations of the null model."""
import numpy as np

from paper_1901_10026_gb300 import synth


def _simple_edges(G):
    a = np.minimum(G.src, G.dst).astype(np.int64)
    b = np.maximum(G.src, G.dst).astype(np.int64)
    keep = a != b
    return np.unique(a[keep] * G.n + b[keep]).shape[0]


def test_er_exact_has_exactly_m_distinct_edges():
    G = synth.er_exact(3000, 15000, 4, seed=3)
    assert G.m == 15000 and _simple_edges(G) == 15000
    assert G.types.max() < 4 and np.bincount(G.types, minlength=4).min() > 600


def test_cl_sweep_has_exactly_m_distinct_edges_and_skew():
    G = synth.cl_sweep(3000, 15000, 3, seed=4)
    assert _simple_edges(G) == 15000
    deg = np.bincount(np.concatenate([G.src, G.dst]), minlength=G.n)
    assert deg.max() > 20 * np.median(deg[deg > 0])  # power-law hubs


def test_er_average_degree():
    G = synth.er_avg_degree(20000, 10.0, 3, seed=5)
    assert abs(2 * _simple_edges(G) / G.n - 10.0) < 0.3


def test_type_permutations_keep_the_type_counts():
    t = synth.zipf_types(5000, 5, 1.2, synth.rng(7))
    perms = synth.type_permutations(t, 5, seed=2)
    assert len(perms) == 5
    for q in perms:
        assert np.array_equal(np.bincount(q, minlength=5), np.bincount(t, minlength=5))
        assert not np.array_equal(q, t)
    assert all(np.array_equal(a, b) for a, b in zip(perms, synth.type_permutations(t, 5, seed=2)))


def test_er_directed_reciprocity():
    G = synth.er_directed(5000, 40000, 0.25, 2, seed=6)
    m = 40000
    assert G.src.shape[0] > m and abs((G.src.shape[0] - m) / m - 0.25) < 0.02
    # the added arcs are the reverses of earlier ones
    fwd = set(zip(G.src[:m].tolist(), G.dst[:m].tolist()))
    assert all((d, s) in fwd for s, d in zip(G.src[m:].tolist(), G.dst[m:].tolist()))


def test_generators_are_deterministic():
    for make in (lambda: synth.er_exact(500, 2000, 3, seed=9), lambda: synth.cl_sweep(500, 2000, 3, seed=9),
                 lambda: synth.er_directed(500, 2000, 0.3, 3, seed=9), lambda: synth.rmat_23(scale=8)):
        a, b = make(), make()
        assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst)
        assert np.array_equal(a.types, b.types)
