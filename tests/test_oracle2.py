"""Pins of the second oracle (non-induced pattern counts and their inversion):
brute force of the definition on tiny graphs, and agreement with the
paper-method oracle on larger graphs where brute force cannot go.  The
closed-form families (tests/test_oracle_closed_forms.py) run on it too."""
import numpy as np
import pytest

from oracle import brute, o2
from paper_1901_10026_gb300 import synth
from tests import layout


def _cases(count, seed):
    g = synth.rng(920, seed)
    out = []
    for _ in range(count):
        n = int(g.integers(0, 11))
        out.append(synth.tiny_random(n, float(g.uniform(0.15, 0.95)), int(g.integers(1, 5)), g))
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_global_matches_brute_force(seed):
    for G in _cases(80, seed):
        for k in (3, 4):
            got = layout.decode_global(o2.global_counts_of(G, k), G.L, k)
            want = {key: c for key, c in brute.global_graphlets(G.n, G.src, G.dst, G.types, k).items()}
            assert got == want, (G.name, k)


def test_dense_graphs_exercise_every_inversion_term():
    """Graphs dense enough to hold diamonds and 4-cliques, so each subtracted
    multiplicity (6, 4, 12, 3, 2, ...) is non-zero somewhere."""
    g = synth.rng(921, 0)
    seen = set()
    for _ in range(30):
        G = synth.tiny_random(9, 0.7, 2, g)
        got = layout.decode_global(o2.global_counts_of(G), G.L, 4)
        assert got == brute.global_graphlets(G.n, G.src, G.dst, G.types)
        seen |= {h for (h, _), c in got.items() if c}
    assert seen == set(range(9))


@pytest.mark.parametrize("make", [
    lambda: synth.er_1000(seed=1),
    lambda: synth.TypedEdgeList(20000, *synth.chung_lu_exact(20000, 160000, 2.1, synth.rng(922, 0)),
                                synth.zipf_types(20000, 5, 1.2, synth.rng(922, 1)), 5, "cl-20k"),
    lambda: synth.TypedEdgeList(4096, *synth.rmat(12, 16, 0.57, 0.19, 0.19, 0.05, synth.rng(922, 2)),
                                synth.uniform_types(4096, 16, synth.rng(922, 3)), 16, "rmat-12-L16"),
])
def test_agrees_with_the_paper_method_oracle(oracle_mod, make):
    G = make()
    og = oracle_mod.OracleGraph.from_edges(G)
    for k in (3, 4):
        assert np.array_equal(o2.global_counts_of(G, k), og.global_counts(k=k))


def test_invalid_input_is_rejected():
    with pytest.raises(RuntimeError):
        o2.global_counts(3, np.array([0]), np.array([3]), np.zeros(3, np.uint8), 2)
    with pytest.raises(RuntimeError):
        o2.global_counts(3, np.array([0]), np.array([1]), np.array([0, 2, 0], np.uint8), 2)
    assert o2.global_counts(0, np.zeros(0), np.zeros(0), np.zeros(0, np.uint8), 3).sum() == 0
