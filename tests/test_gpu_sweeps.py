"""The paper's synthetic series at reduced size, through the C ABI against the
second oracle, bit-exact: the Erdos-Renyi scalability graphs (average degree
10), the number-of-types sweep on an Erdos-Renyi and a Chung-Lu graph
(L = 2..9), and the type-permutation null model (one topology, permuted type
vectors, also counted together as one batch)."""
import numpy as np
import pytest

import paper_1901_10026_gb300 as tg
from oracle import o2
from paper_1901_10026_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10026_gb300 import build
    build.build()
    o2.build()
    tg.tg_set_tune(reset=True)


@pytest.mark.parametrize("n", [100, 1000, 10000])
def test_er_scalability_series(n):
    G = synth.er_avg_degree(n, 10.0, 3)
    g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    assert abs(2 * g.M / n - 10.0) < 2.0
    assert np.array_equal(tg.tg_count_global(g, 4), o2.global_counts_of(G, 4))


@pytest.mark.parametrize("L", range(2, 10))
def test_number_of_types_sweep(L):
    for G in (synth.er_exact(3000, 15000, L), synth.cl_sweep(3000, 15000, L)):
        g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
        assert g.M == 15000
        assert np.array_equal(tg.tg_count_global(g, 4), o2.global_counts_of(G, 4)), G.name


def test_type_permutation_null_model():
    import torch
    base = synth.cl_sweep(3000, 15000, 5)
    base.types = synth.zipf_types(base.n, 5, 1.2, synth.rng(970))
    perms = synth.type_permutations(base.types, 6)
    for t in perms:
        assert np.array_equal(np.bincount(t, minlength=5), np.bincount(base.types, minlength=5))
    Gs = [base] + [synth.TypedEdgeList(base.n, base.src, base.dst, t, 5) for t in perms]
    graphs = [tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L) for G in Gs]
    want = [o2.global_counts_of(G, 4) for G in Gs]
    for g, w in zip(graphs, want):
        assert np.array_equal(tg.tg_count_global(g, 4), w)
    glen = tg.tg_global_len(5, 4)
    buf = torch.zeros((len(Gs), glen), dtype=torch.int64, device="cuda:0")
    plan = tg.Batch(graphs, 4, tg.TG_BATCH_GLOBAL, [buf[q] for q in range(len(Gs))], cta_threads=256)
    plan.run()
    got = buf.cpu().numpy().view(np.uint64)
    for q in range(len(Gs)):
        assert np.array_equal(got[q], want[q]), q
    plan.close()
