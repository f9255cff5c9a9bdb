"""tg_autotune: the searched configuration is one the tuning accepts, the
counts under it equal the second oracle's, a graph of a cached class takes the
cached tuning without launching a kernel, and the tuning in force afterwards is
the one returned."""
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
    yield
    tg.tg_set_tune(reset=True)
    tg.tg_autotune_reset()


@pytest.mark.parametrize("k", [3, 4])
def test_autotune_counts_and_cache(k):
    tg.tg_set_tune(reset=True)
    tg.tg_autotune_reset()
    G = synth.cl_sweep(5000, 30000, 3)
    g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    best = tg.tg_autotune(g, k)
    assert best["kernel"] == tg.TG_KERNEL_CYCLES
    assert best["unroll"] in (2, 4) and best["hash_slots"] in (4096, 32)
    assert best["c4_bin_fill"] in (0, 8, 32, 128) and best["edge_pass"] in (0, 1)
    assert tg.tg_get_tune() == best
    want = o2.global_counts_of(G, k)
    assert np.array_equal(tg.tg_count_global(g, k), want)
    # same class (same L, k and bit lengths of M and of the maximum degree): cached
    tg.tg_set_tune(reset=True)
    g2 = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    n0 = tg.tg_launch_count()
    assert tg.tg_autotune(g2, k) == best
    assert tg.tg_launch_count() == n0
    assert tg.tg_get_tune() == best
    g.close()
    g2.close()
