"""A global count split across ranks (tg_count_shard), every shard run on one
GPU in turn: the shards' undivided sums add up, after the division by
|E(H)|, to tg_count_global's histogram and to the oracle's, bit-exact.  The
shards slice the per-edge pass and deal out the 4-cycle anchors and 4-clique
lowest nodes, so each shard's own sums differ from an edge range's; only the
total is fixed."""
import numpy as np
import pytest

import oracle
import paper_1901_10026_gb300 as tg
from oracle import o2
from paper_1901_10026_gb300 import synth

pytestmark = pytest.mark.gpu

TUNES = {
    "default": dict(),
    "split-anchors": dict(kernel=tg.TG_KERNEL_CYCLES, unroll=4),
    "tiles-hash": dict(kernel=tg.TG_KERNEL_CYCLES, hash_slots=32),
    "warp-search": dict(kernel=tg.TG_KERNEL_WARP_SEARCH),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10026_gb300 import build
    build.build()
    oracle.build()
    o2.build()
    yield
    tg.tg_set_tune(reset=True)


@pytest.fixture(params=list(TUNES))
def tune(request):
    tg.tg_set_tune(**TUNES[request.param])
    yield request.param
    tg.tg_set_tune(reset=True)


def _graphs():
    yield synth.er_1000(seed=6)
    r = synth.rng(940)
    u, v = synth.chung_lu_exact(20000, 120000, 2.1, r)
    yield synth.TypedEdgeList(20000, u, v, synth.zipf_types(20000, 5, 1.2, r), 5, "cl-20k")
    yield synth.rmat_23(scale=14)
    yield synth.TypedEdgeList(3, np.array([0], np.int32), np.array([1], np.int32),
                              np.array([0, 1, 0], np.uint8), 2, "one-edge")


@pytest.mark.parametrize("k", [3, 4])
def test_shards_add_up_to_the_global_count(tune, k):
    for G in _graphs():
        g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
        want = tg.tg_count_global(g, k)
        if k == 4 and G.m > 1:
            assert np.array_equal(want, o2.global_counts_of(G, 4)), G.name
        for N in (1, 2, 3, 5):
            total = np.zeros_like(want)
            for r in range(N):
                total += tg.tg_count_shard(g, k, r, N)
            got = tg.tg_global_finalize(G.L, k, total)
            assert np.array_equal(got, want), (tune, G.name, k, N)


def test_shard_arguments_are_checked():
    G = synth.er_1000(seed=6)
    g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    for shard, n in ((-1, 2), (2, 2), (0, 0)):
        with pytest.raises(tg.TGError) as e:
            tg.tg_count_shard(g, 4, shard, n)
        assert e.value.status == tg.TG_EINVAL
