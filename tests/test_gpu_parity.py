"""CUDA path (through the C ABI) against the oracle, bit-exact in uint64."""
import numpy as np
import pytest

import oracle
import paper_1901_10026_gb300 as tg
from paper_1901_10026_gb300 import synth

pytestmark = pytest.mark.gpu


# Kernel variants: the tuned defaults (the cycles kernel), the warp/binary-
# search kernel, the bitmap kernel and the reuse kernel, some squeezed so that
# their fallbacks (ids beyond the bitmap, lists too long for the hash, 4-clique
# candidate sets too large for shared memory) carry most of the work.  Counts
# must not change.
VARIANTS = {
    "default": dict(),
    "cycles-small": dict(kernel=tg.TG_KERNEL_CYCLES, cta_threads=64, hash_slots=32, bitmap_bits=96,
                         grid_limit=3, unroll=1),
    "cycles-split": dict(kernel=tg.TG_KERNEL_CYCLES, unroll=4),
    "cycles-split-bitmap": dict(kernel=tg.TG_KERNEL_CYCLES, unroll=4, hash_slots=32),
    # the fused per-edge kernel (T sums kept in shared memory, identities in
    # the same warp), which the library picks on its own only when the T sums
    # of the whole graph would not fit in a quarter of free memory
    "cycles-fused": dict(kernel=tg.TG_KERNEL_CYCLES, edge_pass=tg.TG_EDGE_PASS_FUSED),
    "cycles-fused-small": dict(kernel=tg.TG_KERNEL_CYCLES, edge_pass=tg.TG_EDGE_PASS_FUSED,
                               cta_threads=64, hash_slots=32, bitmap_bits=96, grid_limit=3),
    # the per-edge pass in batches of work units (as on graphs whose T sums
    # do not fit in memory at once)
    "cycles-batched": dict(kernel=tg.TG_KERNEL_CYCLES, edge_batch=700),
    # every costly 4-cycle anchor in the binned waves, or none of them
    "cycles-binned-all": dict(kernel=tg.TG_KERNEL_CYCLES, c4_bin_fill=1),
    "cycles-binned-none": dict(kernel=tg.TG_KERNEL_CYCLES, c4_bin_fill=1 << 20),
    "reuse": dict(kernel=tg.TG_KERNEL_REUSE),
    "warp-search": dict(kernel=tg.TG_KERNEL_WARP_SEARCH),
    "cta-small": dict(kernel=tg.TG_KERNEL_CTA_BITMAP, cta_threads=128, unroll=1, hash_slots=32,
                      bitmap_bits=96),
    "cta-u4": dict(kernel=tg.TG_KERNEL_CTA_BITMAP, cta_threads=512, unroll=4),
    "reuse-small": dict(kernel=tg.TG_KERNEL_REUSE, cta_threads=64, unroll=1, hash_slots=32,
                        bitmap_bits=96),
    "reuse-u4": dict(kernel=tg.TG_KERNEL_REUSE, cta_threads=256, unroll=4, grid_limit=3),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10026_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.init()
    yield
    tg.tg_set_tune(reset=True)


@pytest.fixture(params=list(VARIANTS))
def variant(request):
    tg.tg_set_tune(**VARIANTS[request.param])
    yield request.param
    tg.tg_set_tune(reset=True)


def _both(G):
    return tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L), oracle.OracleGraph.from_edges(G)


def _check_all(G, levels=(tg.TG_GRAPHLET, tg.TG_ORBIT), ks=(3, 4)):
    g, og = _both(G)
    assert g.M == og.M
    u, v = tg.tg_edge_list(g)
    ou, ov = og.edges()
    assert np.array_equal(u, ou) and np.array_equal(v, ov)
    for k in ks:
        for level in levels:
            got = tg.tg_count_per_edge(g, k, level)
            want = og.per_edge(k=k, level="orbit" if level == tg.TG_ORBIT else "graphlet")
            assert got.shape == want.shape
            bad = np.argwhere(got != want)
            assert bad.shape[0] == 0, (G.name, k, level, bad[:5], got[bad[0][0]], want[bad[0][0]])
        gg = tg.tg_count_global(g, k)
        assert np.array_equal(gg, og.global_counts(k=k)), (G.name, k)
    return g, og


def test_er_1000_full_parity(variant):
    """G(n=1000, p=0.01), L=3: every per-edge row (both levels, k=3,4) and the
    global histogram."""
    G = synth.er_1000(seed=1)
    g, og = _check_all(G)
    deg = np.bincount(np.concatenate(og.edges()), minlength=G.n)
    assert g.max_degree == deg.max() and g.n_nonisolated == (deg > 0).sum()


@pytest.mark.parametrize("seed", range(4))
def test_tiny_random_suite(seed, variant):
    r = synth.rng(700, seed)
    for c in range(15):
        n = int(r.integers(2, 40))
        L = int(r.integers(1, 7))
        G = synth.tiny_random(n, float(r.uniform(0.05, 0.9)), L, synth.rng(701, seed, c))
        G.name = f"tiny-{seed}-{c}"
        _check_all(G)


def _graph(n, pairs, types, L, name):
    e = np.array(pairs, np.int32).reshape(-1, 2)
    return synth.TypedEdgeList(n, e[:, 0].copy(), e[:, 1].copy(), np.asarray(types, np.uint8), L, name)


def test_degenerate_graphs(variant):
    # isolated nodes only; one edge; loops and duplicates only; two components
    _check_all(_graph(7, [], [0] * 7, 2, "empty"))
    _check_all(_graph(2, [(0, 1)], [0, 1], 2, "one-edge"))
    _check_all(_graph(3, [(1, 1), (2, 2), (0, 1), (1, 0), (0, 1)], [0, 1, 0], 2, "loops-dups"))
    _check_all(_graph(9, [(0, 1), (1, 2), (2, 0), (5, 6), (6, 7), (7, 8), (8, 5)], [0, 1, 2, 0, 1, 2, 0, 1, 2], 3, "two-comp"))


def test_hub_star_and_cliques(variant):
    r = synth.rng(702)
    s = 5000
    pairs = [(0, x) for x in range(1, s + 1)]
    pairs += [(x, x + 1) for x in range(1, 400)]          # a path among the leaves
    _check_all(_graph(s + 1, pairs, synth.uniform_types(s + 1, 4, r), 4, "hub-star"), ks=(4,))
    import itertools
    n = 60
    _check_all(_graph(n, list(itertools.combinations(range(n), 2)), synth.uniform_types(n, 5, r), 5,
                      "K60"), levels=(tg.TG_ORBIT,))


@pytest.mark.parametrize("L", [1, 2, 16])
def test_type_count_extremes(L, variant):
    G = synth.tiny_random(200, 0.08, L, synth.rng(703, L))
    G.name = f"L{L}"
    _check_all(G)


def test_chung_lu_medium(variant):
    """Chung-Lu n=20,000, 120,000 distinct edges, gamma 2.1, L=5 Zipf types:
    hubs of degree in the thousands, full per-edge parity."""
    g = synth.rng(704)
    u, v = synth.chung_lu_exact(20000, 120000, 2.1, g)
    G = synth.TypedEdgeList(20000, u, v, synth.zipf_types(20000, 5, 1.2, g), 5, "cl-20k")
    _check_all(G, levels=(tg.TG_GRAPHLET,), ks=(4,))


def test_memory_retention_keeps_counts():
    """Scratch from the library's retaining pool (and after a trim) gives the
    same global and per-edge counts as the default pool."""
    g0 = synth.rng(705)
    u, v = synth.chung_lu_exact(20000, 120000, 2.1, g0)
    G = synth.TypedEdgeList(20000, u, v, synth.zipf_types(20000, 5, 1.2, g0), 5, "cl-20k-b")
    g, og = _both(G)
    want_g, want_e = og.global_counts(k=4), og.per_edge(k=4, level="graphlet")
    try:
        tg.tg_set_memory_retention(1 << 30)
        for _ in range(2):
            assert np.array_equal(tg.tg_count_global(g, 4), want_g)
            assert np.array_equal(tg.tg_count_per_edge(g, 4, tg.TG_GRAPHLET), want_e)
        tg.tg_trim_memory()
        assert np.array_equal(tg.tg_count_global(g, 4), want_g)
    finally:
        tg.tg_set_memory_retention(0)
    assert np.array_equal(tg.tg_count_global(g, 4), want_g)


def test_device_inputs_and_outputs():
    import torch
    G = synth.er_1000(seed=2)
    og = oracle.OracleGraph.from_edges(G)
    dev = torch.device("cuda:0")
    g = tg.tg_build_csr(G.n, torch.from_numpy(G.src).to(dev), torch.from_numpy(G.dst).to(dev),
                        torch.from_numpy(G.types).to(dev), G.L)
    out = torch.zeros(tg.tg_global_len(G.L, 4), dtype=torch.uint64, device=dev)
    tg.tg_count_global(g, 4, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), og.global_counts())
    rows = torch.zeros((g.M, tg.tg_slots(G.L, 4, tg.TG_ORBIT)), dtype=torch.uint64, device=dev)
    tg.tg_count_per_edge(g, 4, tg.TG_ORBIT, rows)
    torch.cuda.synchronize()
    assert np.array_equal(rows.cpu().numpy(), og.per_edge(level="orbit"))


def test_sharded_ranges_sum_to_global(variant):
    """Edge-range shards (the unit one rank computes) add up to the global count."""
    G = synth.er_1000(seed=3)
    g, og = _both(G)
    total = np.zeros(tg.tg_global_len(G.L, 4), np.uint64)
    cuts = [0, 1, 997, 2500, g.M - 1, g.M]
    for a, b in zip(cuts[:-1], cuts[1:]):
        total += tg.tg_count_range(g, 4, a, b)
    assert np.array_equal(tg.tg_global_finalize(G.L, 4, total), og.global_counts())


def test_invalid_inputs_are_rejected():
    with pytest.raises(tg.TGError) as e:
        tg.tg_build_csr(3, np.array([0], np.int32), np.array([3], np.int32), np.zeros(3, np.uint8), 2)
    assert e.value.status == tg.TG_EINVAL
    with pytest.raises(tg.TGError) as e:
        tg.tg_build_csr(3, np.array([0], np.int32), np.array([1], np.int32), np.array([0, 2, 0], np.uint8), 2)
    assert e.value.status == tg.TG_EINVAL
    with pytest.raises(tg.TGError):
        tg.tg_build_csr(3, np.array([0], np.int32), np.array([1], np.int32), np.zeros(3, np.uint8), 17)
    g = tg.tg_build_csr(3, np.array([0], np.int32), np.array([1], np.int32), np.zeros(3, np.uint8), 2)
    with pytest.raises(tg.TGError):
        tg.tg_count_global(g, 5)


def test_allocation_failure_unwinds():
    G = synth.er_1000(seed=4)
    for nth in (1, 2, 5, 9):
        tg.tg_debug_fail_alloc(nth)
        try:
            with pytest.raises(tg.TGError) as e:
                tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
            assert e.value.status == tg.TG_ENOMEM
        finally:
            tg.tg_debug_fail_alloc(0)
    g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    tg.tg_debug_fail_alloc(1)
    try:
        with pytest.raises(tg.TGError):
            tg.tg_count_global(g, 4)
    finally:
        tg.tg_debug_fail_alloc(0)
    og = oracle.OracleGraph.from_edges(G)
    assert np.array_equal(tg.tg_count_global(g, 4), og.global_counts())


def test_work_model_matches_host():
    G = synth.er_1000(seed=5)
    g, og = _both(G)
    u, v = og.edges()
    n = G.n
    adj = [set() for _ in range(n)]
    for a, b in zip(u, v):
        adj[a].add(b)
        adj[b].add(a)
    deg = np.array([len(a) for a in adj])
    want = 0
    for a, b in zip(u, v):
        i, j = (a, b) if (deg[a], -a) < (deg[b], -b) else (b, a)
        N = (adj[i] | adj[j]) - {i, j}
        want += 2 * deg[i] + deg[j] + sum(int(deg[w]) for w in N)
    assert tg.tg_work_model(g) == want
