"""tg_count_global_noalloc: the count for callers that cannot allocate device
memory (arena-owned devices, plugins that may not allocate after start-up,
latency-critical loops).  Its result must equal tg_count_global's, call after
call, while the library allocates nothing: the allocation hook below fails
every device allocation the library attempts during those calls."""
import numpy as np
import pytest

import paper_1901_10026_gb300 as tg
from paper_1901_10026_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10026_gb300 import build
    build.build()
    torch.cuda.init()


def _graphs():
    yield synth.er_1000(seed=1)                                   # L = 3
    g = synth.rng(990)
    u, v = synth.chung_lu_exact(5000, 30000, 2.1, g)
    yield synth.TypedEdgeList(5000, u, v, synth.zipf_types(5000, 5, 1.2, g), 5, "cl-5k")
    yield synth.tiny_random(300, 0.05, 9, synth.rng(991))         # largest L for k = 4


@pytest.mark.parametrize("k", [3, 4])
def test_noalloc_matches_count_global_twice(k):
    import torch
    for G in _graphs():
        g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
        want = tg.tg_count_global(g, k)
        dev_out = torch.zeros(tg.tg_global_len(G.L, k), dtype=torch.int64, device="cuda:0")
        host_out = np.zeros(tg.tg_global_len(G.L, k), np.uint64)
        tg.tg_debug_fail_alloc(1)  # any library allocation from here on would fail
        try:
            for _ in range(2):
                tg.tg_count_global_noalloc(g, k, dev_out)
                torch.cuda.synchronize()
                assert np.array_equal(dev_out.cpu().numpy().view(np.uint64), want)
                tg.tg_count_global_noalloc(g, k, host_out)
                assert np.array_equal(host_out, want)
        finally:
            tg.tg_debug_fail_alloc(0)


def test_noalloc_takes_no_device_memory_after_its_first_call():
    """The device's free memory is the same before and after repeated calls
    (the first call on the device, which may load the module, came before)."""
    import torch
    G = synth.er_1000(seed=1)
    g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    out = torch.zeros(tg.tg_global_len(G.L, 4), dtype=torch.int64, device="cuda:0")
    tg.tg_count_global_noalloc(g, 4, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(0)
    for _ in range(3):
        tg.tg_count_global_noalloc(g, 4, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(0)
    assert free1 == free0
    assert np.array_equal(out.cpu().numpy().view(np.uint64), tg.tg_count_global(g, 4))


def test_noalloc_rejects_oversized_histograms():
    G = synth.tiny_random(40, 0.2, 10, synth.rng(992))  # k = 4 at L = 10 exceeds the array
    g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
    out = np.zeros(tg.tg_global_len(G.L, 4), np.uint64)
    with pytest.raises(tg.TGError) as e:
        tg.tg_count_global_noalloc(g, 4, out)
    assert e.value.status == tg.TG_EINVAL
    out3 = np.zeros(tg.tg_global_len(G.L, 3), np.uint64)  # k = 3 fits at any L
    tg.tg_count_global_noalloc(g, 3, out3)
    assert np.array_equal(out3, tg.tg_count_global(g, 3))
