"""Serving loop: continuous batching of counting requests.  Each result in the
mix must equal the same graph counted alone (exact; tolerance 0)."""
import math

import numpy as np
import pytest

import oracle
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
    oracle.build()
    o2.build()
    torch.cuda.init()


def _requests(count, seed, lo=200, hi=60000):
    g = synth.rng(870, seed)
    edges = np.floor(np.exp(g.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)
    return [synth.serve_graph(int(e), (871, seed, r)) for r, e in enumerate(edges)]


def test_results_in_the_mix_equal_solo_counts():
    Gs = _requests(36, 0)
    solo = []
    for G in Gs:
        g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
        solo.append(tg.tg_count_global(g, 4))
        g.close()
    sv = tg.Server(slots=4, batch_max=8, batch_edges=5000)
    tickets = [sv.submit(G.n, G.src, G.dst, G.types, G.L, 4) for G in Gs]
    for G, t, want in zip(Gs, tickets, solo):
        got, lat = sv.wait(t, timeout_ms=120000)
        assert np.array_equal(got, want), G.name
        assert lat > 0
    st = sv.stats()
    sv.close()
    assert st["completed"] == len(Gs) and st["failed"] == 0
    assert st["batched_launches"] >= 1 and st["grouped_requests"] >= 2  # small requests grouped
    assert st["peak_in_flight"] >= 2                                      # work overlapped
    assert st["p99_ms"] >= st["p50_ms"] > 0
    # every request against the independent global oracle, the smallest also
    # against the paper-method oracle
    for G, want in zip(Gs, solo):
        assert np.array_equal(o2.global_counts_of(G, 4), want), G.name
    for G, want in sorted(zip(Gs, solo), key=lambda x: x[0].m)[:4]:
        assert np.array_equal(oracle.OracleGraph.from_edges(G).global_counts(k=4), want)


def test_admission_queue_and_tickets():
    big = synth.serve_graph(300000, (872, 0, 0))
    small = _requests(6, 1, 300, 2000)
    # a request whose estimate exceeds the whole budget can never run
    sv = tg.Server(slots=1, mem_budget_bytes=16 << 20, queue_cap=2)
    with pytest.raises(tg.TGError) as e:
        sv.submit(big.n, big.src, big.dst, big.types, big.L)
    assert e.value.status == tg.TG_ENOMEM_ADMIT
    sv.close()
    sv = tg.Server(slots=1, queue_cap=2, batch_edges=0)
    t_big = sv.submit(big.n, big.src, big.dst, big.types, big.L)
    accepted, busy = [], 0
    for G in small:
        try:
            accepted.append((G, sv.submit(G.n, G.src, G.dst, G.types, G.L)))
        except tg.TGError as err:
            assert err.status == tg.TG_EBUSY
            busy += 1
    assert busy >= 1 and len(accepted) >= 1
    # bounded wait on a request still queued behind the large one
    with pytest.raises(tg.TGError) as e:
        sv.wait(accepted[-1][1], timeout_ms=0)
    assert e.value.status == tg.TG_ETIMEDOUT
    sv.wait(t_big, timeout_ms=120000)
    for G, t in accepted:
        got, _ = sv.wait(t, timeout_ms=120000)
        g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
        assert np.array_equal(got, tg.tg_count_global(g, 4))
    with pytest.raises(tg.TGError) as e:
        sv.wait(t_big, timeout_ms=10)       # already released
    assert e.value.status == tg.TG_ENOTFOUND
    with pytest.raises(tg.TGError) as e:
        sv.wait(123456789, timeout_ms=10)  # never issued
    assert e.value.status == tg.TG_ENOTFOUND
    with pytest.raises(tg.TGError) as e:  # invalid request: id out of range
        sv.submit(3, np.array([0], np.int32), np.array([5], np.int32), np.zeros(3, np.uint8), 2)
    assert e.value.status == tg.TG_EINVAL
    sv.close()


def test_concurrent_counts_of_mixed_sizes():
    """Four workers count, at the same time, graphs whose kernels need very
    different shared memory (small and large node counts, L from 2 to 8): no
    call may fail and every result equals the graph counted alone."""
    Gs = []
    for r in range(16):
        e = 400000 if r % 2 else 3000
        Gs.append(synth.serve_graph(e, (873, 0, r), L=2 + (r % 7)))
    solo = []
    for G in Gs:
        g = tg.tg_build_csr(G.n, G.src, G.dst, G.types, G.L)
        solo.append(tg.tg_count_global(g, 4))
        g.close()
    sv = tg.Server(slots=4, batch_edges=0)  # every request a launch of its own
    tickets = [sv.submit(G.n, G.src, G.dst, G.types, G.L, 4) for G in Gs]
    for G, t, want in zip(Gs, tickets, solo):
        got, _ = sv.wait(t, timeout_ms=300000)
        assert np.array_equal(got, want), G.name
    st = sv.stats()
    sv.close()
    assert st["completed"] == len(Gs) and st["failed"] == 0
    assert st["peak_in_flight"] >= 2
