"""C ABI of libtg.so without a GPU: every declared symbol is exported, and the
host-only helpers (layout, ranks, hash) agree with the paper and the oracle."""
import ctypes
import os
import re
from math import comb

import numpy as np
import pytest

import paper_1901_10026_gb300 as tg
from paper_1901_10026_gb300 import build as tgbuild
from tests import layout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    tgbuild.build()
    return tg.lib()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for m in re.finditer(r"\b(tg_[a-z0-9_]+)\s*\(", text):
                names.add(m.group(1))
    names -= {"tg_alloc_fn", "tg_free_fn"}  # function-pointer typedefs
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    raw = ctypes.CDLL(tgbuild.LIB)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_layout_sizes(lib):
    for L in range(1, 17):
        P = L * (L + 1) // 2
        assert tg.tg_slots(L, 3) == 2 * L
        assert tg.tg_slots(L, 4, tg.TG_GRAPHLET) == 2 * L + 6 * P
        assert tg.tg_slots(L, 4, tg.TG_ORBIT) == 2 * L + 10 * P
        assert tg.tg_global_len(L, 4) == layout.global_blocks(L, 4)[1]
        assert tg.tg_global_len(L, 3) == layout.global_blocks(L, 3)[1]
        for k in (1, 2, 3, 4):
            assert tg.tg_config_count(L, k) == comb(L + k - 1, k)
    assert tg.tg_slots(0, 4) == 0 and tg.tg_slots(17, 4) == 0 and tg.tg_slots(3, 5) == 0


def test_config_rank_is_colex_and_unrank_inverts(lib):
    for L in range(1, 9):
        for k in (1, 2, 3, 4):
            for r, m in enumerate(layout.multisets(L, k)):
                assert tg.tg_config_rank(list(reversed(m))) == r
                assert tg.tg_config_unrank(r, k) == m


def test_paper_hash(lib):
    # Sec. "Typed Motif Hash Functions": types shifted to 1..L, sorted, 0-padded
    assert tg.tg_paper_hash(2, [0, 1, 1], 3) == 2 * 10**4 + 1 * 10**3 + 2 * 10**2 + 2 * 10 + 0
    assert tg.tg_paper_hash(12, [2, 0, 1, 2], 3) == 12 * 10**4 + 1000 + 200 + 30 + 3
    assert tg.tg_paper_hash(7, [9, 10, 0, 11], 12) == 7 * 10**8 + 1 * 10**6 + 10 * 10**4 + 11 * 10**2 + 12
    # every ordering maps to one value; distinct multisets to distinct values
    seen = {}
    for m in layout.multisets(5, 4):
        h = tg.tg_paper_hash(3, list(m), 5)
        assert h not in seen
        seen[h] = m
        assert tg.tg_paper_hash(3, list(reversed(m)), 5) == h
    assert tg.tg_paper_hash(1, [5], 5) == 0  # type out of range


def test_slot_config_matches_row_layout(lib):
    L = 4
    for level, width in ((tg.TG_GRAPHLET, tg.tg_slots(L, 4, 0)), (tg.TG_ORBIT, tg.tg_slots(L, 4, 1))):
        for s in range(width):
            motif, types = tg.tg_slot_config(L, 4, level, 2, 0, s)
            if s < L:
                assert (motif, types) == (1, tuple(sorted((2, 0, s))))
            elif s < 2 * L:
                assert (motif, types) == (2, tuple(sorted((2, 0, s - L))))
            else:
                q, p = divmod(s - 2 * L, L * (L + 1) // 2)
                t, u = layout.pairs(L)[p]
                assert (motif, types) == (q + 3, tuple(sorted((2, 0, t, u))))


def test_host_finalize(lib):
    L = 3
    blocks, n = layout.global_blocks(L, 4)
    eh = {0: 1, 1: 2, 2: 3, 3: 3, 4: 3, 5: 4, 6: 4, 7: 5, 8: 6}
    rng = np.random.default_rng(0)
    want = rng.integers(0, 1000, n).astype(np.uint64)
    sums = want.copy()
    for h, size, off in blocks:
        cnt = comb(L + size - 1, size)
        sums[off:off + cnt] *= np.uint64(eh[h])
    assert np.array_equal(tg.tg_global_finalize(L, 4, sums), want)
    sums[-1] += np.uint64(1)  # 4-clique sums must be multiples of 6
    with pytest.raises(tg.TGError):
        tg.tg_global_finalize(L, 4, sums)


def test_strerror(lib):
    assert tg.tg_strerror(0) == "ok"
    assert tg.tg_strerror(tg.TG_EINVAL) == "invalid argument"
    assert tg.tg_version() >= 100


def test_memory_retention_setting_without_device_work(lib):
    """The retention setting is host state until a pool is made on first
    allocation; setting, trimming and resetting it needs no GPU."""
    tg.tg_set_memory_retention(1 << 30)
    tg.tg_trim_memory()
    tg.tg_set_memory_retention(0)
    tg.tg_trim_memory()
