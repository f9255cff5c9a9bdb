"""The sparse id space (CPU, host-side lookup of the C ABI): ids run block by
block (3-node graphlets or orbits, then 4-node ones), each block over the
sorted type multisets in colex order, derived here from tests/layout.py by
sorting, not by the rank formula."""
import pytest

import paper_1901_10026_gb300 as tg
from tests import layout


@pytest.mark.parametrize("L", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("k,level", [(3, tg.TG_GRAPHLET), (4, tg.TG_GRAPHLET), (4, tg.TG_ORBIT)])
def test_sparse_ids_enumerate_blocks_in_colex_order(L, k, level):
    from paper_1901_10026_gb300 import build
    build.build()
    want = []
    for m in (1, 2):
        want += [(m, ms) for ms in layout.multisets(L, 3)]
    if k == 4:
        last = 12 if level == tg.TG_ORBIT else 8
        for m in range(3, last + 1):
            want += [(m, ms) for ms in layout.multisets(L, 4)]
    assert tg.tg_sparse_ids(L, k, level) == len(want)
    got = [tg.tg_sparse_id(L, k, level, i) for i in range(len(want))]
    assert got == want
    with pytest.raises(tg.TGError):
        tg.tg_sparse_id(L, k, level, len(want))


def test_sparse_ids_reject_bad_arguments():
    assert tg.tg_sparse_ids(0, 4, tg.TG_GRAPHLET) == -1
    assert tg.tg_sparse_ids(3, 5, tg.TG_GRAPHLET) == -1
    assert tg.tg_sparse_ids(3, 4, 7) == -1
