"""R-MAT-23 (the benchmark graph: 2^23 nodes, 16 x 2^23 draws, (0.57, 0.19,
0.19, 0.05), L = 8) counted on the device with the default kernels, against
the golden global counts the second oracle wrote on the CPU
(tests/golden/make_rmat23_o2.py): all 2,256 entries, bit-exact."""
import os

import numpy as np
import pytest

import paper_1901_10026_gb300 as tg
from paper_1901_10026_gb300 import synth
from tests.test_golden_rmat23 import GOLDEN, read_golden

pytestmark = pytest.mark.gpu


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="golden file not written")
def test_rmat23_global_equals_golden():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10026_gb300 import build
    build.build()
    tg.tg_set_tune(reset=True)
    tg.tg_set_memory_retention(64 << 30)
    try:
        head, want = read_golden()
        G = synth.rmat_23()
        dev = torch.device("cuda", 0)
        g = tg.tg_build_csr(G.n, torch.from_numpy(G.src).to(dev), torch.from_numpy(G.dst).to(dev),
                            torch.from_numpy(G.types).to(dev), G.L)
        assert g.M == head["M"]
        out = torch.zeros(tg.tg_global_len(G.L, 4), dtype=torch.int64, device=dev)
        tg.tg_count_global(g, 4, out)
        got = out.cpu().numpy().view(np.uint64)
        bad = np.flatnonzero(got != want)
        assert bad.size == 0, (bad[:5], got[bad[:5]], want[bad[:5]])
        g.close()
    finally:
        tg.tg_set_memory_retention(0)
