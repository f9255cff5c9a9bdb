"""The stored R-MAT-23 global counts (written by tests/golden/make_rmat23_o2.py
from the second oracle alone): the file is intact (its recorded sha256), and
the counts satisfy what the graph fixes: the edge block sums to M, every
typed configuration occurs, and the sizes are the layout's."""
import hashlib
import os
from math import comb

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "rmat23_o2_global.txt")


def read_golden(path=GOLDEN):
    header, vals = {}, []
    for line in open(path):
        if line.startswith("#"):
            if "M = " in line:
                header["M"] = int(line.split("M = ")[1].split()[0])
            if "sha256" in line:
                header["sha256"] = line.split("=")[-1].strip()
            if "entries = " in line:
                header["entries"] = int(line.split("entries = ")[1].split(",")[0])
            continue
        vals.append(int(line))
    return header, np.array(vals, dtype=np.uint64)


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="golden file not written")
def test_golden_file_is_intact_and_consistent():
    h, g = read_golden()
    L = 8
    P = L * (L + 1) // 2
    assert g.shape[0] == h["entries"] == P + 2 * comb(L + 2, 3) + 6 * comb(L + 3, 4)
    assert hashlib.sha256(np.ascontiguousarray(g, dtype="<u8").tobytes()).hexdigest() == h["sha256"]
    assert int(g[:P].sum()) == h["M"] == 129338312
    assert np.count_nonzero(g) == g.shape[0]
