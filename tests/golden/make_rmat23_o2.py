"""Writes rmat23_o2_global.txt: the global typed 2/3/4-node graphlet counts of
the R-MAT scale-23 graph, computed by the second CPU oracle alone.

Graph: R-MAT, 2^23 nodes, 16 * 2^23 draws, quadrant probabilities
(0.57, 0.19, 0.19, 0.05), no noise, L = 8 uniform node types
(``synth.rmat_23()``, seeded; self-loops and duplicates removed by the
oracle's own graph builder).  Counts: induced typed graphlets by type
multiset (Def. "Typed Graphlet Instance"; global counts as in Sec. "Global
Typed Graphlet Counts"), in the library's global layout
[edges][h1][h2][h3..h8], each block in colex order of the sorted multiset.

This script calls only ``oracle.o2`` (plus the seeded input generator); no
value comes from the CUDA library.  It takes hours of CPU time:

    python tests/golden/make_rmat23_o2.py [--threads T]
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "rmat23_o2_global.txt")


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--scale", type=int, default=23)
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args()

    import numpy as np

    from oracle import o2
    from paper_1901_10026_gb300 import synth

    t0 = time.time()
    G = synth.rmat_23(scale=args.scale)
    gen_s = time.time() - t0
    t0 = time.time()
    h = o2.global_counts_of(G, 4, threads=args.threads)
    o2_s = time.time() - t0
    L = G.L
    n_edge_block = L * (L + 1) // 2
    M = int(h[:n_edge_block].sum())
    digest = hashlib.sha256(np.ascontiguousarray(h, dtype="<u8").tobytes()).hexdigest()
    threads = args.threads or o2.max_threads()
    with open(args.out, "w") as f:
        f.write(f"# R-MAT scale {args.scale}, edge factor 16, (0.57, 0.19, 0.19, 0.05), L = {L} uniform types\n")
        f.write(f"# generator: paper_1901_10026_gb300.synth.rmat_23(scale={args.scale})\n")
        f.write(f"# n = {G.n}, draws = {G.m}, M = {M} (edges after simplification)\n")
        f.write(f"# written by tests/golden/make_rmat23_o2.py from oracle.o2 alone "
                f"({o2_s:.0f} s on {threads} host threads)\n")
        f.write(f"# entries = {h.shape[0]}, sha256(little-endian uint64) = {digest}\n")
        for x in h:
            f.write(f"{int(x)}\n")
    print(f"wrote {args.out}: M={M} entries={h.shape[0]} gen {gen_s:.0f} s, o2 {o2_s:.0f} s")
    return 0


if __name__ == "__main__":
    sys.exit(main())
