"""Row and histogram layouts, re-derived in plain Python for the tests.

Per-edge rows (k = 4): [x1: L][x2: L][x3: P]...; P = L(L+1)/2 type pairs (t, t')
with t <= t' in lexicographic order.  Global histogram blocks are indexed by the
colex order of sorted type multisets (compare the largest element first), which
the tests derive here by sorting, not by the rank formula.
"""
from __future__ import annotations

import itertools
from math import comb

EDGES_OF_GRAPHLET = {1: 2, 2: 3, 3: 3, 4: 3, 5: 4, 6: 4, 7: 5, 8: 6}
ORBIT_TO_GRAPHLET = {1: 1, 2: 2, 3: 3, 4: 3, 5: 4, 6: 5, 7: 6, 8: 6, 9: 6, 10: 7, 11: 7, 12: 8}


def pairs(L):
    return [(t, u) for t in range(L) for u in range(t, L)]


def multisets(L, k):
    """All sorted k-multisets over [0, L) in colex order."""
    ms = list(itertools.combinations_with_replacement(range(L), k))
    return sorted(ms, key=lambda m: tuple(reversed(m)))


def colex_index(L, k):
    return {m: r for r, m in enumerate(multisets(L, k))}


def row_width(L, k=4, level="graphlet"):
    if k == 3:
        return 2 * L
    return 2 * L + (10 if level == "orbit" else 6) * (L * (L + 1) // 2)


def decode_orbit_row(row, L):
    """{(orbit, key)} -> count, key = (t,) for 3-node orbits, (t, t') for 4-node."""
    P = L * (L + 1) // 2
    out = {}
    for t in range(L):
        if row[t]:
            out[(1, (t,))] = int(row[t])
        if row[L + t]:
            out[(2, (t,))] = int(row[L + t])
    for o in range(3, 13):
        base = 2 * L + (o - 3) * P
        for p, tu in enumerate(pairs(L)):
            v = int(row[base + p])
            if v:
                out[(o, tu)] = v
    return out


def decode_graphlet_row(row, L):
    P = L * (L + 1) // 2
    out = {}
    for t in range(L):
        if row[t]:
            out[(1, (t,))] = int(row[t])
        if row[L + t]:
            out[(2, (t,))] = int(row[L + t])
    for h in range(3, 9):
        base = 2 * L + (h - 3) * P
        for p, tu in enumerate(pairs(L)):
            v = int(row[base + p])
            if v:
                out[(h, tu)] = v
    return out


def global_blocks(L, k=4):
    """[(graphlet id (0 = edge), size, offset)] of the global histogram."""
    blocks = [(0, 2, 0)]
    off = comb(L + 1, 2)
    for h in (1, 2):
        blocks.append((h, 3, off))
        off += comb(L + 2, 3)
    if k == 4:
        for h in range(3, 9):
            blocks.append((h, 4, off))
            off += comb(L + 3, 4)
    return blocks, off


def decode_global(vec, L, k=4):
    """{(graphlet, multiset)} -> count for the nonzero entries."""
    blocks, total = global_blocks(L, k)
    assert len(vec) == total
    out = {}
    for h, size, off in blocks:
        for r, m in enumerate(multisets(L, size)):
            v = int(vec[off + r])
            if v:
                out[(h, m)] = v
    return out
