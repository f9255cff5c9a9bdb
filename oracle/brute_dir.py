"""Brute-force directed typed 3-node graphlet counts (test infrastructure only).

Every 3-node subset of a tiny digraph whose underlying graph is connected is
classified by its dyad census (mutual, asymmetric and empty pairs) and, where
the census leaves a choice, by the in- and out-degrees its asymmetric arcs
give the nodes: a route independent of the relabelling search of the C
oracle.  Classes and their order: 021D (one node sends both arcs), 021U (one
node receives both), 021C (a directed 2-path), 111D (a mutual pair, the
third node sends to it), 111U (a mutual pair that sends to the third node),
030T (transitive), 030C (directed 3-cycle), 201 (two mutual pairs), 120D (a
mutual pair, the third node sends to both), 120U (a mutual pair sending to the
third node), 120C (a mutual pair and a directed 2-path through the third
node), 210, 300.  Keyed as Def. "Typed Graphlet Instance": class and sorted
multiset of node types.  Pure Python: graphs of a few dozen nodes.
"""
from __future__ import annotations

import itertools

NAMES = ("021D", "021U", "021C", "111D", "111U", "030T", "030C", "201", "120D", "120U", "120C",
         "210", "300")


def arc_set(src, dst):
    return {(int(a), int(b)) for a, b in zip(src, dst) if int(a) != int(b)}


def triad_class(nodes, arcs):
    """Index into NAMES of the induced subdigraph on three nodes, or None."""
    a, b, c = nodes
    mutual, asym = [], []
    for x, y in ((a, b), (a, c), (b, c)):
        f, r = (x, y) in arcs, (y, x) in arcs
        if f and r:
            mutual.append((x, y))
        elif f:
            asym.append((x, y))
        elif r:
            asym.append((y, x))
    if len(mutual) + len(asym) < 2:
        return None
    outd = {v: sum(1 for s, _ in asym if s == v) for v in nodes}
    ind = {v: sum(1 for _, t in asym if t == v) for v in nodes}
    nm, na = len(mutual), len(asym)
    if nm == 0 and na == 2:
        if max(outd.values()) == 2:
            return NAMES.index("021D")
        if max(ind.values()) == 2:
            return NAMES.index("021U")
        return NAMES.index("021C")
    if nm == 1 and na == 1:
        (s, t), = asym
        in_pair = set(mutual[0])
        return NAMES.index("111D") if t in in_pair else NAMES.index("111U")
    if nm == 0 and na == 3:
        return NAMES.index("030C") if all(outd[v] == 1 for v in nodes) else NAMES.index("030T")
    if nm == 2 and na == 0:
        return NAMES.index("201")
    if nm == 1 and na == 2:
        third = (set(nodes) - set(mutual[0])).pop()
        if outd[third] == 2:
            return NAMES.index("120D")
        if ind[third] == 2:
            return NAMES.index("120U")
        return NAMES.index("120C")
    if nm == 2 and na == 1:
        return NAMES.index("210")
    if nm == 3:
        return NAMES.index("300")
    raise AssertionError("unreachable triad census")


def _colex3(t):
    a, b, c = sorted(t)
    return a + (b + 1) * b // 2 + (c + 2) * (c + 1) * c // 6


def counts(n, src, dst, types, L):
    """(canonical edges, per-edge rows as lists of 13 L, global counts list)."""
    arcs = arc_set(src, dst)
    und = sorted({(min(a, b), max(a, b)) for a, b in arcs})
    adj = [set() for _ in range(n)]
    for a, b in und:
        adj[a].add(b)
        adj[b].add(a)
    eidx = {e: q for q, e in enumerate(und)}
    rows = [[0] * (13 * L) for _ in und]
    n3 = (L + 2) * (L + 1) * L // 6
    glob = [0] * (13 * n3)
    for tri in itertools.combinations(range(n), 3):
        c = triad_class(tri, arcs)
        if c is None:
            continue
        glob[c * n3 + _colex3([int(types[v]) for v in tri])] += 1
        for x, y in itertools.combinations(tri, 2):
            if y in adj[x]:
                w = (set(tri) - {x, y}).pop()
                rows[eidx[(min(x, y), max(x, y))]][c * L + int(types[w])] += 1
    return und, rows, glob


# ---------------------------------------------------------------- 4 nodes --
# Directed typed 4-node graphlets: every 4-node subset whose underlying graph
# is connected, classified by the smallest code over the 24 relabellings (the
# code of a digraph on positions 0..3 is the sum of 2^(4a + b) over its arcs
# a -> b); class c is the c-th smallest such code among the connected
# digraphs (199 of them).

_PERMS4 = list(itertools.permutations(range(4)))


def _code4(nodes, arcs):
    c = 0
    for a, x in enumerate(nodes):
        for b, y in enumerate(nodes):
            if a != b and (x, y) in arcs:
                c |= 1 << (4 * a + b)
    return c


def _canon4(code):
    best = None
    for pm in _PERMS4:
        c = 0
        for a in range(4):
            for b in range(4):
                if a != b and (code >> (4 * a + b)) & 1:
                    c |= 1 << (4 * pm[a] + pm[b])
        best = c if best is None or c < best else best
    return best


def _connected4(code):
    adj = [set() for _ in range(4)]
    for a in range(4):
        for b in range(4):
            if a != b and (code >> (4 * a + b)) & 1:
                adj[a].add(b)
                adj[b].add(a)
    seen, stack = {0}, [0]
    while stack:
        v = stack.pop()
        for w in adj[v]:
            if w not in seen:
                seen.add(w)
                stack.append(w)
    return len(seen) == 4


_CLASS4 = None


def class_table4():
    """Sorted canonical codes of the connected 4-node digraphs."""
    global _CLASS4
    if _CLASS4 is None:
        codes = set()
        for code in range(1 << 16):
            if code & 0x8421 or not _connected4(code):
                continue
            codes.add(_canon4(code))
        _CLASS4 = sorted(codes)
    return _CLASS4


def counts4(n, src, dst, types, L):
    """(canonical edges, per-edge rows as lists of 199 P, global counts list)."""
    table = {c: q for q, c in enumerate(class_table4())}
    arcs = arc_set(src, dst)
    und = sorted({(min(a, b), max(a, b)) for a, b in arcs})
    eidx = {e: q for q, e in enumerate(und)}
    P = L * (L + 1) // 2
    rows = [[0] * (199 * P) for _ in und]
    n4 = (L + 3) * (L + 2) * (L + 1) * L // 24

    def colex4(t):
        a, b, c, d = sorted(t)
        return a + (b + 1) * b // 2 + (c + 2) * (c + 1) * c // 6 + (d + 3) * (d + 2) * (d + 1) * d // 24

    glob = [0] * (199 * n4)
    for quad in itertools.combinations(range(n), 4):
        code = _code4(quad, arcs)
        if not _connected4(code):
            continue
        c = table[_canon4(code)]
        glob[c * n4 + colex4([int(types[v]) for v in quad])] += 1
        for x, y in itertools.combinations(quad, 2):
            if (min(x, y), max(x, y)) in eidx:
                t, u = sorted(int(types[v]) for v in quad if v not in (x, y))
                rows[eidx[(min(x, y), max(x, y))]][c * P + t * L - t * (t - 1) // 2 + (u - t)] += 1
    return und, rows, glob
