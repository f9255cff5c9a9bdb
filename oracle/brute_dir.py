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
