"""Brute-force typed graphlet counts straight from the definitions.

Test infrastructure only.  For every 3- and 4-node subset of a tiny graph it
checks that the induced subgraph is connected (Def. "Untyped Graphlet"),
identifies the graphlet by its edge count and degree sequence, keys it by the
sorted multiset of node types (Def. "Typed Graphlet Instance", condition 2),
and credits each of its edges with the edge's orbit (Table 2: the position of
the edge in the graphlet, read off the two endpoint degrees inside the
subgraph).  Pure Python loops: only for graphs of a dozen or so nodes.

Orbit ids follow Table 2: g1 3-path, g2 triangle, g3 4-path end edge, g4
4-path centre edge, g5 4-star, g6 4-cycle, g7 tailed-triangle tail edge, g8
tailed-triangle edge opposite the degree-3 node, g9 tailed-triangle edge at the
degree-3 node, g10 chordal-cycle outer edge, g11 chordal-cycle chord, g12
4-clique.  Graphlets: h1 3-path, h2 triangle, h3 4-path, h4 4-star, h5 4-cycle,
h6 tailed triangle, h7 chordal cycle, h8 4-clique.
"""
from __future__ import annotations

import itertools
from collections import defaultdict

ORBIT_GRAPHLET = {1: 1, 2: 2, 3: 3, 4: 3, 5: 4, 6: 5, 7: 6, 8: 6, 9: 6, 10: 7, 11: 7, 12: 8}
EDGES_OF = {1: 2, 2: 3, 3: 3, 4: 3, 5: 4, 6: 4, 7: 5, 8: 6}


def simple_graph(n, src, dst):
    adj = [set() for _ in range(n)]
    for a, b in zip(src, dst):
        a, b = int(a), int(b)
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    edges = sorted({(min(a, b), max(a, b)) for a in range(n) for b in adj[a]})
    return adj, edges


def _connected(nodes, adj):
    nodes = list(nodes)
    seen = {nodes[0]}
    stack = [nodes[0]]
    s = set(nodes)
    while stack:
        x = stack.pop()
        for y in adj[x]:
            if y in s and y not in seen:
                seen.add(y)
                stack.append(y)
    return len(seen) == len(s)


def _orbit(sub_edges, deg, e):
    """Orbit id of edge e inside the induced graphlet (Table 2)."""
    k = len(deg)
    m = len(sub_edges)
    a, b = deg[e[0]], deg[e[1]]
    lo, hi = min(a, b), max(a, b)
    if k == 3:
        return 1 if m == 2 else 2
    if m == 3:
        if max(deg.values()) == 3:
            return 5
        return 3 if lo == 1 else 4
    if m == 4:
        if max(deg.values()) == 2:
            return 6
        if lo == 1:
            return 7
        return 8 if hi == 2 else 9
    if m == 5:
        return 11 if lo == 3 else 10
    return 12


def per_edge_orbits(n, src, dst, types, kmax=4):
    """{edge: {(orbit, key): count}} where key = sorted types of the other nodes."""
    adj, edges = simple_graph(n, src, dst)
    out = {e: defaultdict(int) for e in edges}
    for k in range(3, kmax + 1):
        for nodes in itertools.combinations(range(n), k):
            if not _connected(nodes, adj):
                continue
            sub = [(a, b) for a, b in itertools.combinations(nodes, 2) if b in adj[a]]
            deg = {v: 0 for v in nodes}
            for a, b in sub:
                deg[a] += 1
                deg[b] += 1
            for e in sub:
                g = _orbit(sub, deg, e)
                rest = tuple(sorted(int(types[v]) for v in nodes if v not in e))
                out[e][(g, rest)] += 1
    return edges, out


def global_graphlets(n, src, dst, types, kmax=4):
    """{(graphlet, sorted type multiset): number of induced instances} (+ edges as h0)."""
    adj, edges = simple_graph(n, src, dst)
    out = defaultdict(int)
    for a, b in edges:
        out[(0, tuple(sorted((int(types[a]), int(types[b])))))] += 1
    for k in range(3, kmax + 1):
        for nodes in itertools.combinations(range(n), k):
            if not _connected(nodes, adj):
                continue
            sub = [(a, b) for a, b in itertools.combinations(nodes, 2) if b in adj[a]]
            deg = {v: 0 for v in nodes}
            for a, b in sub:
                deg[a] += 1
                deg[b] += 1
            g = _orbit(sub, deg, sub[0])
            h = ORBIT_GRAPHLET[g]
            out[(h, tuple(sorted(int(types[v]) for v in nodes)))] += 1
    return dict(out)
