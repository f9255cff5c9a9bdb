"""The algebra the CUDA counting path is built on, checked on the CPU against
the paper-method oracle (plain Python, no CUDA code).

For an edge (i, j) with d_i <= d_j, every enumerated orbit of Alg. 2-3 is
written through Alg. 1's typed triangle counts tau, per-node sums Theta and D,
sums over the triangle nodes T (B, C, DT), the ordered non-induced 4-cycle
pairs C4 and the adjacent pairs inside T (Q); g4, g5, g9, g11 keep the closed
forms of Sec. "Combinatorial Relationships".  For global counts Q and C4 may
be dropped per edge and added back through the type-multiset totals of
4-cliques and non-induced 4-cycles.  Both are compared here with the oracle.
"""
import itertools
from math import comb

import numpy as np
import pytest

from paper_1901_10026_gb300 import synth
from tests import layout


def _graph(G):
    n, L = G.n, G.L
    adj = [set() for _ in range(n)]
    for a, b in zip(G.src, G.dst):
        if a != b:
            adj[int(a)].add(int(b))
            adj[int(b)].add(int(a))
    return adj, [int(t) for t in G.types]


def _identity_rows(G, adj, ty, drop_q_c4=False):
    """Per-edge orbit rows (canonical edge order) from the identities."""
    n, L = G.n, G.L
    deg = [len(x) for x in adj]
    edges = sorted((a, b) for a in range(n) for b in adj[a] if a < b)

    def tau(a, b):
        out = np.zeros(L, np.int64)
        for w in adj[a] & adj[b]:
            out[ty[w]] += 1
        return out

    def dvec(w):
        out = np.zeros(L, np.int64)
        for z in adj[w]:
            out[ty[z]] += 1
        return out

    theta = np.zeros((n, L, L), np.int64)
    dv = np.zeros((n, L, L), np.int64)
    for x in range(n):
        for w in adj[x]:
            theta[x, ty[w]] += tau(x, w)
            dv[x, ty[w]] += dvec(w)
    rows = []
    for a, b in edges:
        i, j = (a, b) if deg[a] <= deg[b] else (b, a)
        ti, tj = ty[i], ty[j]
        T = adj[i] & adj[j]
        Tn = np.bincount([ty[w] for w in T], minlength=L)
        Si = np.bincount([ty[w] for w in adj[i] - T - {j}], minlength=L)
        Sj = np.bincount([ty[w] for w in adj[j] - T - {i}], minlength=L)
        B = np.zeros((L, L), np.int64)
        C = B.copy()
        DT = B.copy()
        Q = B.copy()
        C4 = B.copy()
        for y in T:
            B[ty[y]] += tau(j, y)
            C[ty[y]] += tau(i, y)
            DT[ty[y]] += dvec(y)
        if not drop_q_c4:
            for y in T:
                for z in adj[y] & T:
                    Q[ty[y], ty[z]] += 1
            for x in adj[i] - {j}:
                for w in adj[x] & adj[j]:
                    if w != i:
                        C4[ty[x], ty[w]] += 1
        Ai = np.zeros((L, L), np.int64)
        Ai[:, ti] = Tn
        Aj = np.zeros((L, L), np.int64)
        Aj[:, tj] = Tn
        S6 = C4 - B + Ai
        TSj, TSi = B - Q - Ai, C - Q - Aj
        Ei = np.zeros((L, L), np.int64)
        Ei[ti, :] = Tn
        Ej = np.zeros((L, L), np.int64)
        Ej[tj, :] = Tn
        SSj, SSi = theta[j] - B - Ei, theta[i] - C - Ej
        Di = np.zeros((L, L), np.int64)
        Di[ti, :] = dvec(i)
        Dj = np.zeros((L, L), np.int64)
        Dj[tj, :] = dvec(j)
        DSj, DSi = dv[j] - DT - Di, dv[i] - DT - Dj
        SjSj, SiSi, G6 = SSj - TSj.T, SSi - TSi.T, S6 - TSi.T
        Bi = np.zeros((L, L), np.int64)
        Bi[:, ti] = Si
        Bj = np.zeros((L, L), np.int64)
        Bj[:, tj] = Sj
        Y = DSi - Bi - SSi - G6 + DSj - Bj - SSj - G6.T
        Z = DT - Ai - Aj - Q - TSi - TSj
        P = L * (L + 1) // 2
        row = np.zeros(2 * L + 10 * P, np.int64)
        row[:L] = Si + Sj
        row[L:2 * L] = Tn
        sym = lambda X, t, u: X[t, u] if t == u else X[t, u] + X[u, t]
        c2 = lambda x: x * (x - 1) // 2
        for pr, (t, u) in enumerate(layout.pairs(L)):
            s7 = sym(SiSi + SjSj, t, u)
            assert s7 % 2 == 0
            g12, g10, g7 = sym(Q, t, u) // 2, sym(TSi + TSj, t, u), s7 // 2
            g6, g3, g8 = sym(G6, t, u), sym(Y, t, u), sym(Z, t, u)
            if t == u:
                g4 = Si[t] * Sj[t] - g6
                g5 = c2(Si[t]) + c2(Sj[t]) - g7
                g9 = Tn[t] * (Si[t] + Sj[t]) - g10
                g11 = c2(Tn[t]) - g12
            else:
                g4 = Si[t] * Sj[u] + Si[u] * Sj[t] - g6
                g5 = Si[t] * Si[u] + Sj[t] * Sj[u] - g7
                g9 = Tn[t] * (Si[u] + Sj[u]) + Tn[u] * (Si[t] + Sj[t]) - g10
                g11 = Tn[t] * Tn[u] - g12
            for o, val in enumerate((g3, g4, g5, g6, g7, g8, g9, g10, g11, g12)):
                row[2 * L + o * P + pr] = val
        rows.append((ti, tj, row))
    return rows


def _cases(count, seed):
    g = synth.rng(950, seed)
    return [synth.tiny_random(int(g.integers(4, 16)), float(g.uniform(0.2, 0.9)), int(g.integers(1, 4)), g)
            for _ in range(count)]


@pytest.mark.parametrize("seed", [0, 1])
def test_per_edge_identities_equal_the_oracle(oracle_mod, seed):
    for G in _cases(12, seed):
        adj, ty = _graph(G)
        og = oracle_mod.OracleGraph.from_edges(G)
        want = og.per_edge(k=4, level="orbit").astype(np.int64)
        got = np.array([r for _, _, r in _identity_rows(G, adj, ty)]).reshape(want.shape)
        assert np.array_equal(got, want), G.name


@pytest.mark.parametrize("seed", [2, 3])
def test_global_shortcut_equals_the_oracle(oracle_mod, seed):
    for G in _cases(10, seed):
        adj, ty = _graph(G)
        L = G.L
        blocks, total = layout.global_blocks(L, 4)
        off = {h: o for h, _, o in blocks}
        idx = {s: layout.colex_index(L, s) for s in (2, 3, 4)}
        hist = np.zeros(total, np.int64)
        for ti, tj, row in _identity_rows(G, adj, ty, drop_q_c4=True):
            P = L * (L + 1) // 2
            hist[off[0] + idx[2][tuple(sorted((ti, tj)))]] += 1
            for t in range(L):
                hist[off[1] + idx[3][tuple(sorted((ti, tj, t)))]] += row[t]
                hist[off[2] + idx[3][tuple(sorted((ti, tj, t)))]] += row[L + t]
            for pr, (t, u) in enumerate(layout.pairs(L)):
                g = [row[2 * L + o * P + pr] for o in range(10)]
                key = idx[4][tuple(sorted((ti, tj, t, u)))]
                for h, v in zip(range(3, 9), (g[0] + g[1], g[2], g[3], g[4] + g[5] + g[6], g[7] + g[8], g[9])):
                    hist[off[h] + key] += v
        # the dropped terms, from the type-multiset totals (brute force here)
        nc4 = np.zeros(comb(L + 3, 4), np.int64)
        k4 = nc4.copy()
        for quad in itertools.combinations(range(G.n), 4):
            key = idx[4][tuple(sorted(ty[x] for x in quad))]
            a, b, c, d = quad
            for p, q, r, s in ((a, b, c, d), (a, b, d, c), (a, c, b, d)):
                if q in adj[p] and r in adj[q] and s in adj[r] and p in adj[s]:
                    nc4[key] += 1
            if all(y in adj[x] for x, y in itertools.combinations(quad, 2)):
                k4[key] += 1
        for h, cc4, ck4 in ((3, -12, -36), (4, 0, -12), (5, 4, 12), (6, 0, 48), (7, 0, -30), (8, 0, 6)):
            hist[off[h]:off[h] + len(nc4)] += cc4 * nc4 + ck4 * k4
        div = {0: 1, 1: 2, 2: 3, 3: 3, 4: 3, 5: 4, 6: 4, 7: 5, 8: 6}
        out = np.zeros(total, np.int64)
        for h, size, o in blocks:
            ln = comb(L + size - 1, size)
            assert np.all(hist[o:o + ln] % div[h] == 0), (G.name, h)
            out[o:o + ln] = hist[o:o + ln] // div[h]
        assert np.array_equal(out.astype(np.uint64), oracle_mod.OracleGraph.from_edges(G).global_counts(k=4)), G.name
