/*
 * Second CPU oracle: global typed 3- and 4-node graphlet counts by a route
 * that is independent of the paper's per-edge method (Rossi et al.,
 * "Heterogeneous Network Motifs", arXiv 1901.10026).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests load it.  It shares no code,
 * header or helper with the first oracle (tg_oracle.c) or with the CUDA
 * library, and calls neither.
 *
 * What it computes: for every sorted multiset of node types, the number of
 * induced 2-, 3- and 4-node connected subgraphs of each shape (Def. "Typed
 * Graphlet Instance"; global counts as in Sec. "Global Typed Graphlet
 * Counts").  It does not follow Alg. 1-3.  Instead it counts NON-induced
 * copies of each pattern on a node set (subgraphs, not induced subgraphs),
 * with textbook methods, and then inverts the standard containment
 * multiplicities.  All copies of a pattern inside one 4-node set share that
 * set's type multiset, so the inversion holds per multiset:
 *
 *   non-induced counts N_X, per multiset
 *     edges   one per edge
 *     P3      per centre v, pairs of leaves from the typed degrees of v
 *     tri     per edge (u,v), common neighbours by type; each triangle is
 *             seen from its three edges, so the sum is divided by 3
 *     S4      per centre v, triples of leaves from the typed degrees
 *     P4      per middle edge (u,v): x in G(u)\{v}, y in G(v)\{u}, x != y,
 *             from typed degrees, minus the x = y (common neighbour) pairs
 *     C4      per node a of highest degree rank in the cycle: typed counts
 *             c_t(a,b) of wedges a-u-b with u, b ranked below a; pairs of
 *             such wedges close one 4-cycle each
 *     TT      per triangle {u,v,w} and tail vertex w: the neighbours of w
 *             other than u, v (counted from edge (u,v) with apex w)
 *     D       per diagonal edge (u,v): pairs of common neighbours
 *     K4      oriented by degree rank, each clique once from its lowest node
 *
 *   induced counts (multiplicities of spanning subgraphs of 4-node graphs)
 *     K4 = N_K4
 *     D  = N_D  - 6 K4
 *     TT = N_TT - 4 D - 12 K4
 *     C4 = N_C4 - D - 3 K4
 *     S4 = N_S4 - TT - 2 D - 4 K4
 *     P4 = N_P4 - 2 TT - 4 C4 - 6 D - 12 K4
 *     P3 = N_P3 - 3 tri
 *
 * Arithmetic is uint64 modulo 2^64; every true count is below 2^64, so the
 * differences are exact.
 *
 * Graphlet ids follow the paper (h3 4-path, h4 4-star, h5 4-cycle, h6 tailed
 * triangle, h7 chordal cycle, h8 4-clique; h1 3-path, h2 triangle).  Output:
 *     [edge: C(L+1,2)][h1: C(L+2,3)][h2: C(L+2,3)][h3..h8: C(L+3,4) each]
 * (k = 3 stops after h2), each block indexed by the colex rank of the sorted
 * type multiset c_1 <= ... <= c_k, i.e. sum over m of C(c_m + m - 1, m).
 *
 * Graph input: self-loops are dropped, duplicate and reversed edges merged.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static uint64_t binom2(uint64_t a, int b) {
    /* C(a, b) for small b by the product formula (exact: each prefix is a
       binomial coefficient) */
    if ((int64_t)a < b) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= b; ++i) r = r * (a - (uint64_t)b + (uint64_t)i) / (uint64_t)i;
    return r;
}

static void sort_small_u8(int *c, int k) {
    for (int i = 1; i < k; ++i) {
        int x = c[i], j = i - 1;
        while (j >= 0 && c[j] > x) {
            c[j + 1] = c[j];
            --j;
        }
        c[j + 1] = x;
    }
}

/* colex rank of a multiset of k types (any order on input) */
static int64_t mrank(const int *types, int k) {
    int c[4];
    for (int i = 0; i < k; ++i) c[i] = types[i];
    sort_small_u8(c, k);
    int64_t r = 0;
    for (int m = 1; m <= k; ++m) r += (int64_t)binom2((uint64_t)(c[m - 1] + m - 1), m);
    return r;
}

static int64_t r2(int a, int b) {
    int c[2] = {a, b};
    return mrank(c, 2);
}
static int64_t r3(int a, int b, int d) {
    int c[3] = {a, b, d};
    return mrank(c, 3);
}
static int64_t r4(int a, int b, int d, int e) {
    int c[4] = {a, b, d, e};
    return mrank(c, 4);
}

typedef struct {
    int64_t n, M;
    int L;
    int64_t *off;   /* n+1 */
    int32_t *adj;   /* 2M, each row sorted by id */
    uint8_t *type;  /* n */
    int64_t *rnk;   /* degree rank: position in (degree, id) ascending order */
    int64_t *dt;    /* n*L typed degrees */
    int64_t *uoff;  /* n+1: neighbours of higher degree rank ("up" lists) */
    int32_t *up;    /* M */
} G2;

static int cmp_u64(const void *a, const void *b) {
    const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

static const G2 *g_sort_graph;
static int cmp_deg_id(const void *a, const void *b) {
    const int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    const int64_t dx = g_sort_graph->off[x + 1] - g_sort_graph->off[x];
    const int64_t dy = g_sort_graph->off[y + 1] - g_sort_graph->off[y];
    if (dx != dy) return dx < dy ? -1 : 1;
    return x < y ? -1 : x > y;
}

static void g2_free(G2 *g) {
    free(g->off);
    free(g->adj);
    free(g->type);
    free(g->rnk);
    free(g->dt);
    free(g->uoff);
    free(g->up);
}

static int g2_build(G2 *g, int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                    const uint8_t *types, int L) {
    memset(g, 0, sizeof(*g));
    if (n < 0 || m < 0 || L < 1 || L > 16 || n >= ((int64_t)1 << 31)) return -1;
    for (int64_t v = 0; v < n; ++v)
        if (types[v] >= L) return -1;
    uint64_t *key = (uint64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
    if (!key) return -1;
    int64_t q = 0;
    for (int64_t e = 0; e < m; ++e) {
        const int64_t a = src[e], b = dst[e];
        if (a < 0 || b < 0 || a >= n || b >= n) {
            free(key);
            return -1;
        }
        if (a == b) continue;
        const uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
        key[q++] = (lo << 32) | hi;
    }
    qsort(key, (size_t)q, sizeof(uint64_t), cmp_u64);
    int64_t M = 0;
    for (int64_t e = 0; e < q; ++e)
        if (e == 0 || key[e] != key[e - 1]) key[M++] = key[e];
    g->n = n;
    g->M = M;
    g->L = L;
    g->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->adj = (int32_t *)malloc((size_t)(2 * M > 0 ? 2 * M : 1) * sizeof(int32_t));
    g->type = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    g->rnk = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    g->dt = (int64_t *)calloc((size_t)(n > 0 ? n : 1) * (size_t)L, sizeof(int64_t));
    int64_t *fill = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!g->off || !g->adj || !g->type || !g->rnk || !g->dt || !fill || !order) {
        free(key);
        free(fill);
        free(order);
        g2_free(g);
        return -1;
    }
    memcpy(g->type, types, (size_t)n);
    for (int64_t e = 0; e < M; ++e) {
        ++g->off[(key[e] >> 32) + 1];
        ++g->off[(key[e] & 0xffffffffu) + 1];
    }
    for (int64_t v = 0; v < n; ++v) g->off[v + 1] += g->off[v];
    for (int64_t v = 0; v < n; ++v) fill[v] = g->off[v];
    /* pairs ascending by (lo, hi): row w receives its smaller neighbours
       (as hi) before its larger ones (as lo), each ascending */
    for (int64_t e = 0; e < M; ++e) {
        const int64_t a = (int64_t)(key[e] >> 32), b = (int64_t)(key[e] & 0xffffffffu);
        g->adj[fill[a]++] = (int32_t)b;
        g->adj[fill[b]++] = (int32_t)a;
    }
    for (int64_t v = 0; v < n; ++v) {
        order[v] = v;
        for (int64_t p = g->off[v]; p < g->off[v + 1]; ++p) ++g->dt[v * L + g->type[g->adj[p]]];
    }
    g_sort_graph = g;
    qsort(order, (size_t)n, sizeof(int64_t), cmp_deg_id);
    for (int64_t r = 0; r < n; ++r) g->rnk[order[r]] = r;
    g->uoff = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->up = (int32_t *)malloc((size_t)(M > 0 ? M : 1) * sizeof(int32_t));
    if (!g->uoff || !g->up) {
        free(key);
        free(fill);
        free(order);
        g2_free(g);
        return -1;
    }
    for (int64_t v = 0; v < n; ++v) {
        g->uoff[v + 1] = g->uoff[v];
        for (int64_t p = g->off[v]; p < g->off[v + 1]; ++p)
            if (g->rnk[g->adj[p]] > g->rnk[v]) g->up[g->uoff[v + 1]++] = g->adj[p];
    }
    free(key);
    free(fill);
    free(order);
    return 0;
}

enum { N_EDGE, N_P3, N_TRI3, N_S4, N_P4, N_C4, N_TT, N_D, N_K4, N_KINDS };

int tgo2_global_len(int L, int k) {
    if (L < 1 || (k != 3 && k != 4)) return -1;
    int64_t len = (int64_t)binom2((uint64_t)L + 1, 2) + 2 * (int64_t)binom2((uint64_t)L + 2, 3);
    if (k == 4) len += 6 * (int64_t)binom2((uint64_t)L + 3, 4);
    return (int)len;
}

int tgo2_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int tgo2_count_global(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                      const uint8_t *types, int L, int k, uint64_t *out, int threads) {
    if (k != 3 && k != 4) return -1;
    G2 g;
    if (g2_build(&g, n, m, src, dst, types, L) != 0) return -1;
    const int64_t len2 = (int64_t)binom2((uint64_t)L + 1, 2);
    const int64_t len3 = (int64_t)binom2((uint64_t)L + 2, 3);
    const int64_t len4 = (int64_t)binom2((uint64_t)L + 3, 4);
    const int64_t lens[N_KINDS] = {len2, len3, len3, len4, len4, len4, len4, len4, len4};
    int64_t base[N_KINDS + 1];
    base[0] = 0;
    for (int i = 0; i < N_KINDS; ++i) base[i + 1] = base[i] + lens[i];
    const int64_t H = base[N_KINDS];
#ifdef _OPENMP
    int nt = threads > 0 ? threads : omp_get_max_threads();
#else
    int nt = 1;
    (void)threads;
#endif
    uint64_t *acc = (uint64_t *)calloc((size_t)nt * (size_t)H, sizeof(uint64_t));
    if (!acc) {
        g2_free(&g);
        return -1;
    }
    int failed = 0;
    const int four = (k == 4);
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
#ifdef _OPENMP
        const int tid = omp_get_thread_num();
#else
        const int tid = 0;
#endif
        uint64_t *h = acc + (size_t)tid * (size_t)H;
        int64_t *stamp = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        int64_t *stamp2 = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        uint32_t *cnt = four ? (uint32_t *)calloc((size_t)(n > 0 ? n : 1) * (size_t)L, 4) : NULL;
        int64_t *touched = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        int64_t *wlist = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        if (!stamp || !stamp2 || (four && !cnt) || !touched || !wlist) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        } else {
            for (int64_t v = 0; v < n; ++v) stamp[v] = stamp2[v] = -1;
        }
        const int ok = stamp && stamp2 && (!four || cnt) && touched && wlist;
        int64_t Tt[16];
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t u = 0; u < n; ++u) {
            if (!ok) continue;
            const int pu = g.type[u];
            const int64_t *du = g.dt + u * L;
            /* node-centred stars: pairs (P3) and triples (S4) of leaves */
            for (int t = 0; t < L; ++t)
                for (int s = t; s < L; ++s) {
                    const uint64_t c = (s == t) ? binom2((uint64_t)du[t], 2)
                                                : (uint64_t)du[t] * (uint64_t)du[s];
                    if (c) h[base[N_P3] + r3(pu, t, s)] += c;
                    if (!four) continue;
                    for (int r = s; r < L; ++r) {
                        uint64_t c3;
                        if (t == s && s == r) c3 = binom2((uint64_t)du[t], 3);
                        else if (t == s) c3 = binom2((uint64_t)du[t], 2) * (uint64_t)du[r];
                        else if (s == r) c3 = (uint64_t)du[t] * binom2((uint64_t)du[s], 2);
                        else c3 = (uint64_t)du[t] * (uint64_t)du[s] * (uint64_t)du[r];
                        if (c3) h[base[N_S4] + r4(pu, t, s, r)] += c3;
                    }
                }
            /* edges (u,v) with v ranked below u: each edge exactly once */
            for (int64_t p = g.off[u]; p < g.off[u + 1]; ++p) stamp[g.adj[p]] = u;
            for (int64_t p = g.off[u]; p < g.off[u + 1]; ++p) {
                const int64_t v = g.adj[p];
                if (g.rnk[v] > g.rnk[u]) continue;
                const int pv = g.type[v];
                const int64_t *dv = g.dt + v * L;
                h[base[N_EDGE] + r2(pu, pv)] += 1;
                for (int t = 0; t < L; ++t) Tt[t] = 0;
                for (int64_t q = g.off[v]; q < g.off[v + 1]; ++q) {
                    const int64_t w = g.adj[q];
                    if (stamp[w] != u) continue;  /* w is a common neighbour */
                    const int pw = g.type[w];
                    ++Tt[pw];
                    if (!four) continue;
                    /* tailed triangles with the tail at w (edge (u,v) opposite) */
                    const int64_t *dw = g.dt + w * L;
                    for (int t = 0; t < L; ++t) {
                        const int64_t c = dw[t] - (pu == t) - (pv == t);
                        if (c > 0) h[base[N_TT] + r4(pu, pv, pw, t)] += (uint64_t)c;
                    }
                }
                for (int t = 0; t < L; ++t)
                    if (Tt[t]) h[base[N_TRI3] + r3(pu, pv, t)] += (uint64_t)Tt[t];
                if (!four) continue;
                for (int t = 0; t < L; ++t) {
                    /* diamonds with diagonal (u,v): pairs of common neighbours */
                    if (Tt[t] > 1) h[base[N_D] + r4(pu, pv, t, t)] += binom2((uint64_t)Tt[t], 2);
                    for (int s = t + 1; s < L; ++s)
                        if (Tt[t] && Tt[s])
                            h[base[N_D] + r4(pu, pv, t, s)] += (uint64_t)Tt[t] * (uint64_t)Tt[s];
                    /* 4-paths x-u-v-y with middle edge (u,v) */
                    const int64_t xu = du[t] - (pv == t);
                    for (int s = 0; s < L; ++s) {
                        const int64_t yv = dv[s] - (pu == s);
                        int64_t c = xu * yv - (s == t ? Tt[t] : 0);
                        if (c > 0) h[base[N_P4] + r4(pu, pv, t, s)] += (uint64_t)c;
                    }
                }
            }
            if (!four) continue;
            /* 4-cycles whose highest-ranked node is u: wedges u-w-b with w and
               b ranked below u, counted by the type of w */
            int64_t nb = 0;
            for (int64_t p = g.off[u]; p < g.off[u + 1]; ++p) {
                const int64_t w = g.adj[p];
                if (g.rnk[w] > g.rnk[u]) continue;
                const int pw = g.type[w];
                for (int64_t q = g.off[w]; q < g.off[w + 1]; ++q) {
                    const int64_t b = g.adj[q];
                    if (b == u || g.rnk[b] > g.rnk[u]) continue;
                    uint32_t *cb = cnt + (size_t)b * (size_t)L;
                    int any = 0;
                    for (int t = 0; t < L; ++t) any |= (cb[t] != 0);
                    if (!any) touched[nb++] = b;
                    ++cb[pw];
                }
            }
            for (int64_t z = 0; z < nb; ++z) {
                const int64_t b = touched[z];
                const int pb = g.type[b];
                uint32_t *cb = cnt + (size_t)b * (size_t)L;
                for (int t = 0; t < L; ++t) {
                    if (cb[t] > 1) h[base[N_C4] + r4(pu, pb, t, t)] += binom2(cb[t], 2);
                    for (int s = t + 1; s < L; ++s)
                        if (cb[t] && cb[s])
                            h[base[N_C4] + r4(pu, pb, t, s)] += (uint64_t)cb[t] * (uint64_t)cb[s];
                }
                for (int t = 0; t < L; ++t) cb[t] = 0;
            }
            /* 4-cliques {u < v < w < x} in degree rank, from u, along up lists */
            for (int64_t p = g.uoff[u]; p < g.uoff[u + 1]; ++p) {
                const int64_t v = g.up[p];
                /* W = common neighbours of u and v ranked above v */
                int64_t nw = 0;
                for (int64_t q = g.uoff[v]; q < g.uoff[v + 1]; ++q) {
                    const int64_t w = g.up[q];
                    if (stamp[w] == u) {
                        wlist[nw++] = w;
                        stamp2[w] = v;
                    }
                }
                for (int64_t a = 0; a < nw; ++a) {
                    const int64_t w = wlist[a];
                    for (int64_t q = g.uoff[w]; q < g.uoff[w + 1]; ++q) {
                        const int64_t x = g.up[q];
                        if (stamp2[x] == v)
                            h[base[N_K4] + r4(pu, g.type[v], g.type[w], g.type[x])] += 1;
                    }
                }
                for (int64_t a = 0; a < nw; ++a) stamp2[wlist[a]] = -1;
            }
        }
        free(stamp);
        free(stamp2);
        free(cnt);
        free(touched);
        free(wlist);
    }
    if (failed) {
        free(acc);
        g2_free(&g);
        return -1;
    }
    for (int t = 1; t < nt; ++t)
        for (int64_t i = 0; i < H; ++i) acc[i] += acc[(size_t)t * (size_t)H + i];
    const uint64_t *N = acc;
    /* triangles: each seen once from each of its three edges */
    int rc = 0;
    for (int64_t r = 0; r < len3; ++r)
        if (N[base[N_TRI3] + r] % 3) rc = -2;
    uint64_t *o = out;
    memcpy(o, N + base[N_EDGE], (size_t)len2 * 8);
    for (int64_t r = 0; r < len3; ++r) {
        const uint64_t tri = N[base[N_TRI3] + r] / 3;
        o[len2 + r] = N[base[N_P3] + r] - 3 * tri;
        o[len2 + len3 + r] = tri;
    }
    if (four) {
        uint64_t *h4 = o + len2 + 2 * len3;
        for (int64_t r = 0; r < len4; ++r) {
            const uint64_t K4 = N[base[N_K4] + r];
            const uint64_t D = N[base[N_D] + r] - 6 * K4;
            const uint64_t TT = N[base[N_TT] + r] - 4 * D - 12 * K4;
            const uint64_t C4 = N[base[N_C4] + r] - D - 3 * K4;
            const uint64_t S4 = N[base[N_S4] + r] - TT - 2 * D - 4 * K4;
            const uint64_t P4 = N[base[N_P4] + r] - 2 * TT - 4 * C4 - 6 * D - 12 * K4;
            h4[0 * len4 + r] = P4;  /* h3 */
            h4[1 * len4 + r] = S4;  /* h4 */
            h4[2 * len4 + r] = C4;  /* h5 */
            h4[3 * len4 + r] = TT;  /* h6 */
            h4[4 * len4 + r] = D;   /* h7 */
            h4[5 * len4 + r] = K4;  /* h8 */
        }
    }
    free(acc);
    g2_free(&g);
    return rc;
}
