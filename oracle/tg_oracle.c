/*
 * CPU oracle for exact typed 3- and 4-node graphlet counting
 * (Rossi et al., "Heterogeneous Network Motifs", arXiv 1901.10026).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark load it.  It shares no
 * code, header, table or helper with the CUDA library, and it never calls it.
 *
 * What it computes (per undirected edge (i,j) of a node-typed simple graph):
 *   - Alg. 1: mark Gamma_i (lambda_1), scan Gamma_j to split triangles T_ij
 *     (lambda_3) from 3-stars centred at j (S_j, lambda_2), then S_i =
 *     Gamma_i \ (T_ij u {j}) (Def. "Typed 3-Star Nodes Centered at i"); the
 *     typed cardinalities |T^t|, |S_i^t|, |S_j^t| give the 3-node orbits
 *     g1 (3-path, |S_i^t|+|S_j^t|, Eq. "Typed 3-Stars (for an edge)") and
 *     g2 (triangle, |T^t|).
 *   - Alg. 2 (path-based): for w_k in S_i then S_j, for w_r in Gamma_{w_k}
 *     minus {i,j}: unmarked -> g3 (4-path edge); same S-set and w_r <= w_k ->
 *     g7 (tailed-triangle tail edge); in the S_j pass, w_r in S_i -> g6
 *     (4-cycle).
 *   - Alg. 3 (triangle-based): for w_k in T, w_r in Gamma_{w_k}: w_r in T and
 *     w_r <= w_k -> g12 (4-clique); w_r in S_i u S_j -> g10 (chordal-cycle
 *     edge); unmarked and not i, j -> g8 (tailed-triangle centre).
 *   - Sec. "Combinatorial Relationships": for every type pair t <= t' the
 *     closed forms for g4 (4-path centre), g5 (4-star), g9 (tailed-triangle
 *     tri-edge) and g11 (chordal-cycle centre).
 *   - Sec. "From Typed Orbits to Graphlets": h3 = g3+g4, h4 = g5, h5 = g6,
 *     h6 = g7+g8+g9, h7 = g10+g11, h8 = g12; h1 = g1, h2 = g2.
 *   - Sec. "Global Typed Graphlet Counts", Eq. C = x^T e / |E(H)|: global
 *     counts are per-edge sums divided by the graphlet's edge count, keyed by
 *     the sorted multiset of node types (Def. "Typed Graphlet Instance").
 *
 * Readings of the text taken here (each checked against brute force in the
 * tests):
 *   - T_ij is Gamma_i intersect Gamma_j (the union written once in Sec. 4.2 is
 *     a typo; Def. "Typed Triangle Nodes" uses the intersection).
 *   - S_i excludes j (Def. "Typed 3-Star Nodes Centered at i"), although
 *     Alg. 1's S_i loop is written over Gamma_i \ T_ij.
 *   - Type pairs of enumerated orbits are unordered {phi(w_k), phi(w_r)}; the
 *     per-edge key of a 4-node orbit is (g, t, t') with t <= t', which is in
 *     bijection with the multiset {phi_i, phi_j, t, t'} once phi_i, phi_j are
 *     fixed.
 *   - "w_r <= w_k" is a symmetry break on node ids; with a simple graph
 *     w_r != w_k, so it is "<" on the original ids here.
 *   - Self-loops are dropped and duplicate or reversed edges merged.
 *
 * Per-edge row layout (orbit level, k = 4), P = L(L+1)/2 type pairs in
 * lexicographic order of (t, t'), t <= t':
 *     [g1: L][g2: L][g3: P][g4: P]...[g12: P]           (2L + 10P entries)
 * graphlet level, k = 4:
 *     [h1: L][h2: L][h3: P]...[h8: P]                   (2L + 6P entries)
 * k = 3 keeps only the first 2L entries.
 *
 * Global layout: [edge: C(L+1,2)][h1: C(L+2,3)][h2: C(L+2,3)]
 *                [h3..h8: C(L+3,4) each, k = 4 only]
 * each block indexed by the colex rank of the sorted type multiset
 * c_1 <= ... <= c_k:  rank = sum_m C(c_m + m - 1, m), m = 1..k.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n;       /* nodes */
    int64_t M;       /* undirected edges after simplification */
    int32_t L;       /* node types */
    int64_t *rowptr; /* n+1 */
    int32_t *adj;    /* 2M, each list ascending by node id */
    uint8_t *type;   /* n */
    int32_t *eu;     /* M, canonical edges: eu < ev, ascending (eu, ev) */
    int32_t *ev;
} tgo_graph;

/* ---------------------------------------------------------------- graph -- */

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

void tgo_free(tgo_graph *g) {
    if (!g) return;
    free(g->rowptr);
    free(g->adj);
    free(g->type);
    free(g->eu);
    free(g->ev);
    free(g);
}

/* Returns NULL on invalid input (id out of range, type >= L, L < 1) or OOM. */
tgo_graph *tgo_build(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                     const uint8_t *type, int32_t L) {
    if (n < 0 || m < 0 || L < 1 || L > 16) return NULL;
    for (int64_t v = 0; v < n; ++v)
        if (type[v] >= L) return NULL;
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
    if (!key) return NULL;
    int64_t k = 0;
    for (int64_t e = 0; e < m; ++e) {
        int64_t a = src[e], b = dst[e];
        if (a < 0 || a >= n || b < 0 || b >= n) { free(key); return NULL; }
        if (a == b) continue; /* self-loop dropped */
        int64_t lo = a < b ? a : b, hi = a < b ? b : a;
        key[k++] = ((uint64_t)lo << 32) | (uint64_t)hi;
    }
    qsort(key, (size_t)k, sizeof(uint64_t), cmp_u64);
    int64_t M = 0;
    for (int64_t e = 0; e < k; ++e)
        if (e == 0 || key[e] != key[e - 1]) key[M++] = key[e];

    tgo_graph *g = (tgo_graph *)calloc(1, sizeof(tgo_graph));
    if (!g) { free(key); return NULL; }
    g->n = n; g->M = M; g->L = L;
    g->rowptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * M > 0 ? 2 * M : 1));
    g->type = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    g->eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
    g->ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
    if (!g->rowptr || !g->adj || !g->type || !g->eu || !g->ev) { free(key); tgo_free(g); return NULL; }
    if (n > 0) memcpy(g->type, type, (size_t)n);
    for (int64_t e = 0; e < M; ++e) {
        g->eu[e] = (int32_t)(key[e] >> 32);
        g->ev[e] = (int32_t)(key[e] & 0xffffffffu);
        g->rowptr[g->eu[e] + 1]++;
        g->rowptr[g->ev[e] + 1]++;
    }
    free(key);
    for (int64_t v = 0; v < n; ++v) g->rowptr[v + 1] += g->rowptr[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!fill) { tgo_free(g); return NULL; }
    for (int64_t v = 0; v < n; ++v) fill[v] = g->rowptr[v];
    for (int64_t e = 0; e < M; ++e) {
        g->adj[fill[g->eu[e]]++] = g->ev[e];
        g->adj[fill[g->ev[e]]++] = g->eu[e];
    }
    free(fill);
    for (int64_t v = 0; v < n; ++v)
        qsort(g->adj + g->rowptr[v], (size_t)(g->rowptr[v + 1] - g->rowptr[v]), sizeof(int32_t), cmp_i32);
    return g;
}

int64_t tgo_num_edges(const tgo_graph *g) { return g->M; }

void tgo_edges(const tgo_graph *g, int32_t *u, int32_t *v) {
    memcpy(u, g->eu, sizeof(int32_t) * (size_t)g->M);
    memcpy(v, g->ev, sizeof(int32_t) * (size_t)g->M);
}

/* ---------------------------------------------------------- layout ------- */

static int64_t binom(int64_t a, int64_t b) {
    if (b < 0 || a < b) return 0;
    int64_t r = 1;
    for (int64_t i = 1; i <= b; ++i) r = r * (a - b + i) / i;
    return r;
}

int64_t tgo_npairs(int32_t L) { return (int64_t)L * (L + 1) / 2; }

int64_t tgo_slots(int32_t L, int32_t k, int32_t orbit_level) {
    int64_t P = tgo_npairs(L);
    if (k == 3) return 2 * (int64_t)L;
    return 2 * (int64_t)L + (orbit_level ? 10 : 6) * P;
}

int64_t tgo_global_len(int32_t L, int32_t k) {
    int64_t len = binom(L + 1, 2) + 2 * binom(L + 2, 3);
    if (k == 4) len += 6 * binom(L + 3, 4);
    return len;
}

/* index of the unordered pair (a, b), a <= b, in lexicographic order */
static uint64_t choose2(uint64_t x) { return x < 2 ? 0 : x * (x - 1) / 2; }

static int64_t pair_index(int32_t L, int32_t a, int32_t b) {
    if (a > b) { int32_t t = a; a = b; b = t; }
    return (int64_t)a * L - (int64_t)a * (a - 1) / 2 + (b - a);
}

/* colex rank of a sorted multiset c[0] <= ... <= c[k-1] */
int64_t tgo_rank(const int32_t *c, int32_t k) {
    int64_t r = 0;
    for (int32_t m = 1; m <= k; ++m) r += binom(c[m - 1] + m - 1, m);
    return r;
}

static void sort_small(int32_t *c, int32_t k) {
    for (int32_t a = 1; a < k; ++a) {
        int32_t x = c[a], b = a - 1;
        while (b >= 0 && c[b] > x) { c[b + 1] = c[b]; --b; }
        c[b + 1] = x;
    }
}

/* ------------------------------------------------------ per-edge count --- */

enum { PSI_NONE = 0, PSI_L1 = 1, PSI_L2 = 2, PSI_L3 = 3 };

/*
 * Orbit-level row for edge e (layout above).  psi has n zero bytes on entry
 * and is zero again on return.
 */
static void count_edge(const tgo_graph *g, int64_t e, uint8_t *psi, uint64_t *row) {
    const int32_t L = g->L;
    const int64_t P = tgo_npairs(L);
    int32_t a = g->eu[e], b = g->ev[e];
    int64_t da = g->rowptr[a + 1] - g->rowptr[a], db = g->rowptr[b + 1] - g->rowptr[b];
    /* Thm. (3-node time complexity): enumerate Gamma_i twice with d_i <= d_j. */
    int32_t i = a, j = b;
    if (db < da) { i = b; j = a; }
    const int32_t *Gi = g->adj + g->rowptr[i];
    const int32_t *Gj = g->adj + g->rowptr[j];
    int64_t di = g->rowptr[i + 1] - g->rowptr[i], dj = g->rowptr[j + 1] - g->rowptr[j];
    const uint8_t *phi = g->type;

    uint64_t *g1 = row, *g2 = row + L;
    uint64_t *go[13];
    for (int o = 3; o <= 12; ++o) go[o] = row + 2 * L + (int64_t)(o - 3) * P;
    memset(row, 0, sizeof(uint64_t) * (size_t)(2 * L + 10 * P));

    uint64_t Tn[16] = {0}, Si[16] = {0}, Sj[16] = {0};

    /* Alg. 1: mark Gamma_i \ {j} */
    for (int64_t x = 0; x < di; ++x)
        if (Gi[x] != j) psi[Gi[x]] = PSI_L1;
    /* Alg. 1: triangles and 3-paths centred at j */
    for (int64_t x = 0; x < dj; ++x) {
        int32_t k = Gj[x];
        if (k == i) continue;
        if (psi[k] == PSI_L1) { Tn[phi[k]]++; psi[k] = PSI_L3; }
        else { Sj[phi[k]]++; psi[k] = PSI_L2; }
    }
    /* Alg. 1: 3-paths centred at i (Gamma_i minus T minus j) */
    for (int64_t x = 0; x < di; ++x) {
        int32_t k = Gi[x];
        if (k == j) continue;
        if (psi[k] == PSI_L1) Si[phi[k]]++;
    }
    for (int32_t t = 0; t < L; ++t) { g1[t] = Si[t] + Sj[t]; g2[t] = Tn[t]; }

    /* Alg. 2, S_i pass */
    for (int64_t x = 0; x < di; ++x) {
        int32_t wk = Gi[x];
        if (wk == j || psi[wk] != PSI_L1) continue;
        const int32_t *Gk = g->adj + g->rowptr[wk];
        int64_t dk = g->rowptr[wk + 1] - g->rowptr[wk];
        for (int64_t y = 0; y < dk; ++y) {
            int32_t wr = Gk[y];
            if (wr == i || wr == j) continue;
            if (psi[wr] == PSI_NONE) go[3][pair_index(L, phi[wk], phi[wr])]++;
            else if (psi[wr] == PSI_L1 && wr < wk) go[7][pair_index(L, phi[wk], phi[wr])]++;
        }
    }
    /* Alg. 2, S_j pass */
    for (int64_t x = 0; x < dj; ++x) {
        int32_t wk = Gj[x];
        if (wk == i || psi[wk] != PSI_L2) continue;
        const int32_t *Gk = g->adj + g->rowptr[wk];
        int64_t dk = g->rowptr[wk + 1] - g->rowptr[wk];
        for (int64_t y = 0; y < dk; ++y) {
            int32_t wr = Gk[y];
            if (wr == i || wr == j) continue;
            if (psi[wr] == PSI_NONE) go[3][pair_index(L, phi[wk], phi[wr])]++;
            else if (psi[wr] == PSI_L2 && wr < wk) go[7][pair_index(L, phi[wk], phi[wr])]++;
            else if (psi[wr] == PSI_L1) go[6][pair_index(L, phi[wk], phi[wr])]++;
        }
    }
    /* Alg. 3 */
    for (int64_t x = 0; x < di; ++x) {
        int32_t wk = Gi[x];
        if (wk == j || psi[wk] != PSI_L3) continue;
        const int32_t *Gk = g->adj + g->rowptr[wk];
        int64_t dk = g->rowptr[wk + 1] - g->rowptr[wk];
        for (int64_t y = 0; y < dk; ++y) {
            int32_t wr = Gk[y];
            if (psi[wr] == PSI_L3 && wr < wk) go[12][pair_index(L, phi[wk], phi[wr])]++;
            else if (psi[wr] == PSI_L1 || psi[wr] == PSI_L2) {
                if (wr == i || wr == j) continue;
                go[10][pair_index(L, phi[wk], phi[wr])]++;
            } else if (psi[wr] == PSI_NONE) {
                if (wr == i || wr == j) continue;
                go[8][pair_index(L, phi[wk], phi[wr])]++;
            }
        }
    }
    /* Closed forms for every t <= t' (Sec. "Combinatorial Relationships") */
    for (int32_t t = 0; t < L; ++t) {
        for (int32_t u = t; u < L; ++u) {
            int64_t p = pair_index(L, t, u);
            if (t == u) {
                go[4][p] = Si[t] * Sj[t] - go[6][p];
                go[5][p] = choose2(Si[t]) + choose2(Sj[t]) - go[7][p];
                go[9][p] = Tn[t] * (Si[t] + Sj[t]) - go[10][p];
                go[11][p] = choose2(Tn[t]) - go[12][p];
            } else {
                go[4][p] = Si[t] * Sj[u] + Si[u] * Sj[t] - go[6][p];
                go[5][p] = Si[t] * Si[u] + Sj[t] * Sj[u] - go[7][p];
                go[9][p] = Tn[t] * (Si[u] + Sj[u]) + Tn[u] * (Si[t] + Sj[t]) - go[10][p];
                go[11][p] = Tn[t] * Tn[u] - go[12][p];
            }
        }
    }
    /* Alg. 1: reset Psi */
    for (int64_t x = 0; x < di; ++x) psi[Gi[x]] = PSI_NONE;
    for (int64_t x = 0; x < dj; ++x) psi[Gj[x]] = PSI_NONE;
}

/* Sec. "From Typed Orbits to Graphlets": orbit row -> graphlet row */
static void orbit_to_graphlet(int32_t L, const uint64_t *orb, uint64_t *out) {
    int64_t P = tgo_npairs(L);
    const uint64_t *go[13];
    for (int o = 3; o <= 12; ++o) go[o] = orb + 2 * L + (int64_t)(o - 3) * P;
    for (int32_t t = 0; t < 2 * L; ++t) out[t] = orb[t];
    uint64_t *h[9];
    for (int q = 3; q <= 8; ++q) h[q] = out + 2 * L + (int64_t)(q - 3) * P;
    for (int64_t p = 0; p < P; ++p) {
        h[3][p] = go[3][p] + go[4][p];
        h[4][p] = go[5][p];
        h[5][p] = go[6][p];
        h[6][p] = go[7][p] + go[8][p] + go[9][p];
        h[7][p] = go[10][p] + go[11][p];
        h[8][p] = go[12][p];
    }
}

/*
 * Per-edge rows for the edges listed in `edges` (canonical edge indices), or
 * for every edge in canonical order when edges == NULL (count = M).
 * level: 0 = graphlet, 1 = orbit.  threads <= 0 uses the OpenMP default.
 */
int tgo_count_per_edge(const tgo_graph *g, int32_t k, int32_t level, const int64_t *edges,
                       int64_t count, uint64_t *rows, int32_t threads) {
    if (k != 3 && k != 4) return -1;
    const int32_t L = g->L;
    const int64_t P = tgo_npairs(L);
    const int64_t full = 2 * L + 10 * P;
    const int64_t width = tgo_slots(L, k, level);
    if (!edges) count = g->M;
    int err = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel
    {
        uint8_t *psi = (uint8_t *)calloc((size_t)(g->n > 0 ? g->n : 1), 1);
        uint64_t *orb = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)full);
        uint64_t *grl = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)full);
        if (!psi || !orb || !grl) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t q = 0; q < count; ++q) {
            if (!psi || !orb || !grl) continue;
            int64_t e = edges ? edges[q] : q;
            count_edge(g, e, psi, orb);
            const uint64_t *src = orb;
            if (!level) { orbit_to_graphlet(L, orb, grl); src = grl; }
            memcpy(rows + q * width, src, sizeof(uint64_t) * (size_t)width);
        }
        free(psi); free(orb); free(grl);
    }
    return err;
}

/*
 * Global typed graphlet counts (Eq. C = x^T e / |E(H)|).  Returns 0, or -3 if
 * a per-edge sum is not divisible by |E(H)| (which would mean a counting bug).
 */
int tgo_count_global(const tgo_graph *g, int32_t k, uint64_t *out, int32_t threads) {
    if (k != 3 && k != 4) return -1;
    const int32_t L = g->L;
    const int64_t P = tgo_npairs(L);
    const int64_t full = 2 * L + 10 * P;
    const int64_t len = tgo_global_len(L, k);
    const int64_t off1 = binom(L + 1, 2), n3 = binom(L + 2, 3), n4 = binom(L + 3, 4);
    const int64_t off2 = off1 + n3, off4 = off1 + 2 * n3;
    memset(out, 0, sizeof(uint64_t) * (size_t)len);
    int err = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel
    {
        uint8_t *psi = (uint8_t *)calloc((size_t)(g->n > 0 ? g->n : 1), 1);
        uint64_t *orb = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)full);
        uint64_t *grl = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)full);
        uint64_t *acc = (uint64_t *)calloc((size_t)len, sizeof(uint64_t));
        if (!psi || !orb || !grl || !acc) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t e = 0; e < g->M; ++e) {
            if (!psi || !orb || !grl || !acc) continue;
            count_edge(g, e, psi, orb);
            orbit_to_graphlet(L, orb, grl);
            int32_t ti = g->type[g->eu[e]], tj = g->type[g->ev[e]];
            int32_t c[4];
            c[0] = ti; c[1] = tj; sort_small(c, 2);
            acc[tgo_rank(c, 2)] += 1;
            for (int32_t t = 0; t < L; ++t) {
                c[0] = ti; c[1] = tj; c[2] = t; sort_small(c, 3);
                int64_t r = tgo_rank(c, 3);
                acc[off1 + r] += grl[t];
                acc[off2 + r] += grl[L + t];
            }
            if (k == 4) {
                for (int32_t t = 0; t < L; ++t)
                    for (int32_t u = t; u < L; ++u) {
                        c[0] = ti; c[1] = tj; c[2] = t; c[3] = u; sort_small(c, 4);
                        int64_t r = tgo_rank(c, 4), p = pair_index(L, t, u);
                        for (int q = 0; q < 6; ++q)
                            acc[off4 + q * n4 + r] += grl[2 * L + q * P + p];
                    }
            }
        }
#pragma omp critical
        {
            if (acc)
                for (int64_t x = 0; x < len; ++x) out[x] += acc[x];
        }
        free(psi); free(orb); free(grl); free(acc);
    }
    if (err) return err;
    /* |E(H)|: h1 = 2, h2 = 3, h3..h8 = 3,3,4,4,5,6 (Table 2) */
    static const uint64_t eh4[6] = {3, 3, 4, 4, 5, 6};
    for (int64_t r = 0; r < n3; ++r) {
        if (out[off1 + r] % 2 || out[off2 + r] % 3) return -3;
        out[off1 + r] /= 2;
        out[off2 + r] /= 3;
    }
    if (k == 4)
        for (int q = 0; q < 6; ++q)
            for (int64_t r = 0; r < n4; ++r) {
                uint64_t *x = &out[off4 + q * n4 + r];
                if (*x % eh4[q]) return -3;
                *x /= eh4[q];
            }
    return 0;
}

/* Unordered pair index (exported so tests can decode rows independently). */
int64_t tgo_pair_index(int32_t L, int32_t a, int32_t b) { return pair_index(L, a, b); }

int32_t tgo_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
