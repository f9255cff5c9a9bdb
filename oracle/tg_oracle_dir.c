/*
 * Directed typed 3-node graphlet oracle (test infrastructure only; loaded by
 * tests/, never by the library).
 *
 * Follows Sec. "Directed Typed Graphlets": every typed neighbourhood Gamma_i^t
 * is split into out-neighbours Gamma_i^{t,+} and in-neighbours
 * Gamma_i^{t,-}, and Alg. 1 runs per edge (i, j) of the underlying undirected
 * graph over the split sets: the neighbours of i are marked with the
 * direction of their pair with i (mark array Psi, as Alg. 1); a neighbour w of
 * j that carries a mark is a triangle node (T_ij^{t,+/-}), the others are
 * 3-star nodes S_j^{t,+/-}, and the marked nodes never met from j are
 * S_i^{t,+/-}.  Each combination of directions gives one directed motif; its
 * class is found by trying the six relabellings of the three nodes against
 * the class representatives (the 13 connected triads, in the order and with
 * the representatives the library's header defines).
 *
 * Output layouts: per-edge rows of 13 L counts (class c, type of the third
 * node t at c L + t), edges in canonical order (u < v, original ids,
 * ascending); global counts of 13 C(L+2, 3) entries (class c's block at
 * c C(L+2, 3), inside it the colex rank of the sorted type multiset), each the
 * per-edge sum divided by the class's number of underlying edges (2 for the
 * path classes 0-4 and 7, 3 for the others).
 *
 * Parity status: pinned by brute force over all node triples of tiny
 * digraphs, by closed forms (tournaments, bidirected cliques, directed cycles
 * and stars) and by the sum over classes equalling the undirected 3-node
 * counts (tests/test_oracle_directed.py).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NCLS 13

/* representatives on nodes 0, 1, 2: arcs (from, to), -1 terminated */
static const int REP[NCLS][7][2] = {
    {{1, 0}, {1, 2}, {-1, 0}},                                  /* 021D */
    {{0, 1}, {2, 1}, {-1, 0}},                                  /* 021U */
    {{0, 1}, {1, 2}, {-1, 0}},                                  /* 021C */
    {{0, 1}, {1, 0}, {2, 1}, {-1, 0}},                          /* 111D */
    {{0, 1}, {1, 0}, {1, 2}, {-1, 0}},                          /* 111U */
    {{0, 1}, {2, 1}, {0, 2}, {-1, 0}},                          /* 030T */
    {{0, 1}, {1, 2}, {2, 0}, {-1, 0}},                          /* 030C */
    {{0, 1}, {1, 0}, {1, 2}, {2, 1}, {-1, 0}},                  /* 201  */
    {{1, 0}, {1, 2}, {0, 2}, {2, 0}, {-1, 0}},                  /* 120D */
    {{0, 1}, {2, 1}, {0, 2}, {2, 0}, {-1, 0}},                  /* 120U */
    {{0, 1}, {1, 2}, {0, 2}, {2, 0}, {-1, 0}},                  /* 120C */
    {{0, 1}, {1, 2}, {2, 1}, {0, 2}, {2, 0}, {-1, 0}},          /* 210  */
    {{0, 1}, {1, 0}, {1, 2}, {2, 1}, {0, 2}, {2, 0}, {-1, 0}},  /* 300  */
};

/* adjacency matrix of 3 nodes as 9 bits, bit 3 a + b for the arc a -> b */
static int code_of(const int adj[3][3]) {
    int c = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (adj[a][b]) c |= 1 << (3 * a + b);
    return c;
}

/* smallest code over the six relabellings */
static int canon(const int adj[3][3]) {
    static const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    int best = 1 << 30;
    for (int q = 0; q < 6; ++q) {
        int m[3][3] = {{0}};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (adj[a][b]) m[P[q][a]][P[q][b]] = 1;
        const int c = code_of(m);
        if (c < best) best = c;
    }
    return best;
}

static int rep_canon[NCLS];
static int class_tab[4][4][4];
static int classify_slow(int s01, int s02, int s12);

static void init_classes(void) {
    for (int c = 0; c < NCLS; ++c) {
        int adj[3][3] = {{0}};
        for (int r = 0; REP[c][r][0] >= 0; ++r) adj[REP[c][r][0]][REP[c][r][1]] = 1;
        rep_canon[c] = canon(adj);
    }
    for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y)
            for (int z = 0; z < 4; ++z) class_tab[x][y][z] = classify_slow(x, y, z);
}

/* class of the digraph on (0, 1, 2) given the direction bits of its three
 * pairs (bit 1: lower -> higher, bit 2: higher -> lower), -1 if disconnected */
static int classify_slow(int s01, int s02, int s12) {
    int adj[3][3] = {{0}};
    adj[0][1] = s01 & 1; adj[1][0] = (s01 >> 1) & 1;
    adj[0][2] = s02 & 1; adj[2][0] = (s02 >> 1) & 1;
    adj[1][2] = s12 & 1; adj[2][1] = (s12 >> 1) & 1;
    const int c = canon(adj);
    for (int k = 0; k < NCLS; ++k)
        if (rep_canon[k] == c) return k;
    return -1;
}

static int classify(int s01, int s02, int s12) { return class_tab[s01][s02][s12]; }

static int64_t binom3(int64_t a) { return a < 3 ? 0 : a * (a - 1) * (a - 2) / 6; }
static int64_t colex3(int a, int b, int c) {
    /* a <= b <= c */
    return (int64_t)a + (int64_t)(b + 1) * b / 2 + (int64_t)(c + 2) * (c + 1) * c / 6;
}

typedef struct {
    int64_t u, v;
    int bits;
} arc_t;

static int cmp_arc(const void *x, const void *y) {
    const arc_t *a = (const arc_t *)x, *b = (const arc_t *)y;
    if (a->u != b->u) return a->u < b->u ? -1 : 1;
    if (a->v != b->v) return a->v < b->v ? -1 : 1;
    return 0;
}

int tgod_slots(int L) { return NCLS * L; }
int64_t tgod_global_len(int L) { return (int64_t)NCLS * binom3(L + 2); }

/* Number of canonical edges of the underlying simple graph. */
int64_t tgod_edges(int64_t n, int64_t m, const int32_t *src, const int32_t *dst);

/*
 * rows: M x 13 L (may be NULL); global: 13 C(L+2,3) (may be NULL).
 * Returns 0, or -1 on bad input, -2 on a sum not divisible.
 */
int tgod_count(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint8_t *type,
               int L, uint64_t *rows, uint64_t *global) {
    if (n < 1 || m < 0 || L < 1 || L > 16) return -1;
    init_classes();
    /* both directions of every arc, merged per ordered pair */
    arc_t *a = (arc_t *)malloc(sizeof(arc_t) * (size_t)(2 * m + 1));
    int64_t na = 0;
    for (int64_t e = 0; e < m; ++e) {
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) {
            free(a);
            return -1;
        }
        if (src[e] == dst[e]) continue;
        a[na].u = src[e]; a[na].v = dst[e]; a[na].bits = 1; ++na;  /* u -> v: out of u */
        a[na].u = dst[e]; a[na].v = src[e]; a[na].bits = 2; ++na;  /* into v's list as in */
    }
    qsort(a, (size_t)na, sizeof(arc_t), cmp_arc);
    int64_t k = 0;
    for (int64_t x = 0; x < na; ++x) {
        if (k > 0 && a[k - 1].u == a[x].u && a[k - 1].v == a[x].v) a[k - 1].bits |= a[x].bits;
        else a[k++] = a[x];
    }
    /* CSR of the split neighbourhoods: neighbour and direction bits */
    int64_t *rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t x = 0; x < k; ++x) rp[a[x].u + 1]++;
    for (int64_t v = 0; v < n; ++v) rp[v + 1] += rp[v];
    int64_t *nb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k + 1));
    int *st = (int *)malloc(sizeof(int) * (size_t)(k + 1));
    for (int64_t x = 0; x < k; ++x) {
        nb[x] = a[x].v;
        st[x] = a[x].bits;
    }
    free(a);
    const int64_t n3 = binom3(L + 2);
    const int S = NCLS * L;
    uint64_t *sums = (uint64_t *)calloc((size_t)(NCLS * n3), sizeof(uint64_t));
    int *psi = (int *)calloc((size_t)n, sizeof(int));   /* direction of (i, w) seen from i, 0 unmarked */
    char *met = (char *)calloc((size_t)n, 1);
    uint64_t *row = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)S);
    int64_t e = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t x = rp[i]; x < rp[i + 1]; ++x) {
            const int64_t j = nb[x];
            if (j <= i) continue;
            /* edge (i, j), i < j: canonical order */
            const int sij = st[x];
            memset(row, 0, sizeof(uint64_t) * (size_t)S);
            for (int64_t y = rp[i]; y < rp[i + 1]; ++y) psi[nb[y]] = st[y];
            for (int64_t y = rp[j]; y < rp[j + 1]; ++y) {
                const int64_t w = nb[y];
                if (w == i) continue;
                const int sjw = st[y];
                int c;
                if (psi[w]) {
                    /* w in T_ij: pairs (i, j), (i, w), (j, w) */
                    c = classify(sij, psi[w], sjw);
                    met[w] = 1;
                } else {
                    /* w in S_j: pairs (i, j) and (j, w); node 0 = i, 1 = j, 2 = w */
                    c = classify(sij, 0, sjw);
                }
                row[c * L + type[w]]++;
            }
            for (int64_t y = rp[i]; y < rp[i + 1]; ++y) {
                const int64_t w = nb[y];
                if (w == j || met[w]) continue;
                /* w in S_i: pairs (i, j) and (i, w) */
                const int c = classify(sij, st[y], 0);
                row[c * L + type[w]]++;
            }
            for (int64_t y = rp[i]; y < rp[i + 1]; ++y) {
                psi[nb[y]] = 0;
                met[nb[y]] = 0;
            }
            if (rows) memcpy(rows + e * S, row, sizeof(uint64_t) * (size_t)S);
            for (int c = 0; c < NCLS; ++c)
                for (int t = 0; t < L; ++t) {
                    if (!row[c * L + t]) continue;
                    int p = type[i], q = type[j], r = t, z;
                    if (p > q) { z = p; p = q; q = z; }
                    if (q > r) { z = q; q = r; r = z; }
                    if (p > q) { z = p; p = q; q = z; }
                    sums[c * n3 + colex3(p, q, r)] += row[c * L + t];
                }
            ++e;
        }
    }
    int rc = 0;
    if (global)
        for (int c = 0; c < NCLS; ++c) {
            const uint64_t div = (c <= 4 || c == 7) ? 2 : 3;
            for (int64_t q = 0; q < n3; ++q) {
                if (sums[c * n3 + q] % div) rc = -2;
                global[c * n3 + q] = sums[c * n3 + q] / div;
            }
        }
    free(sums);
    free(psi);
    free(met);
    free(row);
    free(rp);
    free(nb);
    free(st);
    return rc;
}

int64_t tgod_edges(int64_t n, int64_t m, const int32_t *src, const int32_t *dst) {
    arc_t *a = (arc_t *)malloc(sizeof(arc_t) * (size_t)(m + 1));
    int64_t na = 0;
    for (int64_t e = 0; e < m; ++e) {
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n || src[e] == dst[e]) continue;
        a[na].u = src[e] < dst[e] ? src[e] : dst[e];
        a[na].v = src[e] < dst[e] ? dst[e] : src[e];
        a[na].bits = 0;
        ++na;
    }
    qsort(a, (size_t)na, sizeof(arc_t), cmp_arc);
    int64_t k = 0;
    for (int64_t x = 0; x < na; ++x)
        if (x == 0 || a[x].u != a[x - 1].u || a[x].v != a[x - 1].v) ++k;
    free(a);
    return k;
}
