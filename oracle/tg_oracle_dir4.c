/*
 * Directed typed 4-node graphlet oracle (test infrastructure only; loaded by
 * tests/, never by the library).
 *
 * Sec. "Directed Typed Graphlets" extends the typed counts to digraphs by
 * splitting every typed neighbourhood into out- and in-neighbours; the paper
 * gives no list of the directed 4-node motifs.  Reading taken here: a
 * directed 4-node graphlet is a connected induced subgraph on four nodes
 * with its arcs (a pair may carry both arcs), keyed by its isomorphism class
 * and the sorted multiset of its node types (as Def. "Typed Graphlet
 * Instance").  There are 199 classes.  Class numbering: the code of a
 * digraph on nodes 0..3 is the sum of 2^(4a + b) over its arcs a -> b; its
 * canonical code is the smallest code over the 24 relabellings; class c is
 * the c-th smallest canonical code among the connected ones.
 *
 * Per edge (i, j) of the underlying graph, the connected 4-node sets that
 * contain it are {i, j, w, r} with w in Gamma_i u Gamma_j (the 3-node
 * extension of Alg. 1) and r either another node of Gamma_i u Gamma_j or a
 * neighbour of w outside it; each set is met once.  Its class comes from the
 * six pair states, its key from the types of w and r.
 *
 * Output layouts: per-edge rows of 199 P counts (P = L(L+1)/2; class c, type
 * pair {t, u} of the two other nodes at c P + pair(t, u) with pair(a, b) =
 * a L - a(a-1)/2 + (b - a) for a <= b), edges in canonical order (u < v,
 * original ids, ascending); global counts of 199 C(L+3, 4) entries (class c's
 * block at c C(L+3, 4), inside it the colex rank of the sorted type
 * multiset), each the per-edge sum divided by the class's number of
 * underlying edges.
 *
 * Parity status: pinned by brute force over all node quadruples of tiny
 * digraphs, by closed forms (transitive tournaments, bidirected cliques,
 * directed cycles, out- and in-stars) and by the sums over classes of each
 * undirected shape against the undirected 4-node counts
 * (tests/test_oracle_directed4.py).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NCLS4 199

static int ncls = 0;
static int canon_codes[NCLS4];
static int cls_edges[NCLS4];      /* underlying edges of each class */
static int16_t *code2cls = 0;     /* 65536 entries: class of a canonical code, or -1 */

static const int PERM[24][4] = {
    {0, 1, 2, 3}, {0, 1, 3, 2}, {0, 2, 1, 3}, {0, 2, 3, 1}, {0, 3, 1, 2}, {0, 3, 2, 1},
    {1, 0, 2, 3}, {1, 0, 3, 2}, {1, 2, 0, 3}, {1, 2, 3, 0}, {1, 3, 0, 2}, {1, 3, 2, 0},
    {2, 0, 1, 3}, {2, 0, 3, 1}, {2, 1, 0, 3}, {2, 1, 3, 0}, {2, 3, 0, 1}, {2, 3, 1, 0},
    {3, 0, 1, 2}, {3, 0, 2, 1}, {3, 1, 0, 2}, {3, 1, 2, 0}, {3, 2, 0, 1}, {3, 2, 1, 0}};

static int canon(int code) {
    int best = 1 << 30;
    for (int q = 0; q < 24; ++q) {
        int c = 0;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                if (a != b && ((code >> (4 * a + b)) & 1)) c |= 1 << (4 * PERM[q][a] + PERM[q][b]);
        if (c < best) best = c;
    }
    return best;
}

static int connected(int code) {
    int adj[4] = {0, 0, 0, 0};
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            if (a != b && ((code >> (4 * a + b)) & 1)) {
                adj[a] |= 1 << b;
                adj[b] |= 1 << a;
            }
    int seen = 1, grow = 1;
    while (grow) {
        grow = 0;
        for (int v = 0; v < 4; ++v)
            if ((seen >> v) & 1 && (adj[v] | seen) != seen) {
                seen |= adj[v];
                grow = 1;
            }
    }
    return seen == 15;
}

static int cmp_int(const void *x, const void *y) {
    const int a = *(const int *)x, b = *(const int *)y;
    return (a > b) - (a < b);
}

static void init_classes4(void) {
    if (code2cls) return;
    code2cls = (int16_t *)malloc(sizeof(int16_t) * 65536);
    for (int c = 0; c < 65536; ++c) code2cls[c] = -1;
    /* codes with no self-arc bits only */
    int found[NCLS4 + 1];
    int k = 0;
    char *mark = (char *)calloc(65536, 1);
    for (int code = 0; code < 65536; ++code) {
        if (code & 0x8421) continue; /* bits 4a + a */
        if (!connected(code)) continue;
        const int c = canon(code);
        if (!mark[c]) {
            mark[c] = 1;
            if (k < NCLS4 + 1) found[k] = c;
            ++k;
        }
    }
    free(mark);
    ncls = k;
    if (k != NCLS4) return;
    qsort(found, NCLS4, sizeof(int), cmp_int);
    for (int c = 0; c < NCLS4; ++c) {
        canon_codes[c] = found[c];
        code2cls[found[c]] = (int16_t)c;
        int und = 0;
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (((found[c] >> (4 * a + b)) & 1) || ((found[c] >> (4 * b + a)) & 1)) ++und;
        cls_edges[c] = und;
    }
}

int tgod4_classes(int32_t *codes, int32_t *edges) {
    init_classes4();
    if (ncls != NCLS4) return -1;
    for (int c = 0; c < NCLS4; ++c) {
        if (codes) codes[c] = canon_codes[c];
        if (edges) edges[c] = cls_edges[c];
    }
    return NCLS4;
}

static int64_t binom4(int64_t a) { return a < 4 ? 0 : a * (a - 1) * (a - 2) * (a - 3) / 24; }

static int64_t colex4(int a, int b, int c, int d) {
    /* a <= b <= c <= d */
    return (int64_t)a + (int64_t)(b + 1) * b / 2 + (int64_t)(c + 2) * (c + 1) * c / 6 +
           (int64_t)(d + 3) * (d + 2) * (d + 1) * d / 24;
}

typedef struct {
    int64_t u, v;
    int bits;
} arc4_t;

static int cmp_arc4(const void *x, const void *y) {
    const arc4_t *a = (const arc4_t *)x, *b = (const arc4_t *)y;
    if (a->u != b->u) return a->u < b->u ? -1 : 1;
    if (a->v != b->v) return a->v < b->v ? -1 : 1;
    return 0;
}

/* direction bits of the pair (x, y) seen from x (1: x -> y, 2: y -> x), 0 if none */
static int state(const int64_t *rp, const int64_t *nb, const int *st, int64_t x, int64_t y) {
    int64_t lo = rp[x], hi = rp[x + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (nb[mid] < y) lo = mid + 1;
        else hi = mid;
    }
    return (lo < rp[x + 1] && nb[lo] == y) ? st[lo] : 0;
}

int tgod4_slots(int L) { return NCLS4 * L * (L + 1) / 2; }
int64_t tgod4_global_len(int L) { return (int64_t)NCLS4 * binom4(L + 3); }

/*
 * rows: M x 199 P (may be NULL); global: 199 C(L+3, 4) (may be NULL).
 * Returns 0, -1 on bad input or a class table that is not 199 long, -2 on a
 * sum not divisible.
 */
int tgod4_count(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint8_t *type,
                int L, uint64_t *rows, uint64_t *global) {
    if (n < 1 || m < 0 || L < 1 || L > 16) return -1;
    init_classes4();
    if (ncls != NCLS4) return -1;
    arc4_t *a = (arc4_t *)malloc(sizeof(arc4_t) * (size_t)(2 * m + 1));
    int64_t na = 0;
    for (int64_t e = 0; e < m; ++e) {
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) {
            free(a);
            return -1;
        }
        if (src[e] == dst[e]) continue;
        a[na].u = src[e]; a[na].v = dst[e]; a[na].bits = 1; ++na;
        a[na].u = dst[e]; a[na].v = src[e]; a[na].bits = 2; ++na;
    }
    qsort(a, (size_t)na, sizeof(arc4_t), cmp_arc4);
    int64_t k = 0;
    for (int64_t x = 0; x < na; ++x) {
        if (k > 0 && a[k - 1].u == a[x].u && a[k - 1].v == a[x].v) a[k - 1].bits |= a[x].bits;
        else a[k++] = a[x];
    }
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
    const int P = L * (L + 1) / 2;
    const int S = NCLS4 * P;
    const int64_t n4 = binom4(L + 3);
    uint64_t *sums = (uint64_t *)calloc((size_t)(NCLS4 * n4), sizeof(uint64_t));
    uint64_t *row = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)S);
    char *inC = (char *)calloc((size_t)n, 1);
    int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k + 2));
    int64_t e = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t x = rp[i]; x < rp[i + 1]; ++x) {
            const int64_t j = nb[x];
            if (j <= i) continue;
            memset(row, 0, sizeof(uint64_t) * (size_t)S);
            /* C = (Gamma_i u Gamma_j) \ {i, j} */
            int64_t nc = 0;
            for (int64_t y = rp[i]; y < rp[i + 1]; ++y)
                if (nb[y] != j && !inC[nb[y]]) { inC[nb[y]] = 1; cand[nc++] = nb[y]; }
            for (int64_t y = rp[j]; y < rp[j + 1]; ++y)
                if (nb[y] != i && !inC[nb[y]]) { inC[nb[y]] = 1; cand[nc++] = nb[y]; }
            const int64_t v4[4] = {i, j, 0, 0};
            for (int64_t p = 0; p < nc; ++p) {
                const int64_t w = cand[p];
                /* r in C after w, and r a neighbour of w outside C u {i, j} */
                for (int pass = 0; pass < 2; ++pass) {
                    const int64_t lo = pass == 0 ? p + 1 : rp[w];
                    const int64_t hi = pass == 0 ? nc : rp[w + 1];
                    for (int64_t q = lo; q < hi; ++q) {
                        const int64_t r = pass == 0 ? cand[q] : nb[q];
                        if (pass == 1 && (r == i || r == j || inC[r])) continue;
                        int64_t v[4] = {v4[0], v4[1], w, r};
                        int code = 0;
                        for (int s = 0; s < 4; ++s)
                            for (int t = s + 1; t < 4; ++t) {
                                const int bits = state(rp, nb, st, v[s], v[t]);
                                if (bits & 1) code |= 1 << (4 * s + t);
                                if (bits & 2) code |= 1 << (4 * t + s);
                            }
                        const int c = code2cls[canon(code)];
                        if (c < 0) continue; /* not connected: cannot happen */
                        int tw = type[w], tr = type[r];
                        if (tw > tr) { const int z = tw; tw = tr; tr = z; }
                        row[c * P + tw * L - tw * (tw - 1) / 2 + (tr - tw)]++;
                    }
                }
            }
            for (int64_t p = 0; p < nc; ++p) inC[cand[p]] = 0;
            if (rows) memcpy(rows + e * S, row, sizeof(uint64_t) * (size_t)S);
            for (int c = 0; c < NCLS4; ++c)
                for (int t = 0; t < L; ++t)
                    for (int u = t; u < L; ++u) {
                        const uint64_t val = row[c * P + t * L - t * (t - 1) / 2 + (u - t)];
                        if (!val) continue;
                        int q[4] = {type[i], type[j], t, u}, z;
                        for (int s = 0; s < 4; ++s)
                            for (int s2 = s + 1; s2 < 4; ++s2)
                                if (q[s2] < q[s]) { z = q[s]; q[s] = q[s2]; q[s2] = z; }
                        sums[c * n4 + colex4(q[0], q[1], q[2], q[3])] += val;
                    }
            ++e;
        }
    }
    int rc = 0;
    if (global)
        for (int c = 0; c < NCLS4; ++c)
            for (int64_t q = 0; q < n4; ++q) {
                if (sums[c * n4 + q] % (uint64_t)cls_edges[c]) rc = -2;
                global[c * n4 + q] = sums[c * n4 + q] / (uint64_t)cls_edges[c];
            }
    free(sums);
    free(row);
    free(inC);
    free(cand);
    free(rp);
    free(nb);
    free(st);
    return rc;
}
