// Directed typed 3-node graphlets (Sec. "Directed Typed Graphlets").
//
// The paper splits every typed neighbourhood into out- and in-neighbours
// (Gamma_i^{t,+}, Gamma_i^{t,-}) and runs Alg. 1 over the combinations of the
// split sets.  Here the split is two bits per adjacency entry of the
// undirected typed CSR (bit 0: owner -> neighbour, bit 1: neighbour ->
// owner; both for a pair with arcs both ways), set once when the graph is
// built with TG_DIRECTED.  Per edge (i, j) one warp runs Alg. 1 on the
// shorter list: each triangle node w of T_ij comes with the state of (i, w)
// and of (j, w), counted per (state pair, type of w); the 3-star nodes S_i,
// S_j are not enumerated: their counts per (state, type) are the node's
// split typed degrees less j (or i) and less the triangle nodes of that
// state.  The triad class of {i, j, w} follows from the three pair states by
// a table built on the host from the class representatives of the header.
#include <algorithm>
#include <mutex>
#include <vector>

#include "tg_device.cuh"

using namespace tgd;

namespace {

constexpr int kDirThreads = 256;
constexpr int kDirWarps = kDirThreads / 32;

// Arc bits of the pairs of three labelled nodes 0, 1, 2: bit 2 p for the arc
// from the lower to the higher node of pair p, bit 2 p + 1 for the reverse;
// pairs (0, 1), (0, 2), (1, 2).
int arc_bit(int a, int b) {
    const int p = (a + b == 1) ? 0 : (a + b == 2) ? 1 : 2;
    return 2 * p + (a < b ? 0 : 1);
}

// Class of every connected 3-node digraph, by arc mask; -1 for the others.
struct TriadTable {
    int8_t cls[64];
    bool ok = false;
};

TriadTable build_triads() {
    // representatives of the header on A = 0, B = 1, C = 2 (arcs from -> to)
    static const int reps[TG_TRIAD_CLASSES][6][2] = {
        {{1, 0}, {1, 2}, {-1, -1}},                                   // 021D
        {{0, 1}, {2, 1}, {-1, -1}},                                   // 021U
        {{0, 1}, {1, 2}, {-1, -1}},                                   // 021C
        {{0, 1}, {1, 0}, {2, 1}, {-1, -1}},                           // 111D
        {{0, 1}, {1, 0}, {1, 2}, {-1, -1}},                           // 111U
        {{0, 1}, {2, 1}, {0, 2}, {-1, -1}},                           // 030T
        {{0, 1}, {1, 2}, {2, 0}, {-1, -1}},                           // 030C
        {{0, 1}, {1, 0}, {1, 2}, {2, 1}, {-1, -1}},                   // 201
        {{1, 0}, {1, 2}, {0, 2}, {2, 0}, {-1, -1}},                   // 120D
        {{0, 1}, {2, 1}, {0, 2}, {2, 0}, {-1, -1}},                   // 120U
        {{0, 1}, {1, 2}, {0, 2}, {2, 0}, {-1, -1}},                   // 120C
        {{0, 1}, {1, 2}, {2, 1}, {0, 2}, {2, 0}, {-1, -1}},           // 210
        {{0, 1}, {1, 0}, {1, 2}, {2, 1}, {0, 2}, {2, 0}},             // 300
    };
    static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                   {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    TriadTable t;
    std::fill(t.cls, t.cls + 64, (int8_t)-1);
    bool ok = true;
    for (int c = 0; c < TG_TRIAD_CLASSES; ++c)
        for (int q = 0; q < 6; ++q) {
            int mask = 0;
            for (int r = 0; r < 6 && reps[c][r][0] >= 0; ++r)
                mask |= 1 << arc_bit(perm[q][reps[c][r][0]], perm[q][reps[c][r][1]]);
            if (t.cls[mask] >= 0 && t.cls[mask] != c) ok = false;
            t.cls[mask] = (int8_t)c;
        }
    // every mask whose pairs connect the three nodes must have a class
    for (int mask = 0; mask < 64; ++mask) {
        const int pairs = ((mask & 3) != 0) + ((mask & 12) != 0) + ((mask & 48) != 0);
        if ((pairs >= 2) != (t.cls[mask] >= 0)) ok = false;
    }
    t.ok = ok;
    return t;
}

const TriadTable &triads() {
    static std::once_flag once;
    static TriadTable t;
    std::call_once(once, [] { t = build_triads(); });
    return t;
}

// arc mask of a pair state (bit 0: lower-labelled -> higher, bit 1: back)
inline int pair_mask(int state, int a, int b) {
    int m = 0;
    if (state & 1) m |= 1 << arc_bit(a, b);
    if (state & 2) m |= 1 << arc_bit(b, a);
    return m;
}

struct DirParams {
    const int64_t *rowptr;
    const uint32_t *adj;
    const uint8_t *adir;
    const int32_t *toff;
    const uint8_t *ntype;
    const int2 *edges;
    const uint32_t *nd;  // n x 3 L split typed degrees (state 1..3, type)
    int64_t M;
    int32_t L;
    int64_t n3;           // C(L+2, 3)
    uint64_t *rows;       // per-edge mode
    unsigned long long *sums;  // global mode: 13 n3 undivided sums
    unsigned long long *queue;
    unsigned *err;
    int8_t tri[27];  // class of (s_ij, s_iw, s_jw), states 1..3 each
    int8_t path[9];  // class of a 3-path by the states of its ends seen from its centre
};

__global__ void k_arc_bits(const int32_t *src, const int32_t *dst, int64_t m,
                           const int32_t *old2new, const int64_t *rowptr, const uint32_t *adj,
                           const int32_t *toff, const uint8_t *ntype, int L, uint32_t *adir32,
                           unsigned *err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a0 = src[e], b0 = dst[e];
        if (a0 == b0) continue;
        const uint32_t a = (uint32_t)old2new[a0], b = (uint32_t)old2new[b0];
        const int64_t ba = rowptr[a], bb = rowptr[b];
        const int pa = find_pos(adj, ba, toff + (int64_t)a * (L + 1),
                                ((uint32_t)ntype[b] << TG_TSHIFT) | b);
        const int pb = find_pos(adj, bb, toff + (int64_t)b * (L + 1),
                                ((uint32_t)ntype[a] << TG_TSHIFT) | a);
        if (pa < 0 || pb < 0) {
            atomicOr(err, TG_DERR_BOUNDS);
            continue;
        }
        const int64_t qa = ba + pa, qb = bb + pb;
        atomicOr(adir32 + (qa >> 2), 1u << (8 * (int)(qa & 3)));  // a -> b: out of a
        atomicOr(adir32 + (qb >> 2), 2u << (8 * (int)(qb & 3)));  // a -> b: into b
    }
}

// Split typed degrees: nd[v][(s - 1) L + t] = neighbours of v of type t whose
// pair with v has state s.  One warp per node, counters in shared memory.
__global__ void __launch_bounds__(kDirThreads) k_dir_degrees(const int64_t *rowptr,
                                                             const uint32_t *adj,
                                                             const uint8_t *adir, int64_t n,
                                                             int L, uint32_t *nd) {
    __shared__ uint32_t cnt[kDirWarps][3 * TG_MAX_TYPES];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * kDirWarps;
    for (int64_t v = blockIdx.x * (int64_t)kDirWarps + warp; v < n; v += nw) {
        for (int k = lane; k < 3 * L; k += 32) cnt[warp][k] = 0u;
        __syncwarp();
        const int64_t b = rowptr[v], d = rowptr[v + 1] - b;
        for (int64_t x = lane; x < d; x += 32) {
            const int st = adir[b + x];
            const int t = (int)(__ldg(adj + b + x) >> TG_TSHIFT);
            if (st) atomicAdd(&cnt[warp][(st - 1) * L + t], 1u);
        }
        __syncwarp();
        for (int k = lane; k < 3 * L; k += 32) nd[v * 3 * L + k] = cnt[warp][k];
        __syncwarp();
    }
}

__device__ __forceinline__ int swap_state(int s) { return ((s & 1) << 1) | ((s >> 1) & 1); }

// One warp per edge (dynamic queue).  kRows: per-edge rows, else the
// undivided sums of the global count (per-CTA shared histogram).
template <bool kRows>
__global__ void __launch_bounds__(kDirThreads) k_dir3(DirParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = p.L, S = TG_TRIAD_CLASSES * L;
    unsigned long long *h = reinterpret_cast<unsigned long long *>(smem);
    const size_t hb = kRows ? 0 : (((size_t)TG_TRIAD_CLASSES * p.n3 * 8 + 15) & ~(size_t)15);
    uint32_t *tri = reinterpret_cast<uint32_t *>(smem + hb) + (size_t)warp * 9 * L;
    if (!kRows) {
        for (int64_t q = threadIdx.x; q < TG_TRIAD_CLASSES * p.n3; q += blockDim.x) h[q] = 0ull;
        __syncthreads();
    }
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(p.queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= (unsigned long long)p.M) break;
        const int64_t e = (int64_t)item;
        const int2 ab = p.edges[e];
        const uint32_t i = (uint32_t)ab.x, j = (uint32_t)ab.y;
        const int ti = p.ntype[i], tj = p.ntype[j];
        const int64_t bi = p.rowptr[i], bj = p.rowptr[j];
        const int di = (int)(p.rowptr[i + 1] - bi), dj = (int)(p.rowptr[j + 1] - bj);
        const int32_t *toi = p.toff + (int64_t)i * (L + 1);
        const int32_t *toj = p.toff + (int64_t)j * (L + 1);
        int sij = 0;
        if (lane == 0) {
            const int q = find_pos(p.adj, bi, toi, ((uint32_t)tj << TG_TSHIFT) | j);
            sij = q >= 0 ? p.adir[bi + q] : 0;
            if (sij == 0) atomicOr(p.err, TG_DERR_BOUNDS);
        }
        sij = __shfl_sync(kFull, sij, 0);
        for (int k = lane; k < 9 * L; k += 32) tri[k] = 0u;
        __syncwarp();
        if (sij != 0) {
            // Alg. 1 on the shorter list: x scanned, y searched
            const bool xi = di <= dj;
            const int64_t bx = xi ? bi : bj, by = xi ? bj : bi;
            const int dx = xi ? di : dj;
            const uint32_t yid = xi ? j : i;
            const int32_t *toy = xi ? toj : toi;
            for (int x = lane; x < dx; x += 32) {
                const uint32_t w = __ldg(p.adj + bx + x);
                if ((w & TG_IDMASK) == yid) continue;
                const int q = find_pos(p.adj, by, toy, w);
                if (q < 0) continue;
                const int sx = p.adir[bx + x], sy = p.adir[by + q];
                if (sx == 0 || sy == 0) {  // every entry carries an arc; never taken
                    atomicOr(p.err, TG_DERR_BOUNDS);
                    continue;
                }
                const int siw = xi ? sx : sy, sjw = xi ? sy : sx;
                atomicAdd(&tri[((siw - 1) * 3 + (sjw - 1)) * L + (int)(w >> TG_TSHIFT)], 1u);
            }
        }
        __syncwarp();
        if (sij != 0) {
            const int sji = swap_state(sij);
            const uint32_t *ndi = p.nd + (int64_t)i * 3 * L, *ndj = p.nd + (int64_t)j * 3 * L;
            for (int k = lane; k < S; k += 32) {
                const int c = k / L, t = k - c * L;
                unsigned long long v = 0;
                for (int s1 = 0; s1 < 3; ++s1)
                    for (int s2 = 0; s2 < 3; ++s2)
                        if (p.tri[(sij - 1) * 9 + s1 * 3 + s2] == c) v += tri[(s1 * 3 + s2) * L + t];
                for (int s = 0; s < 3; ++s) {
                    if (p.path[(sij - 1) * 3 + s] == c) {
                        // S_i members of state s + 1 and type t
                        long long m = (long long)ndi[s * L + t] - ((s + 1 == sij && t == tj) ? 1 : 0);
                        for (int s2 = 0; s2 < 3; ++s2) m -= tri[(s * 3 + s2) * L + t];
                        v += (unsigned long long)m;
                    }
                    if (p.path[(sji - 1) * 3 + s] == c) {
                        long long m = (long long)ndj[s * L + t] - ((s + 1 == sji && t == ti) ? 1 : 0);
                        for (int s1 = 0; s1 < 3; ++s1) m -= tri[(s1 * 3 + s) * L + t];
                        v += (unsigned long long)m;
                    }
                }
                if (kRows) {
                    p.rows[e * S + k] = v;
                } else if (v) {
                    int a = ti, b = tj, cc = t;
                    sort2(a, b);
                    sort2(b, cc);
                    sort2(a, b);
                    atomicAdd(h + (int64_t)c * p.n3 + colex3(a, b, cc), v);
                }
            }
        } else if (kRows) {
            for (int k = lane; k < S; k += 32) p.rows[e * S + k] = 0ull;
        }
        __syncwarp();
    }
    if (!kRows) {
        __syncthreads();
        for (int64_t q = threadIdx.x; q < TG_TRIAD_CLASSES * p.n3; q += blockDim.x)
            if (h[q]) atomicAdd(p.sums + q, h[q]);
    }
}

__global__ void k_dir_finalize(const unsigned long long *sums, uint64_t *out, int64_t n3,
                               unsigned *err) {
    const int64_t len = TG_TRIAD_CLASSES * n3;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < len;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(q / n3);
        const unsigned long long div = (c <= 4 || c == 7) ? 2ull : 3ull;
        if (sums[q] % div) atomicOr(err, TG_DERR_DIVISIBLE);
        out[q] = sums[q] / div;
    }
}

// Per-edge rows (rows != nullptr) or undivided global sums of a TG_DIRECTED graph.
int dir_count(const tg_graph *g, uint64_t *rows, unsigned long long *sums, unsigned *err,
              cudaStream_t s) {
    const TriadTable &tt = triads();
    if (!tt.ok) return TG_EINTERNAL;
    const int L = g->L;
    const int64_t n = g->n, M = g->M;
    if (M == 0) return TG_OK;
    DevBuf<uint32_t> nd;
    DevBuf<unsigned long long> queue;
    if (!nd.alloc((size_t)n * 3 * L, s) || !queue.alloc(1, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(queue.p, 0, 8, s));
    const int64_t ngrid = std::min<int64_t>((n + kDirWarps - 1) / kDirWarps, (int64_t)tg_num_sms() * 16);
    k_dir_degrees<<<(unsigned)ngrid, kDirThreads, 0, s>>>(g->rowptr, g->adj, g->adir, n, L, nd.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    DirParams p{};
    p.rowptr = g->rowptr;
    p.adj = g->adj;
    p.adir = g->adir;
    p.toff = g->toff;
    p.ntype = g->ntype;
    p.edges = g->edges;
    p.nd = nd.p;
    p.M = M;
    p.L = L;
    p.n3 = tg_binom(L + 2, 3);
    p.rows = rows;
    p.sums = sums;
    p.queue = queue.p;
    p.err = err;
    for (int sij = 1; sij <= 3; ++sij)
        for (int s1 = 1; s1 <= 3; ++s1) {
            for (int s2 = 1; s2 <= 3; ++s2)
                p.tri[(sij - 1) * 9 + (s1 - 1) * 3 + (s2 - 1)] =
                    tt.cls[pair_mask(sij, 0, 1) | pair_mask(s1, 0, 2) | pair_mask(s2, 1, 2)];
            // a 3-path: centre 0, ends 1 (state sij) and 2 (state s1), seen from 0
            p.path[(sij - 1) * 3 + (s1 - 1)] = tt.cls[pair_mask(sij, 0, 1) | pair_mask(s1, 0, 2)];
        }
    const void *fn = rows ? (const void *)k_dir3<true> : (const void *)k_dir3<false>;
    const size_t hb = rows ? 0 : (((size_t)TG_TRIAD_CLASSES * p.n3 * 8 + 15) & ~(size_t)15);
    const size_t smem = hb + (size_t)kDirWarps * 9 * L * 4;
    TG_TRY(tg_allow_max_smem(fn));
    int per = 0;
    TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kDirThreads, smem));
    if (per < 1) return TG_ENOMEM;
    const int64_t grid = std::min<int64_t>((int64_t)tg_num_sms() * per, (M + kDirWarps - 1) / kDirWarps);
    if (rows)
        k_dir3<true><<<(unsigned)grid, kDirThreads, smem, s>>>(p);
    else
        k_dir3<false><<<(unsigned)grid, kDirThreads, smem, s>>>(p);
    tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}


// ------------------------------------------------------------- 4 nodes ----
// Directed typed 4-node graphlets: the connected 4-node sets {i, j, w, r}
// through each edge, w in C = (Gamma_i u Gamma_j) \ {i, j} and r either a
// later member of C or a neighbour of w outside C u {i, j} (each set met
// once), classified from their six pair states by a host table.  Classes:
// the 199 connected 4-node digraphs numbered by canonical code (the code of
// a digraph on positions 0..3 is the sum of 2^(4a + b) over its arcs a -> b;
// the canonical code is the smallest over the 24 relabellings).  One warp per
// edge walks the candidate pairs directly: a first form, suited to graphs of
// moderate degree.
constexpr int kDir4Classes = TG_TETRAD_CLASSES;

struct Dir4Table {
    int16_t cls[4096];  // class of each 12-bit pair-state code, -1 if disconnected
    int32_t edges[kDir4Classes];
    bool ok = false;
};

int dir4_canon(int code) {
    static const int perm[24][4] = {
        {0, 1, 2, 3}, {0, 1, 3, 2}, {0, 2, 1, 3}, {0, 2, 3, 1}, {0, 3, 1, 2}, {0, 3, 2, 1},
        {1, 0, 2, 3}, {1, 0, 3, 2}, {1, 2, 0, 3}, {1, 2, 3, 0}, {1, 3, 0, 2}, {1, 3, 2, 0},
        {2, 0, 1, 3}, {2, 0, 3, 1}, {2, 1, 0, 3}, {2, 1, 3, 0}, {2, 3, 0, 1}, {2, 3, 1, 0},
        {3, 0, 1, 2}, {3, 0, 2, 1}, {3, 1, 0, 2}, {3, 1, 2, 0}, {3, 2, 0, 1}, {3, 2, 1, 0}};
    int best = 1 << 30;
    for (int q = 0; q < 24; ++q) {
        int c = 0;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                if (a != b && ((code >> (4 * a + b)) & 1)) c |= 1 << (4 * perm[q][a] + perm[q][b]);
        best = std::min(best, c);
    }
    return best;
}

// arc code of a 12-bit pair-state code (pairs 01, 02, 03, 12, 13, 23, two bits
// each: bit 0 lower -> higher position, bit 1 back) and whether it connects
// the four nodes
int dir4_arcs(int st, bool *conn) {
    static const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {1, 2, 3, 2, 3, 3};
    int code = 0, adj[4] = {0, 0, 0, 0};
    for (int k = 0; k < 6; ++k) {
        const int x = (st >> (2 * k)) & 3;
        if (x & 1) code |= 1 << (4 * pa[k] + pb[k]);
        if (x & 2) code |= 1 << (4 * pb[k] + pa[k]);
        if (x) {
            adj[pa[k]] |= 1 << pb[k];
            adj[pb[k]] |= 1 << pa[k];
        }
    }
    int seen = 1;
    for (int it = 0; it < 4; ++it)
        for (int v = 0; v < 4; ++v)
            if ((seen >> v) & 1) seen |= adj[v];
    *conn = seen == 15;
    return code;
}

Dir4Table build_dir4() {
    Dir4Table t;
    std::vector<int> canon;
    for (int st = 0; st < 4096; ++st) {
        bool conn = false;
        const int code = dir4_arcs(st, &conn);
        if (conn) canon.push_back(dir4_canon(code));
    }
    std::sort(canon.begin(), canon.end());
    canon.erase(std::unique(canon.begin(), canon.end()), canon.end());
    if ((int)canon.size() != kDir4Classes) return t;  // ok stays false
    for (int st = 0; st < 4096; ++st) {
        bool conn = false;
        const int code = dir4_arcs(st, &conn);
        t.cls[st] = conn ? (int16_t)(std::lower_bound(canon.begin(), canon.end(), dir4_canon(code)) -
                                     canon.begin())
                         : (int16_t)-1;
    }
    for (int c = 0; c < kDir4Classes; ++c) {
        int und = 0;
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (((canon[c] >> (4 * a + b)) & 1) || ((canon[c] >> (4 * b + a)) & 1)) ++und;
        t.edges[c] = und;
    }
    t.ok = true;
    return t;
}

const Dir4Table &dir4_table() {
    static std::once_flag once;
    static Dir4Table t;
    std::call_once(once, [] { t = build_dir4(); });
    return t;
}

struct Dir4Params {
    const int64_t *rowptr;
    const uint32_t *adj;
    const uint8_t *adir;
    const int32_t *toff;
    const uint8_t *ntype;
    const int2 *edges;
    const int16_t *cls;  // 4096 entries (device)
    int64_t M;
    int32_t L, P;
    int64_t n4;                // C(L+3, 4)
    unsigned long long *rows;  // per-edge mode: M x 199 P
    unsigned long long *sums;  // global mode: 199 n4 undivided sums
    unsigned long long *queue;
    unsigned *err;
};

// state of the pair (x, w) seen from x: the arc bits of w's entry in Gamma_x, 0 if absent
__device__ __forceinline__ int dir4_state(const Dir4Params &p, int64_t bx, const int32_t *tox,
                                          uint32_t w) {
    const int q = find_pos(p.adj, bx, tox, w);
    return q < 0 ? 0 : (int)p.adir[bx + q];
}

template <bool kRows>
__global__ void __launch_bounds__(kDirThreads) k_dir4(Dir4Params p) {
    const int lane = threadIdx.x & 31;
    const int L = p.L;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(p.queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= (unsigned long long)p.M) break;
        const int64_t e = (int64_t)item;
        const int2 ab = p.edges[e];
        const uint32_t i = (uint32_t)ab.x, j = (uint32_t)ab.y;
        const int ti = p.ntype[i], tj = p.ntype[j];
        const int64_t bi = p.rowptr[i], bj = p.rowptr[j];
        const int di = (int)(p.rowptr[i + 1] - bi), dj = (int)(p.rowptr[j + 1] - bj);
        const int32_t *toi = p.toff + (int64_t)i * (L + 1);
        const int32_t *toj = p.toff + (int64_t)j * (L + 1);
        const int sij = dir4_state(p, bi, toi, ((uint32_t)tj << TG_TSHIFT) | j);
        // member q of C (index space [0, di + dj)): its entry, or 0xffffffff
        // when q is i, j, or a member of Gamma_j already in Gamma_i
        auto member = [&](int q) -> uint32_t {
            if (q < di) {
                const uint32_t w = __ldg(p.adj + bi + q);
                return (w & TG_IDMASK) == j ? 0xffffffffu : w;
            }
            const uint32_t w = __ldg(p.adj + bj + (q - di));
            if ((w & TG_IDMASK) == i || find_pos(p.adj, bi, toi, w) >= 0) return 0xffffffffu;
            return w;
        };
        const int nq = di + dj;
        for (int pw = 0; pw < nq; ++pw) {
            const uint32_t wE = member(pw);  // the same in every lane
            if (wE == 0xffffffffu) continue;
            const uint32_t w = wE & TG_IDMASK;
            const int tw = (int)(wE >> TG_TSHIFT);
            const int siw = pw < di ? (int)p.adir[bi + pw] : 0;
            const int sjw = pw < di ? dir4_state(p, bj, toj, wE) : (int)p.adir[bj + (pw - di)];
            const int64_t bw = p.rowptr[w];
            const int dw = (int)(p.rowptr[w + 1] - bw);
            const int32_t *tow = p.toff + (int64_t)w * (L + 1);
            // pass 0: r a later member of C; pass 1: r a neighbour of w outside C u {i, j}
            const int n0 = nq - (pw + 1);
            for (int x = lane; x < n0 + dw; x += 32) {
                uint32_t rE;
                int sir, sjr, swr;
                if (x < n0) {
                    const int pr = pw + 1 + x;
                    rE = member(pr);
                    if (rE == 0xffffffffu) continue;
                    sir = pr < di ? (int)p.adir[bi + pr] : 0;
                    sjr = pr < di ? dir4_state(p, bj, toj, rE) : (int)p.adir[bj + (pr - di)];
                    swr = dir4_state(p, bw, tow, rE);
                } else {
                    const int xr = x - n0;
                    rE = __ldg(p.adj + bw + xr);
                    const uint32_t r = rE & TG_IDMASK;
                    if (r == i || r == j || find_pos(p.adj, bi, toi, rE) >= 0 ||
                        find_pos(p.adj, bj, toj, rE) >= 0)
                        continue;
                    sir = 0;
                    sjr = 0;
                    swr = (int)p.adir[bw + xr];
                }
                // positions i = 0, j = 1, w = 2, r = 3; each state seen from the lower position
                const int code = sij | (siw << 2) | (sir << 4) | (sjw << 6) | (sjr << 8) | (swr << 10);
                const int c = p.cls[code];
                if (c < 0) {
                    atomicOr(p.err, TG_DERR_BOUNDS);  // a set through the edge is always connected
                    continue;
                }
                const int tr = (int)(rE >> TG_TSHIFT);
                if (kRows) {
                    const int a = min(tw, tr), b = max(tw, tr);
                    atomicAdd(p.rows + e * (int64_t)kDir4Classes * p.P + (int64_t)c * p.P +
                                  (a * L - (a * (a - 1)) / 2 + (b - a)),
                              1ull);
                } else {
                    int q0 = ti, q1 = tj, q2 = tw, q3 = tr;
                    sort2(q0, q1);
                    sort2(q2, q3);
                    sort2(q0, q2);
                    sort2(q1, q3);
                    sort2(q1, q2);
                    atomicAdd(p.sums + (int64_t)c * p.n4 + colex4(q0, q1, q2, q3), 1ull);
                }
            }
        }
    }
}

__global__ void k_dir4_finalize(const unsigned long long *sums, uint64_t *out, int64_t n4,
                                const int32_t *cls_edges, unsigned *err) {
    const int64_t len = (int64_t)kDir4Classes * n4;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < len;
         q += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long div = (unsigned long long)cls_edges[q / n4];
        if (sums[q] % div) atomicOr(err, TG_DERR_DIVISIBLE);
        out[q] = sums[q] / div;
    }
}

// Per-edge rows (rows != nullptr, zeroed here) or undivided global sums (zeroed by the caller).
int dir4_count(const tg_graph *g, unsigned long long *rows, unsigned long long *sums, unsigned *err,
               cudaStream_t s) {
    const Dir4Table &tt = dir4_table();
    if (!tt.ok) return TG_EINTERNAL;
    const int L = g->L;
    const int64_t M = g->M;
    if (M == 0) return TG_OK;
    DevBuf<int16_t> cls;
    DevBuf<unsigned long long> queue;
    if (!cls.alloc(4096, s) || !queue.alloc(1, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemcpyAsync(cls.p, tt.cls, 4096 * sizeof(int16_t), cudaMemcpyHostToDevice, s));
    TG_TRY_CUDA(cudaMemsetAsync(queue.p, 0, 8, s));
    Dir4Params p{};
    p.rowptr = g->rowptr;
    p.adj = g->adj;
    p.adir = g->adir;
    p.toff = g->toff;
    p.ntype = g->ntype;
    p.edges = g->edges;
    p.cls = cls.p;
    p.M = M;
    p.L = L;
    p.P = L * (L + 1) / 2;
    p.n4 = tg_binom(L + 3, 4);
    p.rows = rows;
    p.sums = sums;
    p.queue = queue.p;
    p.err = err;
    if (rows)
        TG_TRY_CUDA(cudaMemsetAsync(rows, 0, (size_t)M * kDir4Classes * p.P * 8, s));
    const int64_t grid = std::min<int64_t>((int64_t)tg_num_sms() * 8, (M + kDirWarps - 1) / kDirWarps);
    if (rows)
        k_dir4<true><<<(unsigned)grid, kDirThreads, 0, s>>>(p);
    else
        k_dir4<false><<<(unsigned)grid, kDirThreads, 0, s>>>(p);
    tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}

int check_dir(const tg_graph *g) {
    if (!g || !g->adir) return TG_EINVAL;
    return TG_OK;
}

}  // namespace

int tg_attach_arcs(tg_graph *g, const int32_t *src, const int32_t *dst, int64_t m,
                   const int32_t *old2new, cudaStream_t s) {
    const int64_t words = (2 * g->M + 3) / 4;
    g->adir = (uint8_t *)tg_dalloc((size_t)std::max<int64_t>(1, words) * 4, s);
    if (!g->adir) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(g->adir, 0, (size_t)std::max<int64_t>(1, words) * 4, s));
    if (m == 0 || g->M == 0) return TG_OK;
    DevBuf<unsigned> err;
    if (!err.alloc(1, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(err.p, 0, 4, s));
    const unsigned grid = (unsigned)std::min<int64_t>((m + 255) / 256, 65535LL * 16);
    k_arc_bits<<<grid, 256, 0, s>>>(src, dst, m, old2new, g->rowptr, g->adj, g->toff, g->ntype,
                                    g->L, reinterpret_cast<uint32_t *>(g->adir), err.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    unsigned herr = 0;
    TG_TRY_CUDA(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return herr ? TG_EINTERNAL : TG_OK;
}

extern "C" int64_t tg_dir_slots(int32_t L) {
    if (L < 1 || L > TG_MAX_TYPES) return -1;
    return (int64_t)TG_TRIAD_CLASSES * L;
}

extern "C" int64_t tg_dir_global_len(int32_t L) {
    if (L < 1 || L > TG_MAX_TYPES) return -1;
    return (int64_t)TG_TRIAD_CLASSES * tg_binom(L + 2, 3);
}

extern "C" int tg_count_directed_per_edge(const tg_graph *g, uint64_t *rows, void *stream) {
    TG_TRY(check_dir(g));
    if (!rows) return TG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->M == 0) return TG_OK;
    const int64_t width = tg_dir_slots(g->L);
    DevBuf<unsigned> err;
    if (!err.alloc(1, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(err.p, 0, 4, s));
    DevBuf<uint64_t> tmp;
    uint64_t *dst = rows;
    const bool dev_out = tg_is_device_ptr(rows);
    if (!dev_out) {
        if (!tmp.alloc((size_t)g->M * width, s)) return TG_ENOMEM;
        dst = tmp.p;
    }
    TG_TRY(dir_count(g, dst, nullptr, err.p, s));
    unsigned herr = 0;
    TG_TRY_CUDA(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, s));
    if (!dev_out)
        TG_TRY_CUDA(cudaMemcpyAsync(rows, dst, (size_t)g->M * width * 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return herr ? TG_EINTERNAL : TG_OK;
}

extern "C" int tg_count_directed_global(const tg_graph *g, uint64_t *out, void *stream) {
    TG_TRY(check_dir(g));
    if (!out) return TG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t len = tg_dir_global_len(g->L);
    DevBuf<unsigned long long> sums;
    DevBuf<unsigned> err;
    if (!sums.alloc(len, s) || !err.alloc(1, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(sums.p, 0, len * 8, s));
    TG_TRY_CUDA(cudaMemsetAsync(err.p, 0, 4, s));
    TG_TRY(dir_count(g, nullptr, sums.p, err.p, s));
    const bool dev_out = tg_is_device_ptr(out);
    DevBuf<uint64_t> tmp;
    uint64_t *dst = out;
    if (!dev_out) {
        if (!tmp.alloc(len, s)) return TG_ENOMEM;
        dst = tmp.p;
    }
    const unsigned grid = (unsigned)std::min<int64_t>((len + 255) / 256, 4096);
    k_dir_finalize<<<grid, 256, 0, s>>>(sums.p, dst, tg_binom(g->L + 2, 3), err.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    unsigned herr = 0;
    TG_TRY_CUDA(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, s));
    if (!dev_out) TG_TRY_CUDA(cudaMemcpyAsync(out, dst, len * 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return herr ? TG_EINTERNAL : TG_OK;
}

extern "C" int64_t tg_dir4_slots(int32_t L) {
    if (L < 1 || L > TG_MAX_TYPES) return -1;
    return (int64_t)kDir4Classes * (L * (L + 1) / 2);
}

extern "C" int64_t tg_dir4_global_len(int32_t L) {
    if (L < 1 || L > TG_MAX_TYPES) return -1;
    return (int64_t)kDir4Classes * tg_binom(L + 3, 4);
}

extern "C" int tg_count_directed4_per_edge(const tg_graph *g, uint64_t *rows, void *stream) {
    TG_TRY(check_dir(g));
    if (!rows) return TG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->M == 0) return TG_OK;
    const int64_t width = tg_dir4_slots(g->L);
    DevBuf<unsigned> err;
    if (!err.alloc(1, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(err.p, 0, 4, s));
    DevBuf<uint64_t> tmp;
    uint64_t *dst = rows;
    const bool dev_out = tg_is_device_ptr(rows);
    if (!dev_out) {
        if (!tmp.alloc((size_t)g->M * width, s)) return TG_ENOMEM;
        dst = tmp.p;
    }
    TG_TRY(dir4_count(g, reinterpret_cast<unsigned long long *>(dst), nullptr, err.p, s));
    unsigned herr = 0;
    TG_TRY_CUDA(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, s));
    if (!dev_out)
        TG_TRY_CUDA(cudaMemcpyAsync(rows, dst, (size_t)g->M * width * 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return herr ? TG_EINTERNAL : TG_OK;
}

extern "C" int tg_count_directed4_global(const tg_graph *g, uint64_t *out, void *stream) {
    TG_TRY(check_dir(g));
    if (!out) return TG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const Dir4Table &tt = dir4_table();
    if (!tt.ok) return TG_EINTERNAL;
    const int64_t len = tg_dir4_global_len(g->L);
    DevBuf<unsigned long long> sums;
    DevBuf<unsigned> err;
    DevBuf<int32_t> ce;
    if (!sums.alloc(len, s) || !err.alloc(1, s) || !ce.alloc(kDir4Classes, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(sums.p, 0, len * 8, s));
    TG_TRY_CUDA(cudaMemsetAsync(err.p, 0, 4, s));
    TG_TRY_CUDA(cudaMemcpyAsync(ce.p, tt.edges, kDir4Classes * 4, cudaMemcpyHostToDevice, s));
    TG_TRY(dir4_count(g, nullptr, sums.p, err.p, s));
    const bool dev_out = tg_is_device_ptr(out);
    DevBuf<uint64_t> tmp;
    uint64_t *dst = out;
    if (!dev_out) {
        if (!tmp.alloc(len, s)) return TG_ENOMEM;
        dst = tmp.p;
    }
    const unsigned grid = (unsigned)std::min<int64_t>((len + 255) / 256, 4096);
    k_dir4_finalize<<<grid, 256, 0, s>>>(sums.p, dst, tg_binom(g->L + 3, 4), ce.p, err.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    unsigned herr = 0;
    TG_TRY_CUDA(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, s));
    if (!dev_out) TG_TRY_CUDA(cudaMemcpyAsync(out, dst, len * 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return herr ? TG_EINTERNAL : TG_OK;
}
