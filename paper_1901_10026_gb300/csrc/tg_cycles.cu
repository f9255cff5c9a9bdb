// Per-edge counts of Alg. 2-3 from two whole-graph enumerations.
//
// The identities in tg_reuse.cu express every enumerated orbit of Alg. 2-3
// through Alg. 1's typed triangle counts tau, per-node sums of tau and of the
// typed degrees, sums over the triangle nodes T_ij, and two more per-edge
// quantities that the paper obtains by walking the neighbour lists of
// S_i u S_j u T_ij:
//   C4_ij[a][b] = ordered pairs (x in Gamma_i^a \ {j}, w in Gamma_j^b \ {i})
//                 with x ~ w, i.e. the non-induced 4-cycles i-j-w-x through
//                 the edge; the 4-cycle term of the identities is
//                 S6 = C4 - B + [b = phi_i] |T^a|
//                 (the x in T part of C4 is sum over y in T^a of tau_jy[b],
//                 less i itself);
//   Q_ij[a][b]  = ordered adjacent pairs (y in T^a, z in T^b), i.e. the
//                 4-cliques through the edge.
// Here both are accumulated per edge from enumerations of the whole graph in
// degree order (a node ranks higher when its new id is smaller):
//   4-cycles: each non-induced 4-cycle a-u-b-u' is met once, at its
//     highest-ranked node a, as two wedges a-u-b and a-u'-b whose other nodes
//     rank below a.  Per anchor a, pass 1 counts the middles u of the wedges
//     ending at each b by type (c_t(b)); pass 2 adds, for every wedge, the
//     cycles it closes with the other middles to its two edges (per-edge
//     mode); the far ends then add C(c_t, 2) and c_t c_t' (global mode) and
//     clear the counters.  Global mode keeps the counters of light anchors in
//     shared memory (k_c4_warp, k_c4_cta) and walks costly ones in warp units
//     over L2-sized waves of counter slots (k_c4_walk, k_c4_pairs).
//   4-cliques (k_k4): each 4-clique x0 < v < w < x (by rank) is met once from
//     its lowest node along "up" lists (neighbours of higher rank) and adds one
//     to each of its six edges, keyed by the unordered types of the two nodes
//     off the edge.
// The enumeration work is the number of degree-ordered wedges plus the
// 4-clique search, instead of sum over w in S_i u S_j u T_ij of d_w per edge.
// The per-edge pass (tg_edges.cu) then needs only Gamma_i n Gamma_j (the T
// sums) and O(L^2) identity and closed-form arithmetic.
#include <algorithm>
#include <new>
#include <vector>

#include "tg_device.cuh"

using namespace tgd;

namespace {

// Inclusive block scan of a packed (count << 52 | length) word; returns the
// inclusive value of this thread and leaves the block total in wsum[32].
__device__ __forceinline__ uint64_t block_scan_packed(uint64_t v, uint64_t *wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    uint64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint64_t y = lane < W ? wsum[lane] : 0ull;
        const uint64_t y0 = y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t z = __shfl_up_sync(kFull, y, o);
            if (lane >= o) y += z;
        }
        if (lane < W) wsum[lane] = y - y0;
        if (lane == W - 1) wsum[32] = y;
    }
    __syncthreads();
    return incl + wsum[warp];
}

constexpr uint64_t kLenMask = ((uint64_t)1 << 41) - 1;

// ------------------------------------------------------------ 4-cycles ----
struct C4Params {
    const int64_t *rowptr;
    const uint32_t *adj;
    const uint32_t *eid;
    const uint8_t *ntype;
    int64_t n;
    int32_t L;
    int32_t tile;              // members staged per tile (<= blockDim.x)
    int32_t acc_l2;            // L * L in per-edge mode, 0 in global mode
    uint32_t *scratch;         // slots of n * L counters (per far end, per type), an
                               // n-entry list of the far ends met and a bitmap of them
                               // (n bits); counters and bitmap zero on entry and on exit
    int64_t slot_words;
    unsigned long long *queue;
    unsigned long long *c4e;   // per-edge mode: M * L * L, [type next to i][type next to j]
    unsigned long long *g4;    // global mode: C(L+3,4) non-induced 4-cycles by type multiset
    int64_t n4;
    const int4 *units;         // split kernel: (slot, anchor, first member, end member)
    const struct C4Unit *wunits;  // walk kernel: position ranges of the split anchors
    int64_t n_units;
    int32_t phase;             // split kernel: the pass of this launch
    int32_t mark;              // pass 0 marks far ends in the slot's bitmap
    unsigned long long *work;  // [4]: wedges
    // dense waves (global mode): the costly anchors heavy[q], their walk
    // positions (member costs d_u, exclusive prefix per anchor at pbase[q]),
    // and the first anchor index of the wave (slot = q - q0)
    const uint32_t *heavy;
    const int64_t *mprefix;
    const int64_t *pbase;
    int64_t q0;
    // slot layout: 32-bit counts at b L + t (half = 0) or 16-bit counts at
    // b Lp + t, Lp = L rounded up to even, two to a word (half = 1); the
    // far-end bitmap starts at word bits_off of the slot
    int32_t half;
    int64_t bits_off;
};

// A warp unit of k_c4_walk: positions [lo, hi) of the walk of split anchor
// q, starting in the list of its member m.
struct C4Unit {
    int64_t lo, hi;
    int32_t q, m;
};

constexpr int kC4Threads = 256;
constexpr int64_t kWaveMax = 128;       // costly anchors of one wave (global mode), at most
constexpr int64_t kWalkUnitMin = 512;    // walk positions of a warp unit, at least

struct C4Smem {
    int64_t *m_end, *m_org;
    uint64_t *wsum;
    unsigned long long *acc;
    uint32_t *m_u, *m_e;
    unsigned long long *s_item, *h4;
    unsigned int *s_nb;
};

__device__ __forceinline__ C4Smem c4_smem(unsigned char *smem, int TM, int acc_l2) {
    C4Smem m;
    m.m_end = reinterpret_cast<int64_t *>(smem);
    m.m_org = m.m_end + TM;
    m.wsum = reinterpret_cast<uint64_t *>(m.m_org + TM);
    m.acc = reinterpret_cast<unsigned long long *>(m.wsum + 34);
    m.m_u = reinterpret_cast<uint32_t *>(m.acc + (size_t)TM * acc_l2);
    m.m_e = m.m_u + TM;
    m.s_item = reinterpret_cast<unsigned long long *>(m.m_e + TM + (TM & 1));
    m.s_nb = reinterpret_cast<unsigned int *>(m.s_item + 1);
    m.h4 = m.s_item + 2;  // global mode: n4 entries
    return m;
}

// One pass over one tile of anchor a's list (list positions [tile, tile_end),
// at most p.tile of them): the members u (neighbours ranked below a) of the
// tile and, for each, the entries b of u's list ranked below a.  The members'
// lists are walked as one sequence of positions, of which only [pos_lo, pos_hi)
// is taken.  Pass 0 counts the middles per (b, type), and lists each b the
// first time it is met (in `list`, count in *nb) or marks it in the slot's
// bitmap (p.mark); pass 1 (per-edge mode only) adds the cycles each wedge
// closes to its two edges.  Returns the length of the tile's sequence.  Called
// by every thread of the CTA (it holds barriers).
__device__ int64_t c4_tile(const C4Params &p, const C4Smem &sm, uint32_t a, int ta, int64_t ba,
                           int tile, int tile_end, int64_t pos_lo, int64_t pos_hi, int phase,
                           uint32_t *cnt, uint32_t *list, unsigned int *nb,
                           unsigned long long &wk) {
    const int tid = threadIdx.x;
    const int L = p.L, L2 = L * L, TM = p.tile;
    const int x = tile + tid;
    bool mem = false;
    uint32_t wu = 0;
    int64_t bu = 0;
    int du = 0;
    if (tid < TM && x < tile_end) {
        wu = __ldg(p.adj + ba + x);
        const uint32_t u = wu & TG_IDMASK;
        if (u > a) {
            bu = p.rowptr[u];
            du = (int)(p.rowptr[u + 1] - bu);
            mem = du > 1;
        }
    }
    const uint64_t incl = block_scan_packed(((uint64_t)mem << 52) | (uint64_t)(mem ? du : 0), sm.wsum);
    const uint64_t tot = sm.wsum[32];
    const int nmem = (int)(tot >> 52);
    const int64_t total = (int64_t)(tot & kLenMask);
    if (mem) {
        const int r = (int)((incl >> 52) - 1);
        const int64_t end = (int64_t)(incl & kLenMask);
        sm.m_end[r] = end;
        sm.m_org[r] = bu - (end - du);
        sm.m_u[r] = wu;
        sm.m_e[r] = __ldg(p.eid + ba + x);
    }
    if (phase == 1)
        for (int q = tid; q < nmem * L2; q += blockDim.x) sm.acc[q] = 0ull;
    __syncthreads();
    const int64_t lim = total < pos_hi ? total : pos_hi;
    for (int64_t base = pos_lo > 0 ? pos_lo : 0; base < lim; base += blockDim.x) {
        const int64_t pos = base + tid;
        if (pos >= lim) continue;
        int lo = 0, hi = nmem - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sm.m_end[mid] > pos)
                hi = mid;
            else
                lo = mid + 1;
        }
        const int64_t at = sm.m_org[lo] + pos;
        const uint32_t wb = __ldg(p.adj + at);
        const uint32_t b = wb & TG_IDMASK;
        if (b <= a) continue;  // b must rank below a (and differ from it)
        const uint32_t wmu = sm.m_u[lo];
        const int tu = (int)(wmu >> TG_TSHIFT);
        uint32_t *cb = cnt + (int64_t)b * L;
        if (phase == 0) {
            atomicAdd(cb + tu, 1u);  // result unused: no round trip
            uint32_t *bw = cnt + p.n * (L + 1) + (b >> 5);
            const uint32_t bit = 1u << (b & 31u);
            if (list) {
                // the first wedge to reach b lists it
                if (!(atomicOr(bw, bit) & bit)) list[atomicAdd(nb, 1u)] = b;
            } else if (p.mark) {
                atomicOr(bw, bit);  // marks b for the scan of k_c4_pairs
            }
            ++wk;
            continue;
        }
        uint32_t c[TG_MAX_TYPES];
        uint32_t sum = 0;
#pragma unroll
        for (int t = 0; t < TG_MAX_TYPES; ++t) {
            c[t] = t < L ? __ldcg(cb + t) : 0u;
            sum += c[t];
        }
        if (sum < 2u) continue;  // no other middle: no cycle
        const int tb = (int)(wb >> TG_TSHIFT);
        const uint32_t u = wmu & TG_IDMASK;
        unsigned long long *row_ub = p.c4e + (int64_t)__ldg(p.eid + at) * L2;
        unsigned long long *row_au = sm.acc + (int64_t)lo * L2 + tb * L;
#pragma unroll
        for (int t = 0; t < TG_MAX_TYPES; ++t) {
            if (t < L) {
                const uint32_t v = c[t] - (t == tu ? 1u : 0u);
                if (v) {
                    // edge (u, b): u's cycle neighbour a, b's is u' (type t);
                    // the row is keyed from its larger-id end
                    atomicAdd(row_ub + (u > b ? ta * L + t : t * L + ta), (unsigned long long)v);
                    // edge (a, u): u (the larger id) sees b, a sees u'
                    atomicAdd(row_au + t, (unsigned long long)v);
                }
            }
        }
    }
    __syncthreads();
    if (phase == 1) {
        for (int q = tid; q < nmem * L2; q += blockDim.x) {
            const unsigned long long v = sm.acc[q];
            if (v) atomicAdd(p.c4e + (int64_t)sm.m_e[q / L2] * L2 + (q % L2), v);
        }
        __syncthreads();
    }
    return total;
}

// Far end b of anchor a (counters cb, per type): global mode adds the cycles
// per type pair of middles (C(c_t, 2) for t = t', c_t c_t' for t < t') under
// the multiset {a, b, t, t'}; both modes then clear b's counters.
// The cycles of one far end b (type tb) of an anchor of type ta, from its
// middle counts c[t] (t < L): C(c_t, 2) for t = t' and c_t c_t' for t < t',
// each under the multiset {ta, tb, t, t'}, into the shared histogram h4.  Only
// the types with a non-zero count are visited.
__device__ __forceinline__ void c4_add(unsigned long long *h4, int L, int ta, int tb,
                                       const uint32_t *c) {
    uint32_t mask = 0;
    for (int t = 0; t < L; ++t)
        if (c[t]) mask |= 1u << t;
    int s0 = ta, s1 = tb;
    sort2(s0, s1);
    for (uint32_t mt = mask; mt; mt &= mt - 1u) {
        const int t = __ffs(mt) - 1;
        const unsigned long long ct = c[t];
        if (ct > 1) {
            int q0 = s0, q1 = s1, q2 = t, q3 = t;
            sort2(q0, q2);
            sort2(q1, q3);
            sort2(q1, q2);
            atomicAdd(h4 + colex4(q0, q1, q2, q3), ct * (ct - 1) / 2);
        }
        for (uint32_t mu = mt & (mt - 1u); mu; mu &= mu - 1u) {
            const int u = __ffs(mu) - 1;
            int q0 = s0, q1 = s1, q2 = t, q3 = u;
            sort2(q0, q2);
            sort2(q1, q3);
            sort2(q1, q2);
            atomicAdd(h4 + colex4(q0, q1, q2, q3), ct * c[u]);
        }
    }
}

__device__ __forceinline__ void c4_one(const C4Params &p, unsigned long long *h4, int ta,
                                       uint32_t *cb, uint32_t b) {
    const int L = p.L;
    uint32_t c[TG_MAX_TYPES];
    uint32_t sum = 0;
    for (int t = 0; t < L; ++t) {
        c[t] = __ldcg(cb + t);
        sum += c[t];
    }
    if (p.g4 && sum > 1) c4_add(h4, L, ta, p.ntype[b], c);  // one middle closes no cycle
    for (int t = 0; t < L; ++t)
        if (c[t]) cb[t] = 0u;
}

// c4_one for a 16-bit slot: b's counts are the halves of its (L + 1) / 2
// words at cw (low half the even type), words no other far end shares.
__device__ __forceinline__ void c4_one16(const C4Params &p, unsigned long long *h4, int ta,
                                         uint32_t *cw, uint32_t b) {
    const int L = p.L, nw = (L + 1) >> 1;
    uint32_t c[TG_MAX_TYPES];
    uint32_t sum = 0;
    for (int q = 0; q < nw; ++q) {
        const uint32_t w = __ldcg(cw + q);
        c[2 * q] = w & 0xffffu;
        if (2 * q + 1 < L) c[2 * q + 1] = w >> 16;
        sum += (w & 0xffffu) + (w >> 16);
        if (w) cw[q] = 0u;
    }
    if (p.g4 && sum > 1) c4_add(h4, L, ta, p.ntype[b], c);  // one middle closes no cycle
}

// Position of the j-th (from 0) set bit of m; m has more than j set bits.
__device__ __forceinline__ int select_bit(uint32_t m, int j) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (j >= c) {
            j -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// The listed far ends of anchor a (entries q0, q0 + step, ... < nb).
__device__ __forceinline__ void c4_pairs(const C4Params &p, const C4Smem &sm, int ta,
                                         uint32_t *cnt, const uint32_t *list, unsigned int nb,
                                         unsigned int q0, unsigned int step) {
    for (unsigned int q = q0; q < nb; q += step) {
        const uint32_t b = __ldcg(list + q);  // written by other threads this anchor
        c4_one(p, sm.h4, ta, cnt + (int64_t)b * p.L, b);
        cnt[p.n * (p.L + 1) + (b >> 5)] = 0u;  // every set bit of the word is listed
    }
}

__device__ __forceinline__ void c4_finish(const C4Params &p, const C4Smem &sm,
                                          unsigned long long wk) {
    if (p.g4) {
        __syncthreads();
        for (int64_t q = threadIdx.x; q < p.n4; q += blockDim.x)
            if (sm.h4[q]) atomicAdd(p.g4 + q, sm.h4[q]);
    }
    if (p.work && wk) atomicAdd(p.work + 4, wk);
}

// The anchors of alist: one CTA per anchor, the passes in turn over the CTA's
// own counter slot.
__global__ void __launch_bounds__(kC4Threads) k_c4(C4Params p, const uint32_t *alist, int64_t na) {
    extern __shared__ __align__(16) unsigned char smem[];
    const C4Smem sm = c4_smem(smem, p.tile, p.acc_l2);
    const int tid = threadIdx.x;
    if (p.g4)
        for (int64_t q = tid; q < p.n4; q += blockDim.x) sm.h4[q] = 0ull;
    uint32_t *cnt = p.scratch + (int64_t)blockIdx.x * p.slot_words;
    uint32_t *list = cnt + p.n * p.L;
    unsigned long long wk = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) *sm.s_item = atomicAdd(p.queue, 1ull);
        __syncthreads();
        const unsigned long long item = *sm.s_item;
        if (item >= (unsigned long long)na) break;
        const uint32_t a = alist[item];
        const int64_t ba = p.rowptr[a];
        const int da = (int)(p.rowptr[a + 1] - ba);
        if (da < 2) continue;  // a cycle through a needs two of its neighbours
        const int ta = p.ntype[a];
        if (tid == 0) *sm.s_nb = 0u;
        __syncthreads();
        for (int tile = 0; tile < da; tile += p.tile)
            c4_tile(p, sm, a, ta, ba, tile, min(da, tile + p.tile), 0, INT64_MAX, 0, cnt, list,
                    sm.s_nb, wk);
        if (!p.g4)
            for (int tile = 0; tile < da; tile += p.tile)
                c4_tile(p, sm, a, ta, ba, tile, min(da, tile + p.tile), 0, INT64_MAX, 1, cnt, list,
                        sm.s_nb, wk);
        __syncthreads();
        c4_pairs(p, sm, ta, cnt, list, *sm.s_nb, tid, blockDim.x);
    }
    c4_finish(p, sm, wk);
}

// Marked (costly) anchors: their tiles are units spread over the whole grid,
// each anchor on a counter slot of its own; one launch per pass, so a pass
// sees every count of the pass before it.
__global__ void __launch_bounds__(kC4Threads) k_c4_split(C4Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const C4Smem sm = c4_smem(smem, p.tile, p.acc_l2);
    const int tid = threadIdx.x;
    if (p.g4)
        for (int64_t q = tid; q < p.n4; q += blockDim.x) sm.h4[q] = 0ull;
    unsigned long long wk = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) *sm.s_item = atomicAdd(p.queue, 1ull);
        __syncthreads();
        const unsigned long long item = *sm.s_item;
        if (item >= (unsigned long long)p.n_units) break;
        const int4 un = p.units[item];
        const uint32_t a = (uint32_t)un.y;
        const int64_t ba = p.rowptr[a];
        uint32_t *cnt = p.scratch + (int64_t)un.x * p.slot_words;
        c4_tile(p, sm, a, p.ntype[a], ba, un.z, un.w, 0, INT64_MAX, p.phase, cnt, nullptr, nullptr,
                wk);
    }
    c4_finish(p, sm, wk);
}

// The far ends of the wave's split anchors (na slots, anchors[slot] the
// anchor of a slot), from the slots' bitmaps: each warp takes 32 bitmap words
// at a time, lists their set bits across the lanes (a scan of the words'
// popcounts) and treats 32 far ends per step, one per lane.  Clears the bitmap
// words it reads.  Shared memory: the type-multiset histogram, one copy per
// warp when `priv` (else one per CTA).
__global__ void __launch_bounds__(kC4Threads) k_c4_pairs(C4Params p, const uint32_t *anchors,
                                                         int na, int priv) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *h4all = reinterpret_cast<unsigned long long *>(smem);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int copies = priv ? (int)(blockDim.x >> 5) : 1;
    if (p.g4) {
        for (int64_t q = threadIdx.x; q < p.n4 * copies; q += blockDim.x) h4all[q] = 0ull;
        __syncthreads();
    }
    unsigned long long *h4 = h4all + (priv ? (int64_t)warp * p.n4 : 0);
    const int L = p.L;
    const int64_t words = (p.n + 31) >> 5;
    const int64_t cps = (words + 31) >> 5;  // chunks of 32 words per slot
    const int64_t total = (int64_t)na * cps;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < total; c += nw) {
        const int64_t slot = c / cps, wc = c - slot * cps;
        uint32_t *cnt = p.scratch + slot * p.slot_words;
        uint32_t *bw = cnt + p.bits_off;
        const int64_t wi = wc * 32 + lane;
        uint32_t m = 0;
        if (wi < words) {
            m = __ldcg(bw + wi);
            if (m) bw[wi] = 0u;
        }
        const int k = __popc(m);
        int incl = k;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int tot = __shfl_sync(kFull, incl, 31);
        if (tot == 0) continue;
        const int ta = p.ntype[anchors[slot]];
        for (int base = 0; base < tot; base += 32) {
            const int kk = base + lane;
            int r = 0;  // the lane whose word holds far end kk
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int v = __shfl_sync(kFull, incl, r + st - 1);
                if (v <= kk) r += st;
            }
            const uint32_t mr = __shfl_sync(kFull, m, r);
            const int er = __shfl_sync(kFull, incl - k, r);
            if (kk < tot) {
                const uint32_t b = (uint32_t)((wc * 32 + r) * 32 + select_bit(mr, kk - er));
                if (p.half)
                    c4_one16(p, h4, ta, cnt + (int64_t)b * ((L + 1) >> 1), b);
                else
                    c4_one(p, h4, ta, cnt + (int64_t)b * L, b);
            }
        }
    }
    if (p.g4) {
        __syncthreads();
        for (int64_t q = threadIdx.x; q < p.n4; q += blockDim.x) {
            unsigned long long v = 0;
            for (int cpy = 0; cpy < copies; ++cpy) v += h4all[cpy * p.n4 + q];
            if (v) atomicAdd(p.g4 + q, v);
        }
    }
}

// ------------------------------------------------- dense waves (global) ----
// Costly anchors when a few counter slots of n L words fit in L2: a wave of
// anchors counts into its slots with fire-and-forget adds only (no far-end
// bitmap), and k_c4_dense_pairs then scans the slots densely.  Work units cut
// each anchor's walk (its members' lists in order) into position ranges of
// about equal length, so one hub member's long list spreads over many CTAs.

// Walk positions of the costly anchors: member x of heavy[q] costs d_u when it
// is a member (u ranked below the anchor, d_u > 1), else 0; mprefix holds the
// exclusive prefix from pbase[q], totals[q] the sum.  One CTA per anchor.
__global__ void k_c4_prefix(const uint32_t *heavy, const int64_t *pbase, const int64_t *rowptr,
                            const uint32_t *adj, int64_t *mprefix, unsigned long long *totals) {
    __shared__ uint64_t wsum[34];
    const int64_t q = blockIdx.x;
    const uint32_t a = heavy[q];
    const int64_t ba = rowptr[a];
    const int da = (int)(rowptr[a + 1] - ba);
    int64_t *out = mprefix + pbase[q];
    uint64_t run = 0;
    for (int c = 0; c < da; c += blockDim.x) {
        const int x = c + threadIdx.x;
        uint64_t v = 0;
        if (x < da) {
            const uint32_t u = __ldg(adj + ba + x) & TG_IDMASK;
            if (u > a) {
                const int64_t du = rowptr[u + 1] - rowptr[u];
                v = du > 1 ? (uint64_t)du : 0ull;
            }
        }
        const uint64_t incl = block_scan_packed(v, wsum);
        if (x < da) out[x] = (int64_t)(run + incl - v);
        run += wsum[32];
        __syncthreads();  // wsum is rewritten by the next chunk's scan
    }
    if (threadIdx.x == 0) totals[q] = run;
}

// Units of the walk waves: unit u belongs to anchor q with ustart[q] <= u <
// ustart[q + 1], covers positions [k tgt[q], min((k + 1) tgt[q], totals[q]))
// for k = u - ustart[q], and starts at the member holding its first position.
__global__ void k_c4_units(const int64_t *ustart, int64_t nq, const int64_t *tgt,
                           const unsigned long long *totals, const int64_t *mprefix,
                           const int64_t *pbase, const uint32_t *heavy, const int64_t *rowptr,
                           C4Unit *units) {
    const int64_t nu = ustart[nq];
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nu;
         u += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nq - 1;  // last q with ustart[q] <= u
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (ustart[mid] <= u)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int64_t q = lo;
        const int64_t f_lo = (u - ustart[q]) * tgt[q];
        const int64_t f_hi = min(f_lo + tgt[q], (int64_t)totals[q]);
        const uint32_t a = heavy[q];
        const int da = (int)(rowptr[a + 1] - rowptr[a]);
        const int64_t *pre = mprefix + pbase[q];
        int m0 = 0, m1 = da - 1;  // last member m with pre[m] <= f_lo
        while (m0 < m1) {
            const int mid = (m0 + m1 + 1) >> 1;
            if (pre[mid] <= f_lo)
                m0 = mid;
            else
                m1 = mid - 1;
        }
        C4Unit un;
        un.lo = f_lo;
        un.hi = f_hi;
        un.q = (int32_t)q;
        un.m = m0;
        units[u] = un;
    }
}

// Positions [f_lo, f_hi) of anchor a's walk, from member m on (its first
// position `at`), by one warp: members are taken 32 at a time, their list
// lengths scanned across the lanes, and each position mapped to its member by
// a 5-step search over the lanes' running sums.  op(b, t_u) runs for every
// entry b ranked below a of a member u.  With stride > 32 the warp takes every
// (stride / 32)-th chunk of 32 members (no window: f_lo = 0, f_hi unbounded).
// One chunk of 32 members (lane values len, bu, tu) of c4_warp_walk, with
// running sums in IT (int when every list is short enough); returns the
// chunk's length.
template <class IT, class Op>
__device__ __forceinline__ int64_t c4_chunk(const C4Params &p, uint32_t a, int64_t len64,
                                            int64_t bu, int tu, int64_t at, int64_t f_lo,
                                            int64_t f_hi, Op &op) {
    const int lane = threadIdx.x & 31;
    const IT len = (IT)len64;
    IT incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const IT y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const IT total = __shfl_sync(kFull, incl, 31);
    const IT lo = (IT)(f_lo > at ? (f_lo - at < (int64_t)total ? f_lo - at : (int64_t)total) : 0);
    const IT hi = (IT)(f_hi - at < (int64_t)total ? f_hi - at : (int64_t)total);
    for (IT b0 = lo; b0 < hi; b0 += 32) {
        const IT pos = b0 + lane;
        int r = 0;  // the first member whose running sum exceeds pos
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const IT v = __shfl_sync(kFull, incl, r + st - 1);
            if (v <= pos) r += st;
        }
        const int64_t bur = __shfl_sync(kFull, bu, r);
        const IT str = __shfl_sync(kFull, incl - len, r);
        const int tur = __shfl_sync(kFull, tu, r);
        if (pos < hi) {
            const uint32_t b = __ldg(p.adj + bur + (int64_t)(pos - str)) & TG_IDMASK;
            if (b > a) op(b, tur);
        }
    }
    return (int64_t)total;
}

// Positions [f_lo, f_hi) of anchor a's walk, from member m on (its first
// position `at`), by one warp: members are taken 32 at a time, their list
// lengths scanned across the lanes, and each position mapped to its member by
// a 5-step search over the lanes' running sums.  op(b, t_u) runs for every
// entry b ranked below a of a member u.  With stride > 32 the warp takes every
// (stride / 32)-th chunk of 32 members (no window: f_lo = 0, f_hi unbounded).
template <class Op>
__device__ __forceinline__ void c4_warp_walk(const C4Params &p, uint32_t a, int64_t ba, int da,
                                             int m, int64_t at, int64_t f_lo, int64_t f_hi,
                                             int stride, Op op) {
    const int lane = threadIdx.x & 31;
    for (; m < da && at < f_hi; m += stride) {
        const int x = m + lane;
        int64_t len = 0, bu = 0;
        int tu = 0;
        if (x < da) {
            const uint32_t wu = __ldg(p.adj + ba + x);
            const uint32_t u = wu & TG_IDMASK;
            if (u > a) {
                bu = p.rowptr[u];
                const int64_t du = p.rowptr[u + 1] - bu;
                if (du > 1) {
                    len = du;
                    tu = (int)(wu >> TG_TSHIFT);
                }
            }
        }
        if (__all_sync(kFull, len < ((int64_t)1 << 26)))  // 32 lists sum below 2^31
            at += c4_chunk<int>(p, a, len, bu, tu, at, f_lo, f_hi, op);
        else
            at += c4_chunk<int64_t>(p, a, len, bu, tu, at, f_lo, f_hi, op);
    }
}

// One chunk of 32 members for k_c4_walk: as c4_chunk, with kWalkUnroll
// batches of 32 positions in flight per step (their list loads, then their
// counter adds, then the bitmap marks), so each lane keeps several returning
// adds outstanding.
constexpr int kWalkUnroll = 4;

template <class IT>
__device__ __forceinline__ int64_t c4_chunk_count(const C4Params &p, uint32_t a, int64_t len64,
                                                  int64_t bu, int tu, int64_t at, int64_t f_lo,
                                                  int64_t f_hi, uint32_t *cnt, uint32_t *bits,
                                                  unsigned long long &wk) {
    const int lane = threadIdx.x & 31;
    const int L = p.L;
    const IT len = (IT)len64;
    IT incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const IT y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const IT total = __shfl_sync(kFull, incl, 31);
    const IT lo = (IT)(f_lo > at ? (f_lo - at < (int64_t)total ? f_lo - at : (int64_t)total) : 0);
    const IT hi = (IT)(f_hi - at < (int64_t)total ? f_hi - at : (int64_t)total);
    const int Lp = L + (L & 1);
    for (IT b0 = lo; b0 < hi; b0 += 32 * kWalkUnroll) {
        uint32_t bv[kWalkUnroll];
        uint32_t *ca[kWalkUnroll];
        int sh[kWalkUnroll];
        bool ok[kWalkUnroll];
#pragma unroll
        for (int q = 0; q < kWalkUnroll; ++q) {
            const IT pos = b0 + 32 * q + lane;
            int r = 0;  // the first member whose running sum exceeds pos
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const IT v = __shfl_sync(kFull, incl, r + st - 1);
                if (v <= pos) r += st;
            }
            const int64_t bur = __shfl_sync(kFull, bu, r);
            const IT str = __shfl_sync(kFull, incl - len, r);
            const int tur = __shfl_sync(kFull, tu, r);
            ok[q] = false;
            bv[q] = 0;
            ca[q] = cnt;
            sh[q] = 0;
            if (pos < hi) {
                const uint32_t b = __ldg(p.adj + bur + (int64_t)(pos - str)) & TG_IDMASK;
                if (b > a) {
                    ok[q] = true;
                    bv[q] = b;
                    if (p.half) {
                        const int64_t k = (int64_t)b * Lp + tur;
                        ca[q] = cnt + (k >> 1);
                        sh[q] = (int)(k & 1) * 16;
                    } else {
                        ca[q] = cnt + (int64_t)b * L + tur;
                    }
                }
            }
        }
        uint32_t old[kWalkUnroll];
#pragma unroll
        for (int q = 0; q < kWalkUnroll; ++q) old[q] = ok[q] ? atomicAdd(ca[q], 1u << sh[q]) : 0xffffffffu;
#pragma unroll
        for (int q = 0; q < kWalkUnroll; ++q) {
            if (!ok[q]) continue;
            ++wk;
            // the first middle of a type at b marks b
            if (!((old[q] >> sh[q]) & (p.half ? 0xffffu : 0xffffffffu)))
                atomicOr(bits + (bv[q] >> 5), 1u << (bv[q] & 31u));
        }
    }
    return (int64_t)total;
}

// Pass 0 of a wave of costly anchors (global mode): one warp per unit, adding
// to the counters of its anchor's slot and marking a far end in the slot's
// bitmap when a count of it leaves zero; k_c4_pairs then takes the marked ends.
constexpr int kC4WalkWarps = 8;

__global__ void __launch_bounds__(kC4WalkWarps * 32) k_c4_walk(C4Params p) {
    const int lane = threadIdx.x & 31;
    unsigned long long wk = 0;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(p.queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= (unsigned long long)p.n_units) break;
        const C4Unit un = p.wunits[item];
        const uint32_t a = p.heavy[un.q];
        const int64_t ba = p.rowptr[a];
        const int da = (int)(p.rowptr[a + 1] - ba);
        uint32_t *cnt = p.scratch + (un.q - p.q0) * p.slot_words;
        uint32_t *bits = cnt + p.bits_off;
        int64_t at = p.mprefix[p.pbase[un.q] + un.m];
        for (int m = un.m; m < da && at < un.hi; m += 32) {
            const int x = m + lane;
            int64_t len = 0, bu = 0;
            int tu = 0;
            if (x < da) {
                const uint32_t wu = __ldg(p.adj + ba + x);
                const uint32_t u = wu & TG_IDMASK;
                if (u > a) {
                    bu = p.rowptr[u];
                    const int64_t du = p.rowptr[u + 1] - bu;
                    if (du > 1) {
                        len = du;
                        tu = (int)(wu >> TG_TSHIFT);
                    }
                }
            }
            if (__all_sync(kFull, len < ((int64_t)1 << 26)))
                at += c4_chunk_count<int>(p, a, len, bu, tu, at, un.lo, un.hi, cnt, bits, wk);
            else
                at += c4_chunk_count<int64_t>(p, a, len, bu, tu, at, un.lo, un.hi, cnt, bits, wk);
        }
    }
    if (p.work) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wk += __shfl_xor_sync(kFull, wk, o);
        if (lane == 0 && wk) atomicAdd(p.work + 4, wk);
    }
}

// One count into the histogram under the sorted multiset {a, b, c, d}.
__device__ __forceinline__ void k4_hist_add(unsigned long long *h4, int a, int b, int c, int d,
                                            unsigned long long v) {
    sort2(a, b);
    sort2(c, d);
    sort2(a, c);
    sort2(b, d);
    sort2(b, c);
    atomicAdd(h4 + colex4(a, b, c, d), v);
}

// ------------------------------------------------- binned waves (global) --
// Anchors whose walk is long against the number of far-end windows it spans
// (hubs): the counters stay on chip.  Every wedge a-u-b of a wave's walks
// becomes the 16-bit entry (b mod 2^wlg) | (type of u) << wlg in the bucket of
// (anchor, b >> wlg).  A count pass sizes the buckets and a fill pass writes
// them, each with one counter add per distinct bucket among a warp's 32
// wedges (a member's list is sorted by (type, id), so neighbouring wedges
// mostly share a window; a run of equal buckets among consecutive lanes takes
// its slots with one add).  k_c4_bin_pairs then gives each bucket to a CTA,
// which counts its entries by (b, t) in a dense shared-memory table of the
// window's 2^wlg far ends and adds each far end's cycle pairs to the
// type-multiset histogram (c4_add).  DRAM sees the walk twice and 2 bytes
// per wedge written and read once, instead of a counter read and write per
// wedge.
struct C4Bin {
    const int64_t *rowptr;
    const uint32_t *adj;
    const uint8_t *ntype;
    int32_t L, wlg, half;
    const uint32_t *heavy;     // the binned anchors
    const int64_t *mprefix;    // walk positions of their members (k_c4_prefix)
    const int64_t *pbase;
    const C4Unit *units;       // warp units of the wave
    int64_t n_units;
    int64_t q0;                // first anchor of the wave (bucket row = q - q0)
    int64_t n;                 // nodes
    int64_t W;                 // far-end windows, ceil(n / 2^wlg)
    uint32_t *cnt;             // K W bucket sizes (count pass), write cursors (fill pass)
    uint16_t *bins;            // the wave's entries, bucket after bucket
    const uint32_t *offs;      // K W + 1 bucket offsets
    int64_t nb;                // buckets of the wave, K W
    unsigned long long *queue;
    unsigned long long *g4;
    int64_t n4;
    unsigned long long *work;  // [4]: wedges
};

constexpr int kBinUnroll = 2;
constexpr int kBinFill = 32;            // default: binned when a walk averages this many wedges per window
constexpr size_t kBinTable = 64 * 1024;  // bytes of the dense far-end table

// One chunk of 32 members (lane values len, bu, tu) of a binned walk unit; as
// c4_chunk, with kBinUnroll batches of 32 positions per step.  Count pass:
// adds each batch's wedges to their buckets' sizes.  Fill pass: takes a run
// of slots from each bucket's cursor and writes the entries.
template <bool kFill, class IT>
__device__ __forceinline__ int64_t c4_chunk_bin(const C4Bin &p, uint32_t a, uint32_t *cb,
                                                int64_t len64, int64_t bu, int tu, int64_t at,
                                                int64_t f_lo, int64_t f_hi,
                                                unsigned long long &wk) {
    const int lane = threadIdx.x & 31;
    const IT len = (IT)len64;
    IT incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const IT y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const IT total = __shfl_sync(kFull, incl, 31);
    const IT lo = (IT)(f_lo > at ? (f_lo - at < (int64_t)total ? f_lo - at : (int64_t)total) : 0);
    const IT hi = (IT)(f_hi - at < (int64_t)total ? f_hi - at : (int64_t)total);
    const uint32_t wmask = (1u << p.wlg) - 1u;
    for (IT b0 = lo; b0 < hi; b0 += 32 * kBinUnroll) {
        uint32_t bv[kBinUnroll], base[kBinUnroll];
        int tv[kBinUnroll];
        bool ok[kBinUnroll];
#pragma unroll
        for (int q = 0; q < kBinUnroll; ++q) {
            const IT pos = b0 + 32 * q + lane;
            int r = 0;  // the first member whose running sum exceeds pos
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const IT v = __shfl_sync(kFull, incl, r + st - 1);
                if (v <= pos) r += st;
            }
            const int64_t bur = __shfl_sync(kFull, bu, r);
            const IT str = __shfl_sync(kFull, incl - len, r);
            const int tur = __shfl_sync(kFull, tu, r);
            ok[q] = false;
            bv[q] = 0;
            tv[q] = 0;
            if (pos < hi) {
                const uint32_t b = __ldg(p.adj + bur + (int64_t)(pos - str)) & TG_IDMASK;
                if (b > a) {
                    ok[q] = true;
                    bv[q] = b;
                    tv[q] = tur;
                }
            }
        }
        // runs of equal buckets among consecutive lanes (a member's list is
        // sorted by (type, id), so consecutive wedges mostly share a window):
        // the first lane of a run takes the run's slots with one add
        int rs[kBinUnroll];
#pragma unroll
        for (int q = 0; q < kBinUnroll; ++q) {
            const int key = ok[q] ? (int)(bv[q] >> p.wlg) : -1;
            const int prev = __shfl_up_sync(kFull, key, 1);
            const unsigned heads = __ballot_sync(kFull, lane == 0 || key != prev);
            const unsigned upto = heads & ((2u << lane) - 1u);  // heads at or below this lane
            rs[q] = 31 - __clz(upto);
            const unsigned above = heads & ~((2u << lane) - 1u);
            const int re = above ? __ffs(above) - 1 : 32;
            base[q] = 0u;
            if (key >= 0 && rs[q] == lane) {
                if (kFill)
                    base[q] = atomicAdd(cb + key, (uint32_t)(re - lane));
                else
                    atomicAdd(cb + key, (uint32_t)(re - lane));
            }
        }
#pragma unroll
        for (int q = 0; q < kBinUnroll; ++q) {
            if (kFill) {
                const uint32_t bb = __shfl_sync(kFull, base[q], rs[q]);
                if (ok[q])
                    p.bins[bb + (uint32_t)(lane - rs[q])] =
                        (uint16_t)((bv[q] & wmask) | ((uint32_t)tv[q] << p.wlg));
            } else if (ok[q]) {
                ++wk;
            }
        }
    }
    return (int64_t)total;
}

// The count (kFill = false) or fill pass of a binned wave: one warp per unit.
template <bool kFill>
__global__ void __launch_bounds__(kC4WalkWarps * 32) k_c4_bin_walk(C4Bin p) {
    const int lane = threadIdx.x & 31;
    unsigned long long wk = 0;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(p.queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= (unsigned long long)p.n_units) break;
        const C4Unit un = p.units[item];
        const uint32_t a = p.heavy[un.q];
        const int64_t ba = p.rowptr[a];
        const int da = (int)(p.rowptr[a + 1] - ba);
        uint32_t *cb = p.cnt + (un.q - p.q0) * p.W;
        int64_t at = p.mprefix[p.pbase[un.q] + un.m];
        for (int m = un.m; m < da && at < un.hi; m += 32) {
            const int x = m + lane;
            int64_t len = 0, bu = 0;
            int tu = 0;
            if (x < da) {
                const uint32_t wu = __ldg(p.adj + ba + x);
                const uint32_t u = wu & TG_IDMASK;
                if (u > a) {
                    bu = p.rowptr[u];
                    const int64_t du = p.rowptr[u + 1] - bu;
                    if (du > 1) {
                        len = du;
                        tu = (int)(wu >> TG_TSHIFT);
                    }
                }
            }
            if (__all_sync(kFull, len < ((int64_t)1 << 26)))
                at += c4_chunk_bin<kFill, int>(p, a, cb, len, bu, tu, at, un.lo, un.hi, wk);
            else
                at += c4_chunk_bin<kFill, int64_t>(p, a, cb, len, bu, tu, at, un.lo, un.hi, wk);
        }
    }
    if (!kFill && p.work) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wk += __shfl_xor_sync(kFull, wk, o);
        if (lane == 0 && wk) atomicAdd(p.work + 4, wk);
    }
}

// The buckets of a binned wave.  A CTA takes runs of kBinRun consecutive
// buckets (consecutive windows of one anchor, mostly) from a queue.  A bucket
// (anchor a of type ta, window w) has its entries counted by (b, t) in the
// dense table (16-bit halves when the wave's anchors have fewer than 2^16
// neighbours, else 32-bit counts); the first entry of a far end puts it on a
// list (a bit per far end keeps it there once).  Then one thread per listed
// far end reads its counts, clears them, and for the types it has (usually
// few) adds C(c_t, 2) and c_t c_t' to the CTA's table acc[type of b][pair]
// in shared memory (atomic adds), which goes into the histogram under
// {ta, tb, t, t'} when the anchor changes.  1024-thread CTAs, two per SM.  Types beyond kBinAccL use c4_add
// straight into a shared histogram instead.
constexpr int kBinPairThreads = 1024;
constexpr int kBinRun = 16;
constexpr int kBinAccL = 8;

__device__ __forceinline__ void bin_flush(unsigned long long *acc, unsigned long long *h4, int L,
                                          int P, int ta) {
    for (int k = threadIdx.x; k < L * P; k += blockDim.x) {
        const unsigned long long v = acc[k];
        if (!v) continue;
        acc[k] = 0ull;
        int t, u;
        unpair(L, k % P, t, u);
        k4_hist_add(h4, ta, k / P, t, u, v);
    }
}

__global__ void __launch_bounds__(kBinPairThreads) k_c4_bin_pairs(C4Bin p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    const int L = p.L, Lp = L + (L & 1), P = L * (L + 1) / 2;
    const bool acc_mode = L <= kBinAccL;
    const int nfar = 1 << p.wlg;
    unsigned long long *h4 = reinterpret_cast<unsigned long long *>(smem);
    size_t off = ((size_t)p.n4 * 8 + 15) & ~(size_t)15;
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(smem + off);  // one per CTA
    if (acc_mode) off += ((size_t)L * P * 8 + 15) & ~(size_t)15;
    uint32_t *tab = reinterpret_cast<uint32_t *>(smem + off);
    const int twords = p.half ? nfar * (Lp >> 1) : nfar * L;
    uint32_t *tbits = tab + twords;                                      // nfar / 32 words
    uint16_t *flist = reinterpret_cast<uint16_t *>(tbits + nfar / 32);  // touched far ends
    const volatile uint32_t *vtab = tab;
    __shared__ unsigned long long s_run;
    __shared__ uint32_t s_nl;
    for (int64_t q = tid; q < p.n4; q += blockDim.x) h4[q] = 0ull;
    if (acc_mode)
        for (int q = tid; q < L * P; q += blockDim.x) acc[q] = 0ull;
    for (int q = tid; q < twords + nfar / 32; q += blockDim.x) tab[q] = 0u;
    if (tid == 0) s_nl = 0u;
    const uint32_t wmask = (uint32_t)nfar - 1u;
    int cur_ta = -1;
    int64_t cur_row = -1;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_run = atomicAdd(p.queue, (unsigned long long)kBinRun);
        __syncthreads();
        const int64_t r0 = (int64_t)s_run;
        if (r0 >= p.nb) break;
        const int64_t r1 = r0 + kBinRun < p.nb ? r0 + kBinRun : p.nb;
        for (int64_t item = r0; item < r1; ++item) {
            const uint32_t c0 = p.offs[item], c1 = p.offs[item + 1];
            if (c0 == c1) continue;  // uniform across the CTA
            const int64_t row = item / p.W;
            const int64_t wbase = (item % p.W) << p.wlg;
            if (row != cur_row) {
                if (acc_mode && cur_ta >= 0) bin_flush(acc, h4, L, P, cur_ta);
                cur_row = row;
                cur_ta = p.ntype[p.heavy[p.q0 + row]];
            }
            const int ta = cur_ta;
            // count the entries by (far end, type); a far end's first entry
            // puts it on the list
            for (uint32_t k0 = c0 + tid; k0 < c1; k0 += 4 * blockDim.x) {
                uint32_t ev[4];
#pragma unroll
                for (int z = 0; z < 4; ++z) {
                    const uint32_t k = k0 + (uint32_t)z * blockDim.x;
                    ev[z] = k < c1 ? (uint32_t)p.bins[k] : 0xffffffffu;
                }
#pragma unroll
                for (int z = 0; z < 4; ++z) {
                    if (ev[z] == 0xffffffffu) continue;
                    const uint32_t bl = ev[z] & wmask;
                    const int t = (int)(ev[z] >> p.wlg);
                    bool first;
                    if (p.half) {
                        const uint32_t idx = bl * (uint32_t)Lp + (uint32_t)t;
                        const int sh = (int)(idx & 1u) * 16;
                        const uint32_t old = atomicAdd(tab + (idx >> 1), 1u << sh);
                        first = ((old >> sh) & 0xffffu) == 0u;
                    } else {
                        first = atomicAdd(tab + bl * (uint32_t)L + (uint32_t)t, 1u) == 0u;
                    }
                    if (first) {
                        const uint32_t bit = 1u << (bl & 31u);
                        if (!(atomicOr(tbits + (bl >> 5), bit) & bit)) flist[atomicAdd(&s_nl, 1u)] = (uint16_t)bl;
                    }
                }
            }
            __syncthreads();
            // one far end per thread: its nonzero types, the pairs among them
            const uint32_t nl = s_nl;
            for (uint32_t x = tid; x < nl; x += blockDim.x) {
                const uint32_t bl = flist[x];
                uint32_t c[TG_MAX_TYPES];
                uint32_t sum = 0, mask = 0;
                if (p.half) {
                    const uint32_t w0 = bl * (uint32_t)(Lp >> 1);
                    for (int q = 0; q < (Lp >> 1); ++q) {
                        const uint32_t w = vtab[w0 + q];
                        tab[w0 + q] = 0u;
                        c[2 * q] = w & 0xffffu;
                        if (2 * q + 1 < L) c[2 * q + 1] = w >> 16;
                        sum += (w & 0xffffu) + (w >> 16);
                        if (w & 0xffffu) mask |= 1u << (2 * q);
                        if (w >> 16) mask |= 1u << (2 * q + 1);
                    }
                } else {
                    for (int t = 0; t < L; ++t) {
                        c[t] = vtab[bl * (uint32_t)L + t];
                        tab[bl * (uint32_t)L + t] = 0u;
                        sum += c[t];
                        if (c[t]) mask |= 1u << t;
                    }
                }
                if (sum < 2) continue;
                const int tb = (int)p.ntype[wbase + bl];
                if (!acc_mode) {
                    c4_add(h4, L, ta, tb, c);
                    continue;
                }
                unsigned long long *ar = acc + (size_t)tb * P;
                for (uint32_t mt = mask; mt; mt &= mt - 1u) {
                    const int t = __ffs(mt) - 1;
                    const unsigned long long ct = c[t];
                    const int rowt = t * L - (t * (t - 1)) / 2;  // pair_index(L, t, u) = rowt + u - t
                    if (ct > 1) atomicAdd(ar + rowt, ct * (ct - 1) / 2);
                    for (uint32_t mu = mt & (mt - 1u); mu; mu &= mu - 1u) {
                        const int u = __ffs(mu) - 1;
                        atomicAdd(ar + rowt + (u - t), ct * c[u]);
                    }
                }
            }
            __syncthreads();
            for (int q = tid; q < nfar / 32; q += blockDim.x) tbits[q] = 0u;
            if (tid == 0) s_nl = 0u;
            __syncthreads();
        }
    }
    if (acc_mode && cur_ta >= 0) bin_flush(acc, h4, L, P, cur_ta);
    __syncthreads();
    for (int64_t q = tid; q < p.n4; q += blockDim.x)
        if (h4[q]) atomicAdd(p.g4 + q, h4[q]);
}

__global__ void k_gather_u64(const unsigned long long *x, const uint32_t *idx, int64_t n,
                             unsigned long long *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = x[idx[i]];
}

// ------------------------------------------------- light anchors (global) --
// Anchors whose walk cost (sum of d_u over their members) is at most half a
// warp's table: one warp per anchor, the far ends in a per-warp shared-memory
// hash set with L 16-bit middle counters per slot (a count never exceeds the
// cost).  No global counters, no CTA barrier between anchors.
constexpr int kC4WarpWarps = 8;
constexpr int kC4WarpLgMax = 9;  // 512 slots per warp

__device__ __forceinline__ uint32_t c4w_count(const uint32_t *cw, int k) {
    const volatile uint32_t *v = cw;
    return (v[k >> 1] >> ((k & 1) * 16)) & 0xffffu;
}

__global__ void __launch_bounds__(kC4WarpWarps * 32, 4) k_c4_warp(C4Params p, const uint32_t *alist,
                                                              int64_t na,
                                                              const unsigned long long *cost,
                                                              int lg_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int L = p.L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int emax = 1 << lg_max;
    const int cwords = (emax * L + 1) >> 1;
    unsigned long long *h4 = reinterpret_cast<unsigned long long *>(smem);
    uint32_t *keys = reinterpret_cast<uint32_t *>(h4 + p.n4) + (size_t)warp * (emax + cwords);
    uint32_t *cw = keys + emax;
    for (int64_t q = threadIdx.x; q < p.n4; q += blockDim.x) h4[q] = 0ull;
    for (int q = lane; q < emax + cwords; q += 32) keys[q] = 0u;
    __syncthreads();
    unsigned long long wk = 0;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(p.queue, 32ull);
        base = __shfl_sync(kFull, base, 0);
        if (base >= (unsigned long long)na) break;
        const int64_t stop = min((int64_t)base + 32, na);
        for (int64_t i = (int64_t)base; i < stop; ++i) {
            const uint32_t a = alist[i];
            const int64_t ba = p.rowptr[a];
            const int da = (int)(p.rowptr[a + 1] - ba);
            const int ta = p.ntype[a];
            const unsigned long long ca = cost[a];
            int lg = 5;
            while ((1ull << lg) < 2 * ca && lg < lg_max) ++lg;
            c4_warp_walk(p, a, ba, da, 0, 0, 0, INT64_MAX, 32, [&](uint32_t b, int tu) {
                const int h = hset_claim(keys, lg, b);
                if (h >= 0) {
                    const int k = h * L + tu;
                    atomicAdd(cw + (k >> 1), 1u << ((k & 1) * 16));
                    ++wk;
                }
            });
            __syncwarp();
            const int e = 1 << lg;
            const volatile uint32_t *vk = keys;
            for (int h = lane; h < e; h += 32) {
                const uint32_t k = vk[h];
                if (!k) continue;
                uint32_t c[TG_MAX_TYPES];
                for (int t = 0; t < L; ++t) c[t] = c4w_count(cw, h * L + t);
                c4_add(h4, L, ta, p.ntype[k - 1u], c);
            }
            __syncwarp();
            for (int q = lane; q < e; q += 32) keys[q] = 0u;
            for (int q = lane; q < ((e * L + 1) >> 1); q += 32) cw[q] = 0u;
            __syncwarp();
        }
    }
    __syncthreads();
    for (int64_t q = threadIdx.x; q < p.n4; q += blockDim.x)
        if (h4[q]) atomicAdd(p.g4 + q, h4[q]);
    if (p.work) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wk += __shfl_xor_sync(kFull, wk, o);
        if (lane == 0 && wk) atomicAdd(p.work + 4, wk);
    }
}

// Anchors of cost up to half a CTA table: one CTA per anchor, its warps taking
// every eighth chunk of 32 members, the far ends in one shared-memory hash set
// with 16-bit middle counters (the cost stays far below 2^16).
constexpr int kC4CtaThreads = 256;
constexpr int kC4CtaLgMax = 13;  // 8192 slots

__global__ void __launch_bounds__(kC4CtaThreads) k_c4_cta(C4Params p, const uint32_t *alist,
                                                          int64_t na,
                                                          const unsigned long long *cost,
                                                          int lg_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int L = p.L;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int stride = blockDim.x;  // 32 members per warp
    const int emax = 1 << lg_max;
    const int cwords = (emax * L + 1) >> 1;
    unsigned long long *h4 = reinterpret_cast<unsigned long long *>(smem);
    unsigned long long *s_item = h4 + p.n4;
    uint32_t *keys = reinterpret_cast<uint32_t *>(s_item + 1);
    uint32_t *cw = keys + emax;
    for (int64_t q = tid; q < p.n4; q += blockDim.x) h4[q] = 0ull;
    for (int q = tid; q < emax + cwords; q += blockDim.x) keys[q] = 0u;
    unsigned long long wk = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) *s_item = atomicAdd(p.queue, 1ull);
        __syncthreads();
        const unsigned long long item = *s_item;
        if (item >= (unsigned long long)na) break;
        const uint32_t a = alist[item];
        const int64_t ba = p.rowptr[a];
        const int da = (int)(p.rowptr[a + 1] - ba);
        const int ta = p.ntype[a];
        const unsigned long long ca = cost[a];
        int lg = 5;
        while ((1ull << lg) < 2 * ca && lg < lg_max) ++lg;
        c4_warp_walk(p, a, ba, da, 32 * warp, 0, 0, INT64_MAX, stride, [&](uint32_t b, int tu) {
            const int h = hset_claim(keys, lg, b);
            if (h >= 0) {
                const int k = h * L + tu;
                atomicAdd(cw + (k >> 1), 1u << ((k & 1) * 16));
                ++wk;
            }
        });
        __syncthreads();
        const int e = 1 << lg;
        const volatile uint32_t *vk = keys;
        for (int h = tid; h < e; h += blockDim.x) {
            const uint32_t k = vk[h];
            if (!k) continue;
            uint32_t c[TG_MAX_TYPES];
            for (int t = 0; t < L; ++t) c[t] = c4w_count(cw, h * L + t);
            c4_add(h4, L, ta, p.ntype[k - 1u], c);
        }
        __syncthreads();
        for (int q = tid; q < e; q += blockDim.x) keys[q] = 0u;
        for (int q = tid; q < ((e * L + 1) >> 1); q += blockDim.x) cw[q] = 0u;
    }
    __syncthreads();
    for (int64_t q = tid; q < p.n4; q += blockDim.x)
        if (h4[q]) atomicAdd(p.g4 + q, h4[q]);
    if (p.work) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wk += __shfl_xor_sync(kFull, wk, o);
        if (lane == 0 && wk) atomicAdd(p.work + 4, wk);
    }
}

// Walk cost of each anchor (sum of d_u over its neighbours u ranked below it)
// and the total.  One warp per node.
__global__ void k_c4_cost(const int64_t *rowptr, const uint32_t *adj, int64_t n,
                          unsigned long long *cost, unsigned long long *total) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long mine = 0;
    for (int64_t a = wid; a < n; a += nw) {
        const int64_t b = rowptr[a];
        const int d = (int)(rowptr[a + 1] - b);
        unsigned long long c = 0;
        for (int x = lane; x < d; x += 32) {
            const uint32_t u = __ldg(adj + b + x) & TG_IDMASK;
            if ((int64_t)u > a) c += (unsigned long long)(rowptr[u + 1] - rowptr[u]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
        if (lane == 0) cost[a] = d >= 2 ? c : 0ull;
        mine += c;
    }
    if (lane == 0 && mine) atomicAdd(total, mine);
}

// Anchor classes by walk cost c (flags[k n + a] = 1 for the class of a):
// kClsSplit c > thr, else kClsWarp 0 < c <= lite, kClsCta lite < c <= mid,
// kClsSlot mid < c (anchors of cost 0 close no cycle and take none).
enum { kClsSplit = 0, kClsWarp, kClsCta, kClsSlot, kClsN };

__global__ void k_c4_mark(const unsigned long long *cost, int64_t n, unsigned long long thr,
                          unsigned long long lite, unsigned long long mid, int pidx, int pcnt,
                          uint32_t *flags) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long c = a % pcnt == pidx ? cost[a] : 0ull;  // other parts' anchors
        int cls = -1;
        if (c > thr)
            cls = kClsSplit;
        else if (c > 0)
            cls = c <= lite ? kClsWarp : c <= mid ? kClsCta : kClsSlot;
#pragma unroll
        for (int k = 0; k < kClsN; ++k) flags[k * n + a] = cls == k ? 1u : 0u;
    }
}

__global__ void k_c4_compact(const uint32_t *flag, const uint32_t *pos, int64_t n,
                             uint32_t *list) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x)
        if (flag[a]) list[pos[a]] = (uint32_t)a;
}

// ------------------------------------------------------------ up lists ----
// Up list of v: its neighbours of higher rank (smaller new id), kept with
// their typed offsets and edge ids.  In a (type, id)-sorted list they are a
// prefix of every typed range.  One warp per node; lane t < L finds the end
// of the prefix of type t.
__global__ void k_up_count(const int64_t *rowptr, const uint32_t *adj, const int32_t *toff,
                           int64_t n, int32_t L, int32_t *utoff, int64_t *utot) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = wid; v < n; v += nw) {
        const int64_t b = rowptr[v];
        const int32_t *to = toff + v * (L + 1);
        int c = 0;
        if (lane < L) {
            int lo = __ldg(to + lane), hi = __ldg(to + lane + 1);
            const int start = lo;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((int64_t)(__ldg(adj + b + mid) & TG_IDMASK) < v)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            c = lo - start;
        }
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane < L) utoff[v * (L + 1) + lane + 1] = incl;
        if (lane == 0) utoff[v * (L + 1)] = 0;
        if (lane == L - 1) utot[v] = incl;
    }
}

__global__ void k_up_fill(const int64_t *rowptr, const uint32_t *adj, const uint32_t *eid,
                          const int32_t *toff, const int32_t *utoff, const int64_t *uoff,
                          int64_t n, int32_t L, uint32_t *uadj, uint32_t *ueid) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = wid; v < n; v += nw) {
        const int64_t b = rowptr[v], ub = uoff[v];
        const int32_t *to = toff + v * (L + 1);
        const int32_t *uto = utoff + v * (L + 1);
        for (int t = 0; t < L; ++t) {
            const int src = __ldg(to + t), dst = __ldg(uto + t);
            const int c = __ldg(uto + t + 1) - dst;
            for (int x = lane; x < c; x += 32) {
                uadj[ub + dst + x] = __ldg(adj + b + src + x);
                ueid[ub + dst + x] = __ldg(eid + b + src + x);
            }
        }
    }
}

// ----------------------------------------------------------- 4-cliques ----
struct K4Params {
    const int64_t *uoff;       // up lists (see k_up_count)
    const uint32_t *uadj;
    const uint32_t *ueid;
    const int32_t *utoff;
    const uint8_t *ntype;
    int64_t n;
    int32_t L, P;
    int32_t cap;               // W entries per warp in shared memory
    unsigned long long *queue;
    unsigned long long *k4e;   // per-edge mode: M * P, 4-cliques by the types of the two
                               // other nodes
    unsigned long long *g4;    // global mode: C(L+3,4) 4-clique counts by type multiset
    int64_t n4;
    unsigned long long *work;  // [5]: candidate tests, [6]: 4-cliques
};

constexpr int kK4Warps = 8;

__device__ __forceinline__ void k4_add(unsigned long long *k4e, int64_t e, int P, int L, int a,
                                       int b, unsigned long long v) {
    atomicAdd(k4e + e * P + pair_index(L, a, b), v);
}

__global__ void __launch_bounds__(kK4Warps * 32) k_k4(K4Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = p.L, P = p.P, cap = p.cap;
    uint32_t *w_ent = reinterpret_cast<uint32_t *>(smem) + (size_t)warp * cap * (3 + L);
    int32_t *w_p0 = reinterpret_cast<int32_t *>(w_ent + cap);  // position in x0's list
    int32_t *w_pv = w_p0 + cap;                                  // position in v's list
    uint32_t *xacc = reinterpret_cast<uint32_t *>(w_pv + cap);  // cap * L
    unsigned long long *h4 = reinterpret_cast<unsigned long long *>(
        smem + (size_t)kK4Warps * cap * (3 + L) * 4);  // global mode: n4 entries
    const bool global = p.g4 != nullptr;
    if (global) {
        for (int64_t q = threadIdx.x; q < p.n4; q += blockDim.x) h4[q] = 0ull;
        __syncthreads();
    }
    const uint32_t below = (1u << lane) - 1u;
    unsigned long long wk_cand = 0, wk_k4 = 0;

    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(p.queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= (unsigned long long)p.n) break;
        const uint32_t x0 = (uint32_t)item;
        const int64_t b0 = p.uoff[x0];
        const int d0 = (int)(p.uoff[x0 + 1] - b0);
        if (d0 < 3) continue;  // x0 is the lowest node: three more above it
        const int t0 = p.ntype[x0];
        const int32_t *to0 = p.utoff + (int64_t)x0 * (L + 1);
        for (int c0 = 0; c0 < d0; c0 += 32) {
            const int xx = c0 + lane;
            uint32_t ev = 0;
            bool isup = false;
            if (xx < d0) {
                ev = __ldg(p.uadj + b0 + xx);
                isup = true;
            }
            unsigned upm = __ballot_sync(kFull, isup);
            while (upm) {
                const int src = __ffs(upm) - 1;
                upm &= upm - 1;
                const uint32_t vent = __shfl_sync(kFull, ev, src);
                const uint32_t v = vent & TG_IDMASK;
                const int tv = (int)(vent >> TG_TSHIFT);
                const int64_t bv = p.uoff[v];
                const int dv = (int)(p.uoff[v + 1] - bv);
                const int32_t *tov = p.utoff + (int64_t)v * (L + 1);
                const int64_t e0v = __ldg(p.ueid + b0 + c0 + src);
                // W = up(v) n up(x0) (= up(v) n Gamma(x0)), in the order of up(v)
                int nw = 0;
                for (int c1 = 0; c1 < dv; c1 += 32) {
                    const int q = c1 + lane;
                    bool ok = false;
                    uint32_t wq = 0;
                    int pos0 = -1;
                    if (q < dv) {
                        wq = __ldg(p.uadj + bv + q);
                        pos0 = find_pos(p.uadj, b0, to0, wq);
                        ok = pos0 >= 0;
                    }
                    const unsigned m = __ballot_sync(kFull, ok);
                    const int r = nw + __popc(m & below);
                    if (ok && r < cap) {
                        w_ent[r] = wq;
                        w_p0[r] = pos0;
                        w_pv[r] = q;
                    }
                    nw += __popc(m);
                }
                if (nw < 2) {
                    __syncwarp();
                    continue;
                }
                const bool staged = nw <= cap;
                if (staged && !global)
                    for (int q = lane; q < nw * L; q += 32) xacc[q] = 0u;
                __syncwarp();
                // every w of W (staged: from shared memory; else re-derived)
                for (int c1 = 0, k = 0; staged ? k < nw : c1 < dv;) {
                    unsigned wm;
                    uint32_t wlane = 0;
                    int p0lane = -1;
                    if (staged) {
                        wm = 1u;
                    } else {
                        const int q = c1 + lane;
                        bool ok = false;
                        if (q < dv) {
                            wlane = __ldg(p.uadj + bv + q);
                            p0lane = find_pos(p.uadj, b0, to0, wlane);
                            ok = p0lane >= 0;
                        }
                        wm = __ballot_sync(kFull, ok);
                    }
                    while (wm) {
                        const int sl = __ffs(wm) - 1;
                        wm &= wm - 1;
                        uint32_t went;
                        int wp0, wpv;
                        if (staged) {
                            went = w_ent[k];
                            wp0 = w_p0[k];
                            wpv = w_pv[k];
                        } else {
                            went = __shfl_sync(kFull, wlane, sl);
                            wp0 = __shfl_sync(kFull, p0lane, sl);
                            wpv = c1 + sl;
                        }
                        const uint32_t w = went & TG_IDMASK;
                        const int tw = (int)(went >> TG_TSHIFT);
                        const int64_t bw = p.uoff[w];
                        const int dw = (int)(p.uoff[w + 1] - bw);
                        const int64_t e0w = __ldg(p.ueid + b0 + wp0);
                        const int64_t evw = __ldg(p.ueid + bv + wpv);
                        for (int c2 = 0; c2 < dw; c2 += 32) {
                            const int r = c2 + lane;
                            int key = -1;
                            if (r < dw) {
                                const uint32_t xe = __ldg(p.uadj + bw + r);
                                {
                                    ++wk_cand;
                                    int64_t e0x = -1, evx = -1;
                                    if (staged) {
                                        int lo = 0, hi = nw;
                                        while (lo < hi) {
                                            const int mid = (lo + hi) >> 1;
                                            if (w_ent[mid] < xe)
                                                lo = mid + 1;
                                            else
                                                hi = mid;
                                        }
                                        if (lo < nw && w_ent[lo] == xe) {
                                            // (x0,x) and (v,x) are summed per x below
                                            if (!global) atomicAdd(xacc + lo * L + tw, 1u);
                                            e0x = 0;
                                        }
                                    } else {
                                        const int px0 = find_pos(p.uadj, b0, to0, xe);
                                        if (px0 >= 0) {
                                            const int pxv = find_pos(p.uadj, bv, tov, xe);
                                            if (pxv >= 0) {
                                                e0x = 0;
                                                if (!global) {
                                                    evx = __ldg(p.ueid + bv + pxv);
                                                    k4_add(p.k4e, __ldg(p.ueid + b0 + px0), P, L,
                                                           tv, tw, 1ull);
                                                    k4_add(p.k4e, evx, P, L, t0, tw, 1ull);
                                                }
                                            }
                                        }
                                    }
                                    if (e0x >= 0) {
                                        key = (int)(xe >> TG_TSHIFT);
                                        if (!global)
                                            k4_add(p.k4e, __ldg(p.ueid + bw + r), P, L, t0, tv,
                                                   1ull);
                                        ++wk_k4;
                                    }
                                }
                            }
                            // edges (x0,v), (x0,w), (v,w), summed over x of one type
                            const unsigned mm = __match_any_sync(kFull, key);
                            if (key >= 0 && lane == __ffs(mm) - 1) {
                                const unsigned long long c = (unsigned long long)__popc(mm);
                                if (global) {
                                    int q0 = t0, q1 = tv, q2 = tw, q3 = key;
                                    sort2(q0, q1);
                                    sort2(q2, q3);
                                    sort2(q0, q2);
                                    sort2(q1, q3);
                                    sort2(q1, q2);
                                    atomicAdd(h4 + colex4(q0, q1, q2, q3), c);
                                } else {
                                    k4_add(p.k4e, e0v, P, L, tw, key, c);
                                    k4_add(p.k4e, e0w, P, L, tv, key, c);
                                    k4_add(p.k4e, evw, P, L, t0, key, c);
                                }
                            }
                        }
                        if (staged) ++k;
                    }
                    if (!staged) c1 += 32;
                }
                if (staged && !global) {
                    __syncwarp();
                    for (int q = lane; q < nw * L; q += 32) {
                        const uint32_t c = xacc[q];
                        if (c) {
                            const int kx = q / L, tw = q % L;
                            k4_add(p.k4e, __ldg(p.ueid + b0 + w_p0[kx]), P, L, tv, tw, c);
                            k4_add(p.k4e, __ldg(p.ueid + bv + w_pv[kx]), P, L, t0, tw, c);
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
    if (global) {
        __syncthreads();
        for (int64_t q = threadIdx.x; q < p.n4; q += blockDim.x)
            if (h4[q]) atomicAdd(p.g4 + q, h4[q]);
    }
    if (p.work) {
        if (wk_cand) atomicAdd(p.work + 5, wk_cand);
        if (wk_k4) atomicAdd(p.work + 6, wk_k4);
    }
}

// 4-cliques by type multiset only (global mode).  As k_k4, each clique is met
// from its lowest node x0 and the next one v; here a warp's work item is a
// run of kK4GChunk oriented edges (x0, v) of the up lists, so the edges of a
// costly x0 spread over many warps.  Membership in up(x0) and in
// W = up(v) n up(x0) is a probe of a per-warp hash set when the set fits (cap
// entries), else a search of the sorted up lists.
struct K4GParams {
    const int64_t *uoff;
    const uint32_t *uadj;
    const int32_t *utoff;
    const uint8_t *ntype;
    int64_t n;
    int64_t m;  // entries of the up lists (edges)
    int32_t L;
    int32_t cap;  // set entries per warp (tables of 2^hlg >= 2 cap slots)
    int32_t hlg;
    int32_t min_d0;  // k_k4_global: only x0 with up lists longer than this
    unsigned long long *queue;
    unsigned long long *g4;
    int64_t n4;
    unsigned long long *work;
    uint32_t *rows;       // k_k4_rows: per CTA rows_stride words of bitmap rows
    int64_t rows_stride;
    int32_t pidx, pcnt;   // only lowest nodes x0 with x0 mod pcnt == pidx
};

constexpr int kK4GWarps = 8;
constexpr int kK4GChunk = 8;  // oriented edges (x0, v) per work item

__global__ void __launch_bounds__(kK4GWarps * 32) k_k4_global(K4GParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = p.L, cap = p.cap, tsz = 1 << p.hlg;
    unsigned long long *h4 = reinterpret_cast<unsigned long long *>(smem);
    const size_t h4b = ((size_t)p.n4 * 8 + 15) & ~(size_t)15;
    uint32_t *went = reinterpret_cast<uint32_t *>(smem + h4b) + (size_t)warp * (cap + 2 * tsz);
    uint32_t *hx = went + cap;
    uint32_t *hw = hx + tsz;
    for (int64_t q = threadIdx.x; q < p.n4; q += blockDim.x) h4[q] = 0ull;
    __syncthreads();
    const uint32_t below = (1u << lane) - 1u;
    unsigned long long wk_cand = 0, wk_k4 = 0;
    const int64_t nchunks = (p.m + kK4GChunk - 1) / kK4GChunk;
    int64_t cur = -1;  // x0 whose up list the hash set hx holds
    int lgx = 5;
    bool xh = false;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(p.queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= (unsigned long long)nchunks) break;
        // the chunk's oriented edges (x0, v): positions q of the up lists
        const int64_t q0 = (int64_t)item * kK4GChunk;
        const int64_t q1 = min(p.m, q0 + kK4GChunk);
        int64_t x0 = 0;
        {
            int64_t lo = 0, hi = p.n - 1;  // last x0 with uoff[x0] <= q0
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (__ldg(p.uoff + mid) <= q0)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            x0 = lo;
        }
        for (int64_t qq = q0; qq < q1; ++qq) {
        while (__ldg(p.uoff + x0 + 1) <= qq) ++x0;
        const int64_t b0 = __ldg(p.uoff + x0);
        const int d0 = (int)(__ldg(p.uoff + x0 + 1) - b0);
        if (d0 < 3 || d0 <= p.min_d0 || x0 % p.pcnt != p.pidx) continue;  // three more above
                                                  // x0; or a bitmap kernel's; or another part's
        const int t0 = p.ntype[x0];
        const int32_t *to0 = p.utoff + x0 * (L + 1);
        if (x0 != cur) {
            cur = x0;
            xh = d0 <= cap;
            lgx = 5;
            while ((1 << lgx) < 2 * d0 && lgx < p.hlg) ++lgx;
            __syncwarp();
            if (xh) {
                for (int q = lane; q < (1 << lgx); q += 32) hx[q] = 0u;
                __syncwarp();
                for (int q = lane; q < d0; q += 32) hset_put(hx, lgx, __ldg(p.uadj + b0 + q) & TG_IDMASK);
                __syncwarp();
            }
        }
        {
            {
                const uint32_t vent = __ldg(p.uadj + qq);
                const uint32_t v = vent & TG_IDMASK;
                const int tv = (int)(vent >> TG_TSHIFT);
                const int64_t bv = p.uoff[v];
                const int dv = (int)(p.uoff[v + 1] - bv);
                const int32_t *tov = p.utoff + (int64_t)v * (L + 1);
                // W = up(v) n up(x0)
                int nw = 0;
                for (int c1 = 0; c1 < dv; c1 += 32) {
                    const int q = c1 + lane;
                    bool ok = false;
                    uint32_t wq = 0;
                    if (q < dv) {
                        wq = __ldg(p.uadj + bv + q);
                        ok = xh ? hset_has(hx, lgx, wq & TG_IDMASK) : find_pos(p.uadj, b0, to0, wq) >= 0;
                    }
                    const unsigned m = __ballot_sync(kFull, ok);
                    const int r = nw + __popc(m & below);
                    if (ok && r < cap) went[r] = wq;
                    nw += __popc(m);
                }
                if (nw < 2) {
                    __syncwarp();
                    continue;
                }
                const bool staged = nw <= cap;
                int lgw = 5;
                while ((1 << lgw) < 2 * nw && lgw < p.hlg) ++lgw;
                if (staged) {
                    for (int q = lane; q < (1 << lgw); q += 32) hw[q] = 0u;
                    __syncwarp();
                    for (int q = lane; q < nw; q += 32) hset_put(hw, lgw, went[q] & TG_IDMASK);
                }
                __syncwarp();
                for (int c1 = 0, k = 0; staged ? k < nw : c1 < dv;) {
                    unsigned wm;
                    uint32_t wlane = 0;
                    if (staged) {
                        wm = 1u;
                    } else {
                        const int q = c1 + lane;
                        bool ok = false;
                        if (q < dv) {
                            wlane = __ldg(p.uadj + bv + q);
                            ok = xh ? hset_has(hx, lgx, wlane & TG_IDMASK)
                                    : find_pos(p.uadj, b0, to0, wlane) >= 0;
                        }
                        wm = __ballot_sync(kFull, ok);
                    }
                    while (wm) {
                        const int sl = __ffs(wm) - 1;
                        wm &= wm - 1;
                        const uint32_t went_k = staged ? went[k] : __shfl_sync(kFull, wlane, sl);
                        const uint32_t w = went_k & TG_IDMASK;
                        const int tw = (int)(went_k >> TG_TSHIFT);
                        const int64_t bw = p.uoff[w];
                        const int dw = (int)(p.uoff[w + 1] - bw);
                        int s0 = t0, s1 = tv, s2 = tw;
                        sort2(s0, s1);
                        sort2(s1, s2);
                        sort2(s0, s1);
                        for (int c2 = 0; c2 < dw; c2 += 32) {
                            const int r = c2 + lane;
                            int key = -1;
                            if (r < dw) {
                                const uint32_t xe = __ldg(p.uadj + bw + r);
                                ++wk_cand;
                                bool in;
                                if (staged) {
                                    in = hset_has(hw, lgw, xe & TG_IDMASK);
                                } else {
                                    in = (xh ? hset_has(hx, lgx, xe & TG_IDMASK)
                                             : find_pos(p.uadj, b0, to0, xe) >= 0) &&
                                         find_pos(p.uadj, bv, tov, xe) >= 0;
                                }
                                if (in) {
                                    key = (int)(xe >> TG_TSHIFT);
                                    ++wk_k4;
                                }
                            }
                            const unsigned mm = __match_any_sync(kFull, key);
                            if (key >= 0 && lane == __ffs(mm) - 1) {
                                int q0 = s0, q1 = s1, q2 = s2, q3 = key;
                                sort2(q2, q3);
                                sort2(q1, q2);
                                sort2(q0, q1);
                                atomicAdd(h4 + colex4(q0, q1, q2, q3), (unsigned long long)__popc(mm));
                            }
                        }
                        if (staged) ++k;
                    }
                    if (!staged) c1 += 32;
                }
                __syncwarp();
            }
        }
        }
    }
    __syncthreads();
    for (int64_t q = threadIdx.x; q < p.n4; q += blockDim.x)
        if (h4[q]) atomicAdd(p.g4 + q, h4[q]);
    if (p.work) {
        if (wk_cand) atomicAdd(p.work + 5, wk_cand);
        if (wk_k4) atomicAdd(p.work + 6, wk_k4);
    }
}

// 4-cliques by type multiset (global mode) from bitmaps.  The cliques whose
// lowest node is x0 are the triangles of the graph on up(x0): with bm_v the
// set of positions (in x0's up list) of up(v) n up(x0), every clique
// x0 < v < w < x is met once, at the pair (v, w in bm_v), as a bit of
// bm_v & bm_w; up(x0) is sorted by (type, id), so the bits of one type form a
// contiguous range and popc(bm_v & bm_w & mask_t) counts the cliques whose
// fourth node has type t.
constexpr int kBitsWarpMax = 32;    // up lists of at most 32: one word, one warp
constexpr int kBitsWarps = 8;

__device__ __forceinline__ uint32_t range_mask(int lo, int hi) {  // bits [lo, hi) of a word
    lo = max(0, min(32, lo));
    hi = max(0, min(32, hi));
    if (hi <= lo) return 0u;
    const uint32_t h = hi == 32 ? 0xffffffffu : ((1u << hi) - 1u);
    const uint32_t l = lo == 32 ? 0xffffffffu : ((1u << lo) - 1u);
    return h & ~l;
}


__global__ void __launch_bounds__(kBitsWarps * 32) k_k4_bits_warp(K4GParams p) {
    __shared__ uint32_t hk[kBitsWarps][2 * kBitsWarpMax], hv[kBitsWarps][2 * kBitsWarpMax];
    __shared__ uint32_t tmask[kBitsWarps][TG_MAX_TYPES];
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *h4 = reinterpret_cast<unsigned long long *>(smem);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = p.L;
    for (int64_t q = threadIdx.x; q < p.n4; q += blockDim.x) h4[q] = 0ull;
    __syncthreads();
    unsigned long long wk = 0, wpairs = 0;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(p.queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= (unsigned long long)p.n) break;
        const uint32_t x0 = (uint32_t)item;
        const int64_t b0 = __ldg(p.uoff + x0);
        const int d0 = (int)(__ldg(p.uoff + x0 + 1) - b0);
        if (d0 < 3 || d0 > kBitsWarpMax || (int64_t)x0 % p.pcnt != p.pidx) continue;
        const int t0 = p.ntype[x0];
        const int32_t *to0 = p.utoff + (int64_t)x0 * (L + 1);
        // position of every up(x0) member, and the type ranges as masks
        hk[warp][lane] = 0u;
        hk[warp][lane + 32] = 0u;
        if (lane < L) tmask[warp][lane] = range_mask(__ldg(to0 + lane), __ldg(to0 + lane + 1));
        __syncwarp();
        const uint32_t ve = lane < d0 ? __ldg(p.uadj + b0 + lane) : 0u;
        if (lane < d0) hmap_put(hk[warp], hv[warp], 6, ve & TG_IDMASK, (uint32_t)lane);
        __syncwarp();
        // bm of the member at position pv, one member at a time
        uint32_t mine = 0;
        for (int pv = 0; pv < d0; ++pv) {
            const uint32_t v = __shfl_sync(kFull, ve, pv) & TG_IDMASK;
            const int64_t bv = __ldg(p.uoff + v);
            const int dv = (int)(__ldg(p.uoff + v + 1) - bv);
            uint32_t acc = 0;
            for (int c = lane; c < dv; c += 32) {
                const uint32_t y = __ldg(p.uadj + bv + c) & TG_IDMASK;
                const uint32_t pos = hmap_get(hk[warp], hv[warp], 6, y);
                if (pos != 0xffffffffu) acc |= 1u << pos;
            }
            acc = __reduce_or_sync(kFull, acc);
            if (lane == pv) mine = acc;
        }
        // pairs (v, w in bm_v): lane pv takes the members w of its bitmap in turn
        const int tv = (int)(ve >> TG_TSHIFT);
        uint32_t m = lane < d0 ? mine : 0u;
        while (__any_sync(kFull, m != 0u)) {
            const int q = m ? __ffs(m) - 1 : 0;
            const uint32_t bw = __shfl_sync(kFull, mine, q);
            const int tw = (int)(__shfl_sync(kFull, ve, q) >> TG_TSHIFT);
            if (m) {
                const uint32_t both = mine & bw;
                for (int t = 0; t < L; ++t) {
                    const int c = __popc(both & tmask[warp][t]);
                    if (c) k4_hist_add(h4, t0, tv, tw, t, (unsigned long long)c);
                }
                wk += __popc(both);
                ++wpairs;
                m &= m - 1;
            }
        }
        __syncwarp();
    }
    __syncthreads();
    for (int64_t q = threadIdx.x; q < p.n4; q += blockDim.x)
        if (h4[q]) atomicAdd(p.g4 + q, h4[q]);
    if (p.work && wk) atomicAdd(p.work + 6, wk);
    if (p.work && wpairs) atomicAdd(p.work + 5, wpairs);
}

// Up lists longer than one word: one CTA per x0 (from `list`).  Positions in
// up(x0) are laid out type by type, each type's range padded to whole 32-bit
// words, so that every word of a bitmap covers one type.  Row q (member q of
// up(x0), node v) is the bitmap of up(v) n up(x0) over these positions; one
// warp builds it from v's up list through a shared-memory map from node id to
// position and stores it in the CTA's slice of global memory (the rows are
// read back from L2).  Every clique x0 < v < w < x is one bit of
// row_v & row_w for a w in row_v: a warp takes v, keeps row_v in registers
// (WPL words per lane), visits the set bits w of row_v in position order and
// adds popc(row_v & row_w) per word to per-lane counters, flushed into the
// type-multiset histogram whenever the type of w changes (the type of x is
// the word's type).  One pair costs one coalesced row load per warp.
constexpr int kRowsThreads = 512;
constexpr int kRowsMaxWords = 128;

template <int WPL>
__device__ __forceinline__ uint32_t rows_pick(const uint32_t (&r)[WPL], int i) {
    uint32_t x = r[0];
#pragma unroll
    for (int k = 1; k < WPL; ++k)
        if (i == k) x = r[k];
    return x;
}

// The per-lane counts of the words a lane holds (w of type tw so far) into
// the histogram under {t0, tv, tw, type of the word}; clears them.
template <int WPL>
__device__ __forceinline__ void rows_flush(unsigned long long *h4, uint32_t (&acc)[WPL],
                                           const int32_t *wt, int words, int lane, int t0, int tv,
                                           int tw, unsigned long long &wk) {
    if (tw < 0) return;
#pragma unroll
    for (int i = 0; i < WPL; ++i) {
        const int kk = lane + 32 * i;
        if (kk < words && acc[i]) {
            k4_hist_add(h4, t0, tv, tw, wt[kk], (unsigned long long)acc[i]);
            wk += acc[i];
        }
        acc[i] = 0u;
    }
}

template <int WPL>
__global__ void __launch_bounds__(kRowsThreads) k_k4_rows(K4GParams p, const uint32_t *list,
                                                          uint32_t nlist) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int L = p.L;
    unsigned long long *h4 = reinterpret_cast<unsigned long long *>(smem);
    const size_t h4b = ((size_t)p.n4 * 8 + 15) & ~(size_t)15;
    uint32_t *hk = reinterpret_cast<uint32_t *>(smem + h4b);  // 2^p.hlg slots
    uint32_t *hv = hk + (1 << p.hlg);
    int32_t *wt = reinterpret_cast<int32_t *>(hv + (1 << p.hlg));  // type of each word
    int32_t *ws = wt + kRowsMaxWords;        // first word of each type, L + 1
    int32_t *to = ws + TG_MAX_TYPES + 1;     // type offsets of up(x0), L + 1
    uint32_t *rb = reinterpret_cast<uint32_t *>(to + TG_MAX_TYPES + 1) + warp * kRowsMaxWords;
    const volatile uint32_t *vrb = rb;
    __shared__ unsigned long long s_item;
    uint32_t *rows = p.rows + (size_t)blockIdx.x * (size_t)p.rows_stride;
    for (int64_t q = tid; q < p.n4; q += blockDim.x) h4[q] = 0ull;
    unsigned long long wk = 0, wpairs = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(p.queue, 1ull);
        __syncthreads();
        const unsigned long long item = s_item;
        if (item >= nlist) break;
        const uint32_t x0 = list[item];
        const int64_t b0 = __ldg(p.uoff + x0);
        const int d0 = (int)(__ldg(p.uoff + x0 + 1) - b0);
        const int t0 = p.ntype[x0];
        const int32_t *to0 = p.utoff + (int64_t)x0 * (L + 1);
        int lg = 5;
        while ((1 << lg) < 2 * d0 && lg < p.hlg) ++lg;
        if (tid <= L) to[tid] = __ldg(to0 + tid);
        if (tid == 0) {
            int w = 0;
            for (int t = 0; t < L; ++t) {
                ws[t] = w;
                w += (__ldg(to0 + t + 1) - __ldg(to0 + t) + 31) >> 5;
            }
            ws[L] = w;
        }
        for (int q = tid; q < (1 << lg); q += blockDim.x) hk[q] = 0u;
        __syncthreads();
        const int words = ws[L];
        for (int k = tid; k < words; k += blockDim.x) {
            int t = 0;
            while (t + 1 < L && ws[t + 1] <= k) ++t;
            wt[k] = t;
        }
        for (int q = tid; q < d0; q += blockDim.x) {
            const uint32_t e = __ldg(p.uadj + b0 + q);
            const int t = (int)(e >> TG_TSHIFT);
            hmap_put(hk, hv, lg, e & TG_IDMASK, (uint32_t)(32 * ws[t] + (q - to[t])));
        }
        __syncthreads();
        // rows: warp per member v
        for (int q = warp; q < d0; q += W) {
            for (int k = lane; k < words; k += 32) rb[k] = 0u;
            __syncwarp();
            const uint32_t v = __ldg(p.uadj + b0 + q) & TG_IDMASK;
            const int64_t bv = __ldg(p.uoff + v);
            const int dv = (int)(__ldg(p.uoff + v + 1) - bv);
            for (int c = lane; c < dv; c += 32) {
                const uint32_t pp = hmap_get(hk, hv, lg, __ldg(p.uadj + bv + c) & TG_IDMASK);
                if (pp != 0xffffffffu) atomicOr(rb + (pp >> 5), 1u << (pp & 31u));
            }
            __syncwarp();
            for (int k = lane; k < words; k += 32) rows[(size_t)q * words + k] = vrb[k];
            __syncwarp();
        }
        __syncthreads();
        // pairs (v, w in row_v): warp per v
        for (int q = warp; q < d0; q += W) {
            const int tv = (int)(__ldg(p.uadj + b0 + q) >> TG_TSHIFT);
            const uint32_t *rowv = rows + (size_t)q * words;
            uint32_t rv[WPL], acc[WPL];
#pragma unroll
            for (int i = 0; i < WPL; ++i) {
                const int kk = lane + 32 * i;
                rv[i] = kk < words ? __ldcg(rowv + kk) : 0u;
                acc[i] = 0u;
            }
            int cur = -1;
            for (int k = 0; k < words; ++k) {
                uint32_t x = __shfl_sync(kFull, rows_pick<WPL>(rv, k >> 5), k & 31);
                if (!x) continue;
                const int tw = wt[k];
                if (tw != cur) {
                    rows_flush<WPL>(h4, acc, wt, words, lane, t0, tv, cur, wk);
                    cur = tw;
                }
                const int qb = to[tw] + 32 * (k - ws[tw]);  // member index of the word's bit 0
                while (x) {
                    const int b = __ffs(x) - 1;
                    x &= x - 1u;
                    const uint32_t *roww = rows + (size_t)(qb + b) * words;
#pragma unroll
                    for (int i = 0; i < WPL; ++i) {
                        const int kk = lane + 32 * i;
                        if (kk < words) acc[i] += (uint32_t)__popc(rv[i] & __ldcg(roww + kk));
                    }
                    ++wpairs;
                }
            }
            rows_flush<WPL>(h4, acc, wt, words, lane, t0, tv, cur, wk);
        }
    }
    __syncthreads();
    for (int64_t q = tid; q < p.n4; q += blockDim.x)
        if (h4[q]) atomicAdd(p.g4 + q, h4[q]);
    if (p.work) {
        // wpairs is the same in every lane of a warp: count it once
        if (lane == 0 && wpairs) atomicAdd(p.work + 5, wpairs);
        if (wk) atomicAdd(p.work + 6, wk);
    }
}

__global__ void k_flag_range(const int64_t *uoff, int64_t n, int lo, int hi, int pidx, int pcnt,
                             uint32_t *flag) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = uoff[v + 1] - uoff[v];
        flag[v] = (d >= lo && d <= hi && v % pcnt == pidx) ? 1u : 0u;
    }
}

__global__ void k_max_i64(const int64_t *x, int64_t n, unsigned long long *mx) {
    unsigned long long m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)x[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(mx, m);
}

// Global mode: the per-edge pass ran with Q = C4 = 0.  Summed over the edges,
// Q and C4 enter the graphlet sums (each identity is linear in them) only
// through the type-multiset totals of 4-cliques K4 and of non-induced
// 4-cycles N_C4; added here to the undivided sums of h3..h8:
//   h3 -12 N_C4 - 36 K4, h4 -12 K4, h5 +4 N_C4 + 12 K4, h6 +48 K4,
//   h7 -30 K4, h8 +6 K4.   (c4 = N_C4, k4 = K4; arithmetic mod 2^64.)
__global__ void k_cyc_correct(unsigned long long *hist, int64_t off4, int64_t n4,
                              const unsigned long long *c4, const unsigned long long *k4) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n4;
         r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long w = c4[r], k = k4[r];
        hist[off4 + 0 * n4 + r] += (unsigned long long)(-12ll) * w + (unsigned long long)(-36ll) * k;
        hist[off4 + 1 * n4 + r] += (unsigned long long)(-12ll) * k;
        hist[off4 + 2 * n4 + r] += 4ull * w + 12ull * k;
        hist[off4 + 3 * n4 + r] += 48ull * k;
        hist[off4 + 4 * n4 + r] += (unsigned long long)(-30ll) * k;
        hist[off4 + 5 * n4 + r] += 6ull * k;
    }
}



// Launch shape of k_c4_pairs: per-warp histogram copies when they fit in 64 KB.
struct PairsConf {
    size_t smem;
    int priv;
    int64_t grid;
};
int c4_pairs_conf(int64_t n4, PairsConf &c) {
    const size_t one = (size_t)n4 * 8;
    c.priv = one * (kC4Threads / 32) <= (size_t)64 * 1024 ? 1 : 0;
    c.smem = c.priv ? one * (kC4Threads / 32) : one;
    TG_TRY(tg_allow_max_smem((const void *)k_c4_pairs));
    int per = 0;
    TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_c4_pairs, kC4Threads, c.smem));
    c.grid = (int64_t)tg_num_sms() * (per > 0 ? per : 1);
    return TG_OK;
}

// shared memory of k_c4_warp / k_c4_cta with tables of 2^lg slots
size_t c4_warp_smem(int64_t n4, int L, int lg) {
    const size_t e = (size_t)1 << lg;
    return (size_t)n4 * 8 + (size_t)kC4WarpWarps * (e + ((e * L + 1) >> 1)) * 4;
}
size_t c4_cta_smem(int64_t n4, int L, int lg) {
    const size_t e = (size_t)1 << lg;
    return (size_t)n4 * 8 + 8 + (e + ((e * L + 1) >> 1)) * 4;
}

// Global-mode waves of the split anchors list[0 .. nheavy) (degrees hdeg):
// walk positions per anchor (k_c4_prefix), warp units of about a quarter of a
// warp's share of each wave (k_c4_units), then per wave of K anchors (K =
// slots of p.scratch) k_c4_walk and k_c4_pairs.
int c4_walk_waves(const C4Params &p, const tg_graph *g, const uint32_t *list, int64_t nheavy,
                  const std::vector<int64_t> &hdeg, int64_t K, cudaStream_t s) {
    PairsConf pc;
    TG_TRY(c4_pairs_conf(p.n4, pc));
    const int64_t pgrid = pc.grid;
    const size_t psmem = pc.smem;
    const int ppriv = pc.priv;
    std::vector<int64_t> pb((size_t)nheavy + 1, 0);
    for (int64_t q = 0; q < nheavy; ++q) pb[q + 1] = pb[q] + hdeg[q];
    DevBuf<int64_t> dpb, dmp;
    DevBuf<unsigned long long> dtot;
    if (!dpb.alloc(nheavy + 1, s) || !dmp.alloc(pb[nheavy], s) || !dtot.alloc(nheavy, s))
        return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemcpyAsync(dpb.p, pb.data(), (nheavy + 1) * 8, cudaMemcpyHostToDevice, s));
    k_c4_prefix<<<(unsigned)nheavy, 256, 0, s>>>(list, dpb.p, g->rowptr, g->adj, dmp.p, dtot.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    std::vector<unsigned long long> tot_h((size_t)nheavy);
    TG_TRY_CUDA(cudaMemcpyAsync(tot_h.data(), dtot.p, nheavy * 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    int wper = 0;
    TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wper, k_c4_walk, kC4WalkWarps * 32, 0));
    if (wper < 1) wper = 1;
    const int64_t walk_grid = (int64_t)tg_num_sms() * wper;
    const int64_t warps = walk_grid * kC4WalkWarps;
    // waves: runs of at most K consecutive anchors of one counter width; an
    // anchor with fewer than 2^16 neighbours counts in 16-bit halves (no
    // count can reach 2^16), the others in 32-bit words
    std::vector<int64_t> wq0, wq1;
    std::vector<int> whalf;
    for (int64_t q = 0; q < nheavy;) {
        const int half = hdeg[q] < 65536 ? 1 : 0;
        int64_t e = q + 1;
        while (e < nheavy && e - q < K && (hdeg[e] < 65536 ? 1 : 0) == half) ++e;
        wq0.push_back(q);
        wq1.push_back(e);
        whalf.push_back(half);
        q = e;
    }
    const int64_t nwaves = (int64_t)wq0.size();
    std::vector<int64_t> us((size_t)nheavy + 1, 0), tg((size_t)nheavy, 1);
    for (int64_t w = 0; w < nwaves; ++w) {
        const int64_t q0 = wq0[w], q1 = wq1[w];
        unsigned long long wt = 0;
        for (int64_t q = q0; q < q1; ++q) wt += tot_h[q];
        const int64_t tgt =
            std::max<int64_t>(kWalkUnitMin, (int64_t)((wt + 4 * warps - 1) / (4 * warps)));
        for (int64_t q = q0; q < q1; ++q) {
            tg[q] = tgt;
            us[q + 1] = us[q] + (int64_t)((tot_h[q] + tgt - 1) / tgt);
        }
    }
    const int64_t nunits = us[nheavy];
    DevBuf<int64_t> dus, dtg;
    DevBuf<C4Unit> dun;
    DevBuf<unsigned long long> dq;
    if (!dus.alloc(nheavy + 1, s) || !dtg.alloc(nheavy, s) || !dun.alloc(nunits ? nunits : 1, s) ||
        !dq.alloc(nwaves, s))
        return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemcpyAsync(dus.p, us.data(), (nheavy + 1) * 8, cudaMemcpyHostToDevice, s));
    TG_TRY_CUDA(cudaMemcpyAsync(dtg.p, tg.data(), nheavy * 8, cudaMemcpyHostToDevice, s));
    TG_TRY_CUDA(cudaMemsetAsync(dq.p, 0, nwaves * 8, s));
    if (nunits > 0) {
        const unsigned ug = (unsigned)std::min<int64_t>((nunits + 255) / 256, 65535LL * 16);
        k_c4_units<<<ug, 256, 0, s>>>(dus.p, nheavy, dtg.p, dtot.p, dmp.p, dpb.p, list, g->rowptr,
                                      dun.p); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    C4Params pd = p;
    pd.phase = 0;
    pd.heavy = list;
    pd.mprefix = dmp.p;
    pd.pbase = dpb.p;
    const int L = p.L;
    for (int64_t w = 0; w < nwaves; ++w) {
        const int64_t q0 = wq0[w], q1 = wq1[w];
        pd.q0 = q0;
        pd.half = whalf[w];
        pd.bits_off = whalf[w] ? p.n * ((L + 1) >> 1) : p.n * (L + 1);
        pd.wunits = dun.p + us[q0];
        pd.n_units = us[q1] - us[q0];
        pd.queue = dq.p + w;
        if (pd.n_units > 0) {
            const int64_t need = (pd.n_units + kC4WalkWarps - 1) / kC4WalkWarps;
            const int64_t grid = std::min<int64_t>(walk_grid, need);
            k_c4_walk<<<(unsigned)grid, kC4WalkWarps * 32, 0, s>>>(pd); tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
        }
        k_c4_pairs<<<(unsigned)pgrid, kC4Threads, psmem, s>>>(pd, list + q0, (int)(q1 - q0), ppriv); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    // the host vectors are read by the copies above before they go out of scope
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}

// Window bits of the binned waves: the largest window whose dense table
// (16-bit counts when half, else 32-bit) fits kBinTable bytes, with room for
// the type in a 16-bit entry.
int c4_bin_wlg(int L, int half) {
    const int Lp = L + (L & 1);
    const size_t per = half ? (size_t)Lp * 2 : (size_t)L * 4;
    int tbits = 1;
    while ((1 << tbits) < L) ++tbits;
    int wlg = 5;
    while (wlg < 16 - tbits && ((size_t)1 << (wlg + 1)) * per <= kBinTable) ++wlg;
    return wlg;
}

// Global-mode binned waves of the anchors list[0 .. na) (degrees hdeg): walk
// positions per anchor (k_c4_prefix), warp units (k_c4_units), then per wave
// (anchors of one counter width, at most `ecap` walk positions in all) the
// count pass, the bucket offsets, the fill pass and the bucket pairs.
int c4_bin_waves(const tg_graph *g, const uint32_t *list, int64_t na,
                 const std::vector<int64_t> &hdeg, int64_t n4, unsigned long long *g4,
                 unsigned long long *work, int64_t ecap, cudaStream_t s) {
    const int L = g->L;
    const int64_t n = g->n;
    std::vector<int64_t> pb((size_t)na + 1, 0);
    for (int64_t q = 0; q < na; ++q) pb[q + 1] = pb[q] + hdeg[q];
    DevBuf<int64_t> dpb, dmp;
    DevBuf<unsigned long long> dtot;
    if (!dpb.alloc(na + 1, s) || !dmp.alloc(pb[na], s) || !dtot.alloc(na, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemcpyAsync(dpb.p, pb.data(), (na + 1) * 8, cudaMemcpyHostToDevice, s));
    k_c4_prefix<<<(unsigned)na, 256, 0, s>>>(list, dpb.p, g->rowptr, g->adj, dmp.p, dtot.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    std::vector<unsigned long long> tot_h((size_t)na);
    TG_TRY_CUDA(cudaMemcpyAsync(tot_h.data(), dtot.p, na * 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    int wper = 0;
    TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wper, k_c4_bin_walk<false>,
                                                              kC4WalkWarps * 32, 0));
    if (wper < 1) wper = 1;
    const int64_t walk_grid = (int64_t)tg_num_sms() * wper;
    const int64_t warps = walk_grid * kC4WalkWarps;
    // waves: consecutive anchors of one counter width, within ecap positions
    // and 2^22 buckets
    std::vector<int64_t> wq0, wq1;
    std::vector<int> whalf;
    int64_t wmax = 0;
    for (int64_t q = 0; q < na;) {
        const int half = hdeg[q] < 65536 ? 1 : 0;
        const int64_t W = (n + ((int64_t)1 << c4_bin_wlg(L, half)) - 1) >> c4_bin_wlg(L, half);
        int64_t e = q + 1;
        unsigned long long tot = tot_h[q];
        while (e < na && (hdeg[e] < 65536 ? 1 : 0) == half && tot + tot_h[e] <= (unsigned long long)ecap &&
               (e - q + 1) * W <= ((int64_t)1 << 22)) {
            tot += tot_h[e];
            ++e;
        }
        wq0.push_back(q);
        wq1.push_back(e);
        whalf.push_back(half);
        wmax = std::max<int64_t>(wmax, (e - q) * W);
        q = e;
    }
    const int64_t nwaves = (int64_t)wq0.size();
    std::vector<int64_t> us((size_t)na + 1, 0), tg((size_t)na, 1);
    unsigned long long wtmax = 0;
    for (int64_t w = 0; w < nwaves; ++w) {
        unsigned long long wt = 0;
        for (int64_t q = wq0[w]; q < wq1[w]; ++q) wt += tot_h[q];
        wtmax = std::max(wtmax, wt);
        const int64_t tgt =
            std::max<int64_t>(kWalkUnitMin, (int64_t)((wt + 4 * warps - 1) / (4 * warps)));
        for (int64_t q = wq0[w]; q < wq1[w]; ++q) {
            tg[q] = tgt;
            us[q + 1] = us[q] + (int64_t)((tot_h[q] + tgt - 1) / tgt);
        }
    }
    const int64_t nunits = us[na];
    DevBuf<int64_t> dus, dtg;
    DevBuf<C4Unit> dun;
    DevBuf<unsigned long long> dq;
    DevBuf<uint32_t> cnt, offs;
    DevBuf<uint16_t> bins;
    if (!dus.alloc(na + 1, s) || !dtg.alloc(na, s) || !dun.alloc(nunits ? nunits : 1, s) ||
        !dq.alloc(3 * nwaves, s) || !cnt.alloc(wmax + 1, s) || !offs.alloc(wmax + 1, s) ||
        !bins.alloc(wtmax ? wtmax : 1, s))
        return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemcpyAsync(dus.p, us.data(), (na + 1) * 8, cudaMemcpyHostToDevice, s));
    TG_TRY_CUDA(cudaMemcpyAsync(dtg.p, tg.data(), na * 8, cudaMemcpyHostToDevice, s));
    TG_TRY_CUDA(cudaMemsetAsync(dq.p, 0, 3 * nwaves * 8, s));
    if (nunits > 0) {
        const unsigned ug = (unsigned)std::min<int64_t>((nunits + 255) / 256, 65535LL * 16);
        k_c4_units<<<ug, 256, 0, s>>>(dus.p, na, dtg.p, dtot.p, dmp.p, dpb.p, list, g->rowptr,
                                      dun.p); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    C4Bin pb0{};
    pb0.rowptr = g->rowptr;
    pb0.adj = g->adj;
    pb0.ntype = g->ntype;
    pb0.L = L;
    pb0.n = n;
    pb0.heavy = list;
    pb0.mprefix = dmp.p;
    pb0.pbase = dpb.p;
    pb0.cnt = cnt.p;
    pb0.bins = bins.p;
    pb0.offs = offs.p;
    pb0.g4 = g4;
    pb0.n4 = n4;
    pb0.work = work;
    TG_TRY(tg_allow_max_smem((const void *)k_c4_bin_pairs));
    for (int64_t w = 0; w < nwaves; ++w) {
        const int64_t q0 = wq0[w], q1 = wq1[w];
        C4Bin pw = pb0;
        pw.half = whalf[w];
        pw.wlg = c4_bin_wlg(L, pw.half);
        pw.W = (n + ((int64_t)1 << pw.wlg) - 1) >> pw.wlg;
        pw.q0 = q0;
        pw.nb = (q1 - q0) * pw.W;
        pw.units = dun.p + us[q0];
        pw.n_units = us[q1] - us[q0];
        if (pw.n_units == 0) continue;
        const int64_t need = (pw.n_units + kC4WalkWarps - 1) / kC4WalkWarps;
        const int64_t grid = std::min<int64_t>(walk_grid, need);
        // bucket sizes, then offsets (one more entry, zero, takes the total)
        TG_TRY_CUDA(cudaMemsetAsync(cnt.p, 0, (pw.nb + 1) * 4, s));
        pw.queue = dq.p + 3 * w;
        k_c4_bin_walk<false><<<(unsigned)grid, kC4WalkWarps * 32, 0, s>>>(pw); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
        TG_TRY(tg_scan_u32(cnt.p, offs.p, pw.nb + 1, s));
        TG_TRY_CUDA(cudaMemcpyAsync(cnt.p, offs.p, pw.nb * 4, cudaMemcpyDeviceToDevice, s));
        pw.queue = dq.p + 3 * w + 1;
        k_c4_bin_walk<true><<<(unsigned)grid, kC4WalkWarps * 32, 0, s>>>(pw); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
        const int Lp = L + (L & 1);
        const size_t nfar = (size_t)1 << pw.wlg;
        const int P = L * (L + 1) / 2;
        const size_t psmem = (((size_t)n4 * 8 + 15) & ~(size_t)15) +
                             (L <= kBinAccL ? (((size_t)L * P * 8 + 15) & ~(size_t)15) : 0) +
                             (pw.half ? nfar * (Lp >> 1) : nfar * L) * 4 + nfar / 32 * 4 + nfar * 2;
        int pper = 0;
        TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pper, k_c4_bin_pairs,
                                                                  kBinPairThreads, psmem));
        if (pper < 1) pper = 1;
        const int64_t pgrid =
            std::min<int64_t>((int64_t)tg_num_sms() * pper, (pw.nb + kBinRun - 1) / kBinRun);
        pw.queue = dq.p + 3 * w + 2;
        k_c4_bin_pairs<<<(unsigned)pgrid, kBinPairThreads, psmem, s>>>(pw); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    // the host vectors are read by the copies above before they go out of scope
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}

}  // namespace

int tg_cyc_cycles(const tg_graph *g, unsigned long long *c4e, unsigned long long *g4,
                  unsigned long long *work, const tg_tune &t, const tg_part &part, cudaStream_t s) {
    if (g->M == 0) return TG_OK;
    const int L = g->L, L2 = L * L;
    const int64_t n = g->n;
    const bool global = g4 != nullptr;
    const int64_t n4 = tg_binom(L + 3, 4);
    const size_t avail = (size_t)tg_smem_optin() - 1024;
    // staged members per tile: their lists, ids and (a, u) accumulators
    const size_t per_member = 8 + 8 + 4 + 4 + (global ? 0 : (size_t)L2 * 8);
    const size_t fixed = 34 * 8 + 16 + 8 + (global ? (size_t)n4 * 8 : 0);
    if (fixed + 32 * per_member > avail) return TG_EINVAL;
    int TM = (int)std::min<size_t>(kC4Threads, (avail - fixed) / per_member);
    TM &= ~31;
    if (TM < 32) return TG_EINVAL;
    const size_t smem = (size_t)TM * per_member + fixed;
    TG_TRY(tg_allow_max_smem((const void *)k_c4));
    TG_TRY(tg_allow_max_smem((const void *)k_c4_split));
    TG_TRY(tg_allow_max_smem((const void *)k_c4_pairs));
    int per_sm = 0;
    TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_c4, kC4Threads, smem));
    if (per_sm < 1) per_sm = 1;
    const int64_t full_grid = (int64_t)tg_num_sms() * per_sm;

    // anchor costs and classes
    DevBuf<unsigned long long> cost, total;
    DevBuf<uint32_t> flags, pos;
    if (!cost.alloc(n, s) || !total.alloc(1, s) || !flags.alloc((size_t)kClsN * n, s) ||
        !pos.alloc((size_t)kClsN * n, s))
        return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(total.p, 0, 8, s));
    const unsigned wgrid = (unsigned)std::min<int64_t>((n * 32 + 255) / 256, 65535LL * 16);
    k_c4_cost<<<wgrid, 256, 0, s>>>(g->rowptr, g->adj, n, cost.p, total.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    unsigned long long tot = 0;
    TG_TRY_CUDA(cudaMemcpyAsync(&tot, total.p, 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    // Global mode: anchors whose far ends fit half a warp table (2^lg_w
    // slots) or half a CTA table (2^lg_c) count in shared memory; costlier
    // ones are split over the grid.  Per-edge mode: anchors above a share of
    // the total are split, the others take one CTA and a counter slot each.
    // hash_slots caps the warp table; unroll 1 splits none, 4 every anchor.
    int lg_w = 0, lg_c = 0;
    if (global) {
        lg_w = kC4WarpLgMax;
        while (lg_w > 5 && ((1 << lg_w) > t.hash_slots ||
                            c4_warp_smem(n4, L, lg_w) > (size_t)tg_smem_optin() - 1024))
            --lg_w;
        lg_c = kC4CtaLgMax;
        while (lg_c > lg_w && c4_cta_smem(n4, L, lg_c) > (size_t)tg_smem_optin() - 1024) --lg_c;
    }
    const unsigned long long lite = global ? (1ull << lg_w) / 2 : 0ull;
    const unsigned long long mid = global ? (1ull << lg_c) / 2 : 0ull;
    unsigned long long thr =
        global ? mid
               : std::max<unsigned long long>(tot / (unsigned long long)(16 * full_grid),
                                              (unsigned long long)1 << 12);
    if (t.unroll == 1) thr = ~0ull;
    if (t.unroll == 4) thr = 0ull;
    const unsigned egrid = (unsigned)std::min<int64_t>((n + 255) / 256, 65535LL * 16);
    k_c4_mark<<<egrid, 256, 0, s>>>(cost.p, n, thr, lite, mid, part.index, part.count, flags.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    for (int k = 0; k < kClsN; ++k) TG_TRY(tg_scan_u32(flags.p + (size_t)k * n, pos.p + (size_t)k * n, n, s));
    uint32_t lastp[kClsN], lastf[kClsN];
    for (int k = 0; k < kClsN; ++k) {
        TG_TRY_CUDA(cudaMemcpyAsync(&lastp[k], pos.p + (size_t)k * n + n - 1, 4, cudaMemcpyDeviceToHost, s));
        TG_TRY_CUDA(cudaMemcpyAsync(&lastf[k], flags.p + (size_t)k * n + n - 1, 4, cudaMemcpyDeviceToHost, s));
    }
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    int64_t ncls[kClsN];
    DevBuf<uint32_t> lists[kClsN];
    for (int k = 0; k < kClsN; ++k) {
        ncls[k] = (int64_t)lastp[k] + lastf[k];
        if (ncls[k] == 0) continue;
        if (!lists[k].alloc(ncls[k], s)) return TG_ENOMEM;
        k_c4_compact<<<egrid, 256, 0, s>>>(flags.p + (size_t)k * n, pos.p + (size_t)k * n, n,
                                           lists[k].p); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    const int64_t nheavy = ncls[kClsSplit];
    const uint32_t *list = lists[kClsSplit].p;
    std::vector<uint32_t> heavy((size_t)nheavy);
    std::vector<int64_t> hdeg((size_t)nheavy);
    if (nheavy > 0) {
        TG_TRY_CUDA(cudaMemcpyAsync(heavy.data(), list, nheavy * 4, cudaMemcpyDeviceToHost, s));
        TG_TRY_CUDA(cudaStreamSynchronize(s));
        // degrees of the split anchors: the list is ascending, so one copy of
        // rowptr up to the largest of them
        const int64_t top = (int64_t)heavy[(size_t)nheavy - 1] + 2;
        std::vector<int64_t> rp((size_t)top);
        TG_TRY_CUDA(cudaMemcpyAsync(rp.data(), g->rowptr, top * 8, cudaMemcpyDeviceToHost, s));
        TG_TRY_CUDA(cudaStreamSynchronize(s));
        for (int64_t q = 0; q < nheavy; ++q) hdeg[q] = rp[heavy[q] + 1] - rp[heavy[q]];
    }

    // counter slots: one per CTA of k_c4, one per split anchor of a wave; all
    // within a quarter of free memory
    const bool walk_waves = global && t.hash_slots >= 64;
    const int64_t slot_words = n * (L + 1) + (n + 31) / 32;
    const size_t slot_bytes = (size_t)slot_words * 4;
    int64_t want = 0;
    if (ncls[kClsSlot] > 0) want = std::min<int64_t>(full_grid, ncls[kClsSlot]);
    if (nheavy > 0)
        want = std::max<int64_t>(want, std::min<int64_t>(walk_waves ? kWaveMax : full_grid, nheavy));
    size_t free_b = 0, total_b = 0;
    TG_TRY_CUDA(cudaMemGetInfo(&free_b, &total_b));
    int64_t slots = std::min<int64_t>(want, (int64_t)(free_b / 4 / (slot_bytes ? slot_bytes : 1)));
    if (want > 0 && slots < 1) {
        if (slot_bytes > free_b / 2) return TG_ENOMEM;
        slots = 1;
    }
    DevBuf<uint32_t> scratch;
    DevBuf<unsigned long long> queue;
    if (!queue.alloc(kClsN, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(queue.p, 0, kClsN * 8, s));
    if (slots > 0) {
        if (!scratch.alloc((size_t)slots * slot_words, s)) return TG_ENOMEM;
        TG_TRY_CUDA(cudaMemsetAsync(scratch.p, 0, (size_t)slots * slot_bytes, s));
    }
    C4Params p{};
    p.rowptr = g->rowptr;
    p.adj = g->adj;
    p.eid = g->eid;
    p.ntype = g->ntype;
    p.n = n;
    p.L = L;
    p.tile = TM;
    p.acc_l2 = global ? 0 : L2;
    p.scratch = scratch.p;
    p.slot_words = slot_words;
    p.queue = queue.p;
    p.c4e = c4e;
    p.g4 = g4;
    p.n4 = n4;
    p.work = work;
    p.mark = 1;
    p.half = 0;
    p.bits_off = n * (L + 1);

    if (nheavy > 0 && walk_waves) {
        // global mode: each split anchor's walk is cut into position ranges of
        // about equal length (warp units); anchors whose walk averages
        // bin_fill wedges per far-end window they span go to the binned waves,
        // the others to waves of `slots` anchors counting in global memory,
        // whose far ends k_c4_pairs takes
        const int64_t bin_fill = t.c4_bin_fill > 0 ? t.c4_bin_fill : kBinFill;
        std::vector<unsigned long long> hcost((size_t)nheavy);
        {
            DevBuf<unsigned long long> hc;
            if (!hc.alloc(nheavy, s)) return TG_ENOMEM;
            k_gather_u64<<<(unsigned)std::min<int64_t>((nheavy + 255) / 256, 4096), 256, 0, s>>>(
                cost.p, list, nheavy, hc.p); tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
            TG_TRY_CUDA(cudaMemcpyAsync(hcost.data(), hc.p, nheavy * 8, cudaMemcpyDeviceToHost, s));
            TG_TRY_CUDA(cudaStreamSynchronize(s));
        }
        size_t fb = 0, tb = 0;
        TG_TRY_CUDA(cudaMemGetInfo(&fb, &tb));
        // bucket entries of one wave: 2 bytes each, within an eighth of free memory
        const int64_t ecap = std::min<int64_t>((int64_t)1 << 31, (int64_t)(fb / 16));
        std::vector<uint32_t> lb, ls;
        std::vector<int64_t> db, ds;
        for (int64_t q = 0; q < nheavy; ++q) {
            const int half = hdeg[q] < 65536 ? 1 : 0;
            const int wlg = c4_bin_wlg(L, half);
            const int64_t span = ((n - 1) >> wlg) - ((int64_t)heavy[q] >> wlg) + 1;
            const bool bin = t.unroll != 1 && hcost[q] >= (unsigned long long)bin_fill * span &&
                             hcost[q] <= (unsigned long long)ecap;
            (bin ? lb : ls).push_back(heavy[q]);
            (bin ? db : ds).push_back(hdeg[q]);
        }
        DevBuf<uint32_t> dlb, dls;
        if (!dlb.alloc(lb.size() + 1, s) || !dls.alloc(ls.size() + 1, s)) return TG_ENOMEM;
        if (!lb.empty()) {
            TG_TRY_CUDA(cudaMemcpyAsync(dlb.p, lb.data(), lb.size() * 4, cudaMemcpyHostToDevice, s));
            TG_TRY(c4_bin_waves(g, dlb.p, (int64_t)lb.size(), db, n4, g4, work, ecap, s));
        }
        if (!ls.empty()) {
            TG_TRY_CUDA(cudaMemcpyAsync(dls.p, ls.data(), ls.size() * 4, cudaMemcpyHostToDevice, s));
            TG_TRY(c4_walk_waves(p, g, dls.p, (int64_t)ls.size(), ds, slots, s));
        }
        TG_TRY_CUDA(cudaStreamSynchronize(s));
    } else if (nheavy > 0) {
        // member tiles of 'TM' members as units (both passes in per-edge mode)
        PairsConf pc;
        TG_TRY(c4_pairs_conf(n4, pc));
        const int64_t pgrid = pc.grid;
        const size_t psmem = pc.smem;
        const int ppriv = pc.priv;
        const int64_t wave = slots;
        std::vector<int4> units;
        std::vector<int64_t> wave_start;
        for (int64_t q0 = 0; q0 < nheavy; q0 += wave) {
            wave_start.push_back((int64_t)units.size());
            for (int64_t q = q0; q < std::min(nheavy, q0 + wave); ++q)
                for (int64_t tl = 0; tl < hdeg[q]; tl += TM)
                    units.push_back(make_int4((int)(q - q0), (int)heavy[q], (int)tl,
                                              (int)std::min<int64_t>(tl + TM, hdeg[q])));
        }
        wave_start.push_back((int64_t)units.size());
        DevBuf<int4> du;
        if (!du.alloc(units.size(), s)) return TG_ENOMEM;
        TG_TRY_CUDA(cudaMemcpyAsync(du.p, units.data(), units.size() * sizeof(int4),
                                    cudaMemcpyHostToDevice, s));
        DevBuf<unsigned long long> wq;
        if (!wq.alloc(2 * (wave_start.size() - 1), s)) return TG_ENOMEM;
        TG_TRY_CUDA(cudaMemsetAsync(wq.p, 0, 2 * (wave_start.size() - 1) * 8, s));
        C4Params ps = p;
        for (size_t w = 0; w + 1 < wave_start.size(); ++w) {
            const int64_t u0 = wave_start[w], nu = wave_start[w + 1] - u0;
            const int64_t a0 = (int64_t)w * wave, na = std::min<int64_t>(wave, nheavy - a0);
            ps.units = du.p + u0;
            ps.n_units = nu;
            const int64_t grid = std::min<int64_t>(full_grid, nu);
            for (int ph = 0; ph < (global ? 1 : 2); ++ph) {
                ps.phase = ph;
                ps.queue = wq.p + 2 * w + ph;
                k_c4_split<<<(unsigned)grid, kC4Threads, smem, s>>>(ps); tg_note_launch();
                TG_TRY_CUDA(cudaGetLastError());
            }
            k_c4_pairs<<<(unsigned)pgrid, kC4Threads, psmem, s>>>(ps, list + a0, (int)na, ppriv); tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
        }
        // the host vectors are read by the copy above before they go out of scope
        TG_TRY_CUDA(cudaStreamSynchronize(s));
    }
    // light anchors: one warp each, a CTA each, in shared memory
    if (ncls[kClsWarp] > 0) {
        const size_t wsmem = c4_warp_smem(n4, L, lg_w);
        TG_TRY(tg_allow_max_smem((const void *)k_c4_warp));
        int wper = 0;
        TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wper, k_c4_warp,
                                                                  kC4WarpWarps * 32, wsmem));
        if (wper < 1) wper = 1;
        int64_t wg = (int64_t)tg_num_sms() * wper;
        wg = std::min<int64_t>(wg, (ncls[kClsWarp] + 32 * kC4WarpWarps - 1) / (32 * kC4WarpWarps));
        C4Params pw = p;
        pw.queue = queue.p + kClsWarp;
        k_c4_warp<<<(unsigned)wg, kC4WarpWarps * 32, wsmem, s>>>(pw, lists[kClsWarp].p,
                                                                  ncls[kClsWarp], cost.p, lg_w); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    if (ncls[kClsCta] > 0) {
        const size_t csmem = c4_cta_smem(n4, L, lg_c);
        TG_TRY(tg_allow_max_smem((const void *)k_c4_cta));
        int cper = 0;
        TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cper, k_c4_cta, kC4CtaThreads,
                                                                  csmem));
        if (cper < 1) cper = 1;
        const int64_t cg = std::min<int64_t>((int64_t)tg_num_sms() * cper, ncls[kClsCta]);
        C4Params pc = p;
        pc.queue = queue.p + kClsCta;
        k_c4_cta<<<(unsigned)cg, kC4CtaThreads, csmem, s>>>(pc, lists[kClsCta].p, ncls[kClsCta],
                                                             cost.p, lg_c); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    // the other anchors, one CTA and counter slot each
    if (ncls[kClsSlot] > 0) {
        C4Params pl = p;
        pl.queue = queue.p + kClsSlot;
        pl.phase = 0;
        const int64_t grid = std::min<int64_t>(slots, ncls[kClsSlot]);
        k_c4<<<(unsigned)grid, kC4Threads, smem, s>>>(pl, lists[kClsSlot].p, ncls[kClsSlot]); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    return TG_OK;
}

int tg_cyc_cliques(const tg_graph *g, unsigned long long *k4e, unsigned long long *g4,
                   unsigned long long *work, const tg_tune &t, const tg_part &part, cudaStream_t s) {
    if (g->M == 0) return TG_OK;
    const int L = g->L;
    const bool global = g4 != nullptr;
    const int64_t n4 = tg_binom(L + 3, 4);
    const size_t hbytes = global ? (size_t)n4 * 8 : 0;
    const size_t avail = (size_t)tg_smem_optin() - 1024 - hbytes;
    const size_t per_entry = (size_t)(3 + L) * 4;
    // W entries staged per warp; hash_slots caps it (a small cap sends large W
    // sets down the path that tests membership in the global lists instead)
    int cap = (int)std::min<size_t>(std::min(512, t.hash_slots), avail / kK4Warps / per_entry);
    cap &= ~31;
    if (cap < 32) return TG_EINVAL;
    const size_t smem = (size_t)kK4Warps * cap * per_entry + hbytes;
    TG_TRY(tg_allow_max_smem((const void *)k_k4));
    int per_sm = 0;
    TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_k4, kK4Warps * 32, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)tg_num_sms() * per_sm;
    const int64_t need = (g->n + kK4Warps - 1) / kK4Warps;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    // up lists: each edge once, at its lower-ranked end
    DevBuf<int32_t> utoff;
    DevBuf<int64_t> utot, uoff;
    DevBuf<uint32_t> uadj, ueid;
    const int64_t n = g->n;
    if (!utoff.alloc((size_t)n * (L + 1), s) || !utot.alloc(n + 1, s) || !uoff.alloc(n + 1, s) ||
        !uadj.alloc(g->M, s) || !ueid.alloc(g->M, s))
        return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(utot.p + n, 0, 8, s));
    const unsigned wgrid = (unsigned)std::min<int64_t>((n * 32 + 255) / 256, 65535LL * 16);
    k_up_count<<<wgrid, 256, 0, s>>>(g->rowptr, g->adj, g->toff, n, L, utoff.p, utot.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    TG_TRY(tg_scan_i64(utot.p, uoff.p, n + 1, s));
    k_up_fill<<<wgrid, 256, 0, s>>>(g->rowptr, g->adj, g->eid, g->toff, utoff.p, uoff.p, n, L,
                                    uadj.p, ueid.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    DevBuf<unsigned long long> queue;
    if (!queue.alloc(1, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(queue.p, 0, 8, s));
    if (global) {
        // hash sets sized to the largest up list, within the hash_slots cap
        DevBuf<unsigned long long> mx;
        if (!mx.alloc(1, s)) return TG_ENOMEM;
        TG_TRY_CUDA(cudaMemsetAsync(mx.p, 0, 8, s));
        k_max_i64<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(utot.p, n, mx.p); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
        unsigned long long maxup = 0;
        TG_TRY_CUDA(cudaMemcpyAsync(&maxup, mx.p, 8, cudaMemcpyDeviceToHost, s));
        TG_TRY_CUDA(cudaStreamSynchronize(s));
        const size_t h4b = ((size_t)n4 * 8 + 15) & ~(size_t)15;
        K4GParams q{};
        q.uoff = uoff.p;
        q.uadj = uadj.p;
        q.utoff = utoff.p;
        q.ntype = g->ntype;
        q.n = n;
        q.m = g->M;
        q.L = L;
        q.queue = queue.p;
        q.g4 = g4;
        q.n4 = n4;
        q.work = work;
        q.pidx = part.index;
        q.pcnt = part.count;
        // bitmap kernels: one word for up lists of at most 32 (warp per x0),
        // padded rows of up to kRowsMaxWords words beyond (CTA per x0, in
        // three widths); a hash_slots cap below 64 sends every x0 to the
        // hash-set kernel instead
        const int bits_max = t.hash_slots >= 64 ? 32 * kRowsMaxWords - 31 * L : 0;
        if (bits_max > 0) {
            TG_TRY(tg_allow_max_smem((const void *)k_k4_bits_warp));
            int wper = 0;
            TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wper, k_k4_bits_warp,
                                                                      kBitsWarps * 32, h4b));
            if (wper < 1) wper = 1;
            int64_t wgrid2 = (int64_t)tg_num_sms() * wper;
            if (wgrid2 > (n + kBitsWarps - 1) / kBitsWarps) wgrid2 = (n + kBitsWarps - 1) / kBitsWarps;
            if (wgrid2 < 1) wgrid2 = 1;
            k_k4_bits_warp<<<(unsigned)wgrid2, kBitsWarps * 32, h4b, s>>>(q); tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
            DevBuf<uint32_t> flag, pos, list;
            const unsigned egrid = (unsigned)std::min<int64_t>((n + 255) / 256, 65535LL * 16);
            for (int wpl = 1; wpl <= 4; wpl *= 2) {
                // up lists whose padded rows need at most 32 * wpl words: every
                // type range adds at most 31 positions of padding
                const int lo = wpl == 1 ? kBitsWarpMax + 1 : 32 * 16 * wpl - 31 * L + 1;
                const int hi = 32 * 32 * wpl - 31 * L;
                if ((unsigned long long)lo > maxup || hi < lo) continue;
                if (!flag.p && (!flag.alloc(n, s) || !pos.alloc(n, s) || !list.alloc(n, s)))
                    return TG_ENOMEM;
                k_flag_range<<<egrid, 256, 0, s>>>(uoff.p, n, lo, hi, part.index, part.count, flag.p); tg_note_launch();
                TG_TRY_CUDA(cudaGetLastError());
                TG_TRY(tg_scan_u32(flag.p, pos.p, n, s));
                k_c4_compact<<<egrid, 256, 0, s>>>(flag.p, pos.p, n, list.p); tg_note_launch();
                TG_TRY_CUDA(cudaGetLastError());
                uint32_t lastp = 0, lastf = 0;
                TG_TRY_CUDA(cudaMemcpyAsync(&lastp, pos.p + n - 1, 4, cudaMemcpyDeviceToHost, s));
                TG_TRY_CUDA(cudaMemcpyAsync(&lastf, flag.p + n - 1, 4, cudaMemcpyDeviceToHost, s));
                TG_TRY_CUDA(cudaStreamSynchronize(s));
                const uint32_t nlist = lastp + lastf;
                if (nlist == 0) continue;
                const int dmax = (int)std::min<unsigned long long>(maxup, (unsigned long long)hi);
                int hlg = 5;
                while ((1 << hlg) < 2 * dmax) ++hlg;
                const size_t rsmem = h4b + (size_t)2 * (1u << hlg) * 4 +
                                     (size_t)(kRowsMaxWords + 2 * (TG_MAX_TYPES + 1)) * 4 +
                                     (size_t)(kRowsThreads / 32) * kRowsMaxWords * 4;
                const void *kfn = wpl == 1 ? (const void *)k_k4_rows<1>
                                  : wpl == 2 ? (const void *)k_k4_rows<2>
                                             : (const void *)k_k4_rows<4>;
                TG_TRY(tg_allow_max_smem(kfn));
                int rper = 0;
                TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rper, kfn, kRowsThreads,
                                                                          rsmem));
                if (rper < 1) rper = 1;
                int64_t rgrid = (int64_t)tg_num_sms() * rper;
                if (rgrid > nlist) rgrid = nlist;
                K4GParams r = q;
                r.hlg = hlg;
                r.rows_stride = (int64_t)dmax * 32 * wpl;
                DevBuf<uint32_t> rows;
                if (!rows.alloc((size_t)rgrid * (size_t)r.rows_stride, s)) return TG_ENOMEM;
                r.rows = rows.p;
                TG_TRY_CUDA(cudaMemsetAsync(queue.p, 0, 8, s));
                if (wpl == 1)
                    k_k4_rows<1><<<(unsigned)rgrid, kRowsThreads, rsmem, s>>>(r, list.p, nlist);
                else if (wpl == 2)
                    k_k4_rows<2><<<(unsigned)rgrid, kRowsThreads, rsmem, s>>>(r, list.p, nlist);
                else
                    k_k4_rows<4><<<(unsigned)rgrid, kRowsThreads, rsmem, s>>>(r, list.p, nlist);
                tg_note_launch();
                TG_TRY_CUDA(cudaGetLastError());
            }
        }
        if (maxup <= (unsigned long long)bits_max) return TG_OK;
        // hash sets for the longer up lists, sized to the largest one, within
        // the hash_slots cap
        int gcap = (int)std::min<unsigned long long>(std::min(1024, t.hash_slots), (maxup + 31) & ~31ull);
        if (gcap < 32) gcap = 32;
        int hlg = 5;
        while ((1 << hlg) < 2 * gcap) ++hlg;
        size_t gsmem = h4b + (size_t)kK4GWarps * (gcap + 2 * (1 << hlg)) * 4;
        while (gsmem > avail + hbytes && gcap > 32) {
            gcap -= 32;
            hlg = 5;
            while ((1 << hlg) < 2 * gcap) ++hlg;
            gsmem = h4b + (size_t)kK4GWarps * (gcap + 2 * (1 << hlg)) * 4;
        }
        TG_TRY(tg_allow_max_smem((const void *)k_k4_global));
        int gper = 0;
        TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&gper, k_k4_global,
                                                                  kK4GWarps * 32, gsmem));
        if (gper < 1) gper = 1;
        int64_t ggrid = (int64_t)tg_num_sms() * gper;
        const int64_t gneed = (g->M / kK4GChunk + kK4GWarps) / kK4GWarps;
        if (ggrid > gneed) ggrid = gneed;
        if (ggrid < 1) ggrid = 1;
        q.cap = gcap;
        q.hlg = hlg;
        q.min_d0 = bits_max;
        TG_TRY_CUDA(cudaMemsetAsync(queue.p, 0, 8, s));
        k_k4_global<<<(unsigned)ggrid, kK4GWarps * 32, gsmem, s>>>(q); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
        return TG_OK;
    }
    K4Params p{};
    p.uoff = uoff.p;
    p.uadj = uadj.p;
    p.ueid = ueid.p;
    p.utoff = utoff.p;
    p.ntype = g->ntype;
    p.n = g->n;
    p.L = L;
    p.P = L * (L + 1) / 2;
    p.cap = cap;
    p.queue = queue.p;
    p.k4e = k4e;
    p.g4 = g4;
    p.n4 = n4;
    p.work = work;
    k_k4<<<(unsigned)grid, kK4Warps * 32, smem, s>>>(p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    return TG_OK;
}

// ---------------------------------------------- global shortcut ----
int tg_cyc_correct(unsigned long long *hist, int L, const unsigned long long *c4w,
                   const unsigned long long *k4, cudaStream_t s) {
    const int64_t n4 = tg_binom(L + 3, 4);
    const int64_t off4 = tg_binom(L + 1, 2) + 2 * tg_binom(L + 2, 3);
    k_cyc_correct<<<(unsigned)((n4 + 255) / 256), 256, 0, s>>>(hist, off4, n4, c4w, k4); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    return TG_OK;
}
