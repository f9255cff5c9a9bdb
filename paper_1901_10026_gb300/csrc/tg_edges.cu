// The per-edge pass of the identities (the CYCLES kernel): for every edge of
// the order, its T sums over Gamma_i n Gamma_j and the closed forms of the
// orbits of Table 2, from Alg. 1's tau, the per-node sums Theta and D, and the
// per-edge 4-cycle and 4-clique counters (zero in whole-graph global mode,
// where tg_cyc_correct adds their totals afterwards).
//
// With ordered L x L matrices (first index: type of the member of the first
// set) B = sum over y in T of tau_jy, C = sum of tau_iy, DT = sum of d_y,
// Q = adjacent ordered pairs inside T, C4 = ordered pairs (x in Gamma_i \ {j},
// w in Gamma_j \ {i}) with x ~ w, S6 = C4 - B + [b = phi_i] |T^a|:
//   TSj = B - Q - [b = phi_i]|T^a|        TSi = C - Q - [b = phi_j]|T^a|
//   SSj = Theta_j - B - [a = phi_i] tau_ij SSi = Theta_i - C - [a = phi_j] tau_ij
//   DSj = D_j - DT - [a = phi_i] d_i      DSi = D_i - DT - [a = phi_j] d_j
//   G6 = S6 - TSi^T, Y and Z as in tg_reuse.cu; g12 = sym(Q)/2,
//   g10 = sym(TSi + TSj), g7 = sym(SiSi + SjSj)/2, g6 = sym(G6), g3 = sym(Y),
//   g8 = sym(Z).
// k_cyc_edge<true> (units of one j, Gamma_j as a shared-memory bitmap) and
// k_cyc_tsum_light (light units, Gamma_j in a per-warp hash map) store B, C,
// DT per edge; k_cyc_finish evaluates the identities per edge from a per-warp
// table of their L x L terms.  k_cyc_edge<false> does both in one kernel when
// the T sums would not fit in a quarter of free memory.
#include <algorithm>
#include <vector>

#include "tg_device.cuh"

using namespace tgd;

namespace {

struct EdgeParams {
    const int64_t *rowptr;
    const uint32_t *adj;
    const uint32_t *eid;
    const int32_t *toff;
    const uint8_t *ntype;
    const int2 *edges;
    const uint32_t *order;
    const uint32_t *ustart;
    const uint32_t *ulist;     // units this launch takes (NULL: units 0 .. nunits - 1)
    uint32_t nunits;
    const uint32_t *tau;       // per edge id, L counts
    const uint32_t *tau_adj;   // per adjacency entry: tau of its edge (L counts)
    const uint32_t *tdeg;      // L = 8: typed degrees, 8 per node (NULL otherwise)
    const uint32_t *theta;
    const uint32_t *dsum;
    const unsigned long long *c4e;
    const unsigned long long *k4e;
    int32_t L, P, k, level;
    int64_t nbits;
    uint32_t *emap;            // per CTA, nbits entries: the entry of y in Gamma_j
    unsigned long long *tsum;  // split mode: B, C and DT (3 L^2 uint64) per order position
    int64_t qbase;             // split mode: order position of tsum's first row
    unsigned long long *queue;
    uint64_t *rows;
    int64_t width;
    unsigned long long *hist;
    int64_t hist_len;
    int32_t hist_smem;
    int64_t off1, off2, off4, n4;
    unsigned long long *work;  // [0]: Gamma_i entries, [3]: T members
};

// The inputs of the identities for one edge (see tg_reuse.cu).
struct EdgeIn {
    int L, ti, tj;
    const unsigned long long *B, *C, *DT;  // ordered [a][b], this warp's shared memory
    const unsigned long long *c4;          // ordered [a][b]
    const unsigned long long *k4;          // unordered pairs
    const uint32_t *thi, *thj, *dvi, *dvj; // ordered [a][b]
    const uint32_t *tn;                    // tau of the edge: |T^t|
    const int32_t *toi, *toj;
};

struct EdgeEval {
    const EdgeIn &in;
    __device__ long long deg_i(int b) const { return __ldg(in.toi + b + 1) - __ldg(in.toi + b); }
    __device__ long long deg_j(int b) const { return __ldg(in.toj + b + 1) - __ldg(in.toj + b); }
    __device__ long long Tn(int a) const { return (long long)__ldg(in.tn + a); }
    __device__ long long Si(int a) const { return deg_i(a) - Tn(a) - (a == in.tj); }
    __device__ long long Sj(int a) const { return deg_j(a) - Tn(a) - (a == in.ti); }
    __device__ long long B(int a, int b) const { return (long long)in.B[a * in.L + b]; }
    __device__ long long C(int a, int b) const { return (long long)in.C[a * in.L + b]; }
    __device__ long long DT(int a, int b) const { return (long long)in.DT[a * in.L + b]; }
    __device__ long long Q(int a, int b) const {
        if (!in.k4) return 0;  // global mode: added from the 4-clique totals
        const long long k = (long long)__ldg(in.k4 + pair_index(in.L, a, b));
        return a == b ? 2 * k : k;
    }
    __device__ long long TSj(int a, int b) const {
        return B(a, b) - Q(a, b) - (b == in.ti ? Tn(a) : 0);
    }
    __device__ long long TSi(int a, int b) const {
        return C(a, b) - Q(a, b) - (b == in.tj ? Tn(a) : 0);
    }
    __device__ long long SSj(int a, int b) const {
        return (long long)__ldg(in.thj + a * in.L + b) - B(a, b) - (a == in.ti ? Tn(b) : 0);
    }
    __device__ long long SSi(int a, int b) const {
        return (long long)__ldg(in.thi + a * in.L + b) - C(a, b) - (a == in.tj ? Tn(b) : 0);
    }
    __device__ long long DSj(int a, int b) const {
        return (long long)__ldg(in.dvj + a * in.L + b) - DT(a, b) - (a == in.ti ? deg_i(b) : 0);
    }
    __device__ long long DSi(int a, int b) const {
        return (long long)__ldg(in.dvi + a * in.L + b) - DT(a, b) - (a == in.tj ? deg_j(b) : 0);
    }
    __device__ long long S6(int a, int b) const {
        const long long c4 = in.c4 ? (long long)__ldg(in.c4 + a * in.L + b) : 0;
        return c4 - B(a, b) + (b == in.ti ? Tn(a) : 0);
    }
    __device__ long long Ypart(int a, int b) const {  // Y without its G6 terms
        return DSi(a, b) - (b == in.ti ? Si(a) : 0) - SSi(a, b) + DSj(a, b) -
               (b == in.tj ? Sj(a) : 0) - SSj(a, b);
    }
    __device__ long long Z(int a, int b) const {
        return DT(a, b) - Tn(a) * ((b == in.ti) + (b == in.tj)) - Q(a, b) - TSi(a, b) -
               TSj(a, b);
    }
};

// Per-edge table of the identities' ordered L x L terms (one warp fills it,
// one lane per entry), so a type pair reads its terms instead of re-deriving
// them: TSi, TSj, SSi, SSj, G6 = S6 - TSi^T, Y without its G6 terms, Z, Q.
enum { XT_TSI = 0, XT_TSJ, XT_SSI, XT_SSJ, XT_G6, XT_YP, XT_Z, XT_Q, XT_N };

__device__ __forceinline__ void fill_terms(const EdgeEval &E, int L, long long *xt) {
    const int lane = threadIdx.x & 31, L2 = L * L;
    for (int m = lane; m < L2; m += 32) {
        const int a = m / L, b = m % L;
        xt[XT_TSI * L2 + m] = E.TSi(a, b);
        xt[XT_TSJ * L2 + m] = E.TSj(a, b);
        xt[XT_SSI * L2 + m] = E.SSi(a, b);
        xt[XT_SSJ * L2 + m] = E.SSj(a, b);
        xt[XT_YP * L2 + m] = E.Ypart(a, b);
        xt[XT_Z * L2 + m] = E.Z(a, b);
        xt[XT_Q * L2 + m] = E.Q(a, b);
        xt[XT_G6 * L2 + m] = E.S6(a, b);
    }
    __syncwarp();
    for (int m = lane; m < L2; m += 32) {
        const int a = m / L, b = m % L;
        xt[XT_G6 * L2 + m] -= xt[XT_TSI * L2 + b * L + a];
    }
    __syncwarp();
}

// Orbits g3..g12 of the type pair (t, u), t <= u, from the table.
__device__ __forceinline__ void pair_orbits_tab(const long long *xt, int L, int t, int u,
                                                uint64_t sit, uint64_t siu, uint64_t sjt,
                                                uint64_t sju, uint64_t tt, uint64_t tu,
                                                uint64_t g[10]) {
    const int L2 = L * L, m = t * L + u, mt = u * L + t;
    auto X = [&](int k, int mm) -> long long { return xt[k * L2 + mm]; };
    auto sym = [&](int k) -> long long { return t == u ? X(k, m) : X(k, m) + X(k, mt); };
    const uint64_t g12 = (uint64_t)(sym(XT_Q) / 2);
    const uint64_t g10 = (uint64_t)(sym(XT_TSI) + sym(XT_TSJ));
    const long long sisi_tu = X(XT_SSI, m) - X(XT_TSI, mt), sisi_ut = X(XT_SSI, mt) - X(XT_TSI, m);
    const long long sjsj_tu = X(XT_SSJ, m) - X(XT_TSJ, mt), sjsj_ut = X(XT_SSJ, mt) - X(XT_TSJ, m);
    const uint64_t g7 =
        (uint64_t)((t == u ? sisi_tu + sjsj_tu : sisi_tu + sjsj_tu + sisi_ut + sjsj_ut) / 2);
    const uint64_t g6 = (uint64_t)sym(XT_G6);
    const long long y_tu = X(XT_YP, m) - X(XT_G6, m) - X(XT_G6, mt);
    const long long y_ut = X(XT_YP, mt) - X(XT_G6, mt) - X(XT_G6, m);
    const uint64_t g3 = (uint64_t)(t == u ? y_tu : y_tu + y_ut);
    const uint64_t g8 = (uint64_t)sym(XT_Z);
    uint64_t g4, g5, g9, g11;
    closed_forms(t == u, sit, siu, sjt, sju, tt, tu, g6, g7, g10, g12, g4, g5, g9, g11);
    g[0] = g3;
    g[1] = g4;
    g[2] = g5;
    g[3] = g6;
    g[4] = g7;
    g[5] = g8;
    g[6] = g9;
    g[7] = g10;
    g[8] = g11;
    g[9] = g12;
}

__device__ __forceinline__ void hadd_e(const EdgeParams &p, unsigned long long *shist, int64_t x,
                                       unsigned long long v) {
    if (!v) return;
    if (p.hist_smem)
        atomicAdd(shist + x, v);
    else
        atomicAdd(p.hist + x, v);
}

// The 2- and 3-node entries of edge e, then the identities and closed forms
// per type pair (t, u) from B, C, DT (this warp's, in shared memory) and the
// per-edge or per-node rows; written to the row of e or added to the
// histogram.  Called by the 32 lanes of the edge's warp.
__device__ void edge_finish(const EdgeParams &p, unsigned long long *shist, int64_t e, int i, int j,
                            int ti, int tj, const int32_t *toi, const int32_t *toj,
                            const uint32_t *tn, const unsigned long long *Bm,
                            const unsigned long long *Cm, const unsigned long long *Dm,
                            long long *xt) {
    const int lane = threadIdx.x & 31;
    const int L = p.L, P = p.P, L2 = L * L;
    // 2- and 3-node entries
    if (p.rows) {
        uint64_t *row = p.rows + e * p.width;
        for (int t = lane; t < L; t += 32) {
            const uint32_t tt = __ldg(tn + t);
            const int64_t si = (int64_t)(__ldg(toi + t + 1) - __ldg(toi + t)) - tt - (t == tj);
            const int64_t sj = (int64_t)(__ldg(toj + t + 1) - __ldg(toj + t)) - tt - (t == ti);
            row[t] = (uint64_t)(si + sj);
            row[L + t] = tt;
        }
    } else {
        if (lane == 0) {
            int a = ti, b = tj;
            sort2(a, b);
            hadd_e(p, shist, (int64_t)a + (int64_t)(b + 1) * b / 2, 1ull);
        }
        for (int t = lane; t < L; t += 32) {
            const uint32_t tt = __ldg(tn + t);
            const int64_t si = (int64_t)(__ldg(toi + t + 1) - __ldg(toi + t)) - tt - (t == tj);
            const int64_t sj = (int64_t)(__ldg(toj + t + 1) - __ldg(toj + t)) - tt - (t == ti);
            int a = ti, b = tj, cc = t;
            sort2(a, b);
            sort2(b, cc);
            sort2(a, b);
            const int64_t r = colex3(a, b, cc);
            hadd_e(p, shist, p.off1 + r, (unsigned long long)(si + sj));
            hadd_e(p, shist, p.off2 + r, (unsigned long long)tt);
        }
    }
    if (p.k == 4) {
        EdgeIn in;
        in.L = L;
        in.ti = ti;
        in.tj = tj;
        in.B = Bm;
        in.C = Cm;
        in.DT = Dm;
        in.c4 = p.c4e ? p.c4e + e * L2 : nullptr;
        in.k4 = p.k4e ? p.k4e + e * P : nullptr;
        in.thi = p.theta + (int64_t)i * L2;
        in.thj = p.theta + (int64_t)j * L2;
        in.dvi = p.dsum + (int64_t)i * L2;
        in.dvj = p.dsum + (int64_t)j * L2;
        in.tn = tn;
        in.toi = toi;
        in.toj = toj;
        const EdgeEval E{in};
        fill_terms(E, L, xt);
        for (int pr = lane; pr < P; pr += 32) {
            int t, u;
            unpair(L, pr, t, u);
            uint64_t g[10];
            pair_orbits_tab(xt, L, t, u, (uint64_t)E.Si(t), (uint64_t)E.Si(u), (uint64_t)E.Sj(t),
                            (uint64_t)E.Sj(u), (uint64_t)E.Tn(t), (uint64_t)E.Tn(u), g);
            if (p.rows) {
                uint64_t *row = p.rows + e * p.width + 2 * L;
                if (p.level == TG_ORBIT) {
#pragma unroll
                    for (int o = 0; o < 10; ++o) row[o * P + pr] = g[o];
                } else {
                    row[0 * P + pr] = g[0] + g[1];
                    row[1 * P + pr] = g[2];
                    row[2 * P + pr] = g[3];
                    row[3 * P + pr] = g[4] + g[5] + g[6];
                    row[4 * P + pr] = g[7] + g[8];
                    row[5 * P + pr] = g[9];
                }
            } else {
                const uint64_t h[6] = {g[0] + g[1], g[2], g[3], g[4] + g[5] + g[6],
                                       g[7] + g[8], g[9]};
                if (h[0] | h[1] | h[2] | h[3] | h[4] | h[5]) {
                    int a = ti, b = tj, cc = t, d = u;
                    sort2(a, b);
                    sort2(cc, d);
                    sort2(a, cc);
                    sort2(b, d);
                    sort2(b, cc);
                    const int64_t r = colex4(a, b, cc, d);
#pragma unroll
                    for (int qq = 0; qq < 6; ++qq) hadd_e(p, shist, p.off4 + qq * p.n4 + r, h[qq]);
                }
            }
        }
    }
}

// T sums of edge e = (i, j): B, C, DT (ordered [a][b], uint64, this warp's
// shared memory, zeroed by the caller) over y in T = Gamma_i n Gamma_j.
// Alg. 1's tau row of e gives |T^a| for every type a, and Gamma_i is sorted by
// (type, id), so the scan skips the type ranges of Gamma_i that hold no T
// member and leaves a range as soon as its |T^a| members are found (T members
// have high degree, i.e. small ids, so they come early in their range).
// find(w, pjy) tells whether the entry w of Gamma_i lies in Gamma_j, and gives
// the adjacency entry of the edge (j, w).  Triangle counts are read per
// adjacency entry: tau_iy at Gamma_i's own entry (along the scan) and tau_jy
// at that entry (Gamma_j's rows stay in L2 while its unit runs).  A chunk
// with at least kLaneGather T members (all of type a) has each member lane
// load its own three rows at once (16-byte loads of 32-byte rows when L = 8,
// the typed degrees from a per-node row array) and sums each row over the
// warp with one reduce-scatter; a sparser chunk gives its members to lane
// groups of 8 (L <= 8) or 16 lanes, lane b of a group reading tau_jy[b],
// tau_iy[b] and d_y^b (three coalesced rows), the groups' values added
// across the warp and added to B, C, DT by the first group.  Called by all
// 32 lanes; adds the entries of Gamma_i it read to *read and the T members to
// *nt (lane-uniform values).
constexpr int kLaneGather = 6;  // members per chunk from which each member lane gathers its own rows

// Sum of v[0..7] over the 32 lanes, scattered: lane x ends with the total of
// index ((x >> 4) & 1) * 4 + ((x >> 3) & 1) * 2 + ((x >> 2) & 1) (nine
// shuffles instead of eight full reductions); returns that index via *idx.
__device__ __forceinline__ uint32_t warp_sum8_scatter(uint32_t (&v)[8], int lane, int *idx) {
    const bool h4 = (lane >> 4) & 1, h3 = (lane >> 3) & 1, h2 = (lane >> 2) & 1;
    uint32_t a[4], b2[2];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t keep = h4 ? v[k + 4] : v[k], give = h4 ? v[k] : v[k + 4];
        a[k] = keep + __shfl_xor_sync(kFull, give, 16);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const uint32_t keep = h3 ? a[k + 2] : a[k], give = h3 ? a[k] : a[k + 2];
        b2[k] = keep + __shfl_xor_sync(kFull, give, 8);
    }
    uint32_t c = (h2 ? b2[1] : b2[0]) + __shfl_xor_sync(kFull, h2 ? b2[0] : b2[1], 4);
    c += __shfl_xor_sync(kFull, c, 2);
    c += __shfl_xor_sync(kFull, c, 1);
    *idx = (h4 ? 4 : 0) + (h3 ? 2 : 0) + (h2 ? 1 : 0);
    return c;
}

template <class Find>
__device__ __forceinline__ void tsum_edge(const EdgeParams &p, int64_t e, int64_t bi,
                                          const int32_t *toi, Find find, unsigned long long *Bm,
                                          unsigned long long *Cm, unsigned long long *Dm,
                                          unsigned long long &read, unsigned long long &nt) {
    const int L = p.L, lane = threadIdx.x & 31;
    const int gsz = L <= 8 ? 8 : 16, ng = 32 / gsz, grp = lane / gsz, b = lane % gsz;
    const uint32_t *tn = p.tau + e * L;
    for (int a = 0; a < L; ++a) {
        const int need = (int)__ldg(tn + a);
        if (need == 0) continue;
        const int r0 = __ldg(toi + a), r1 = __ldg(toi + a + 1);
        int found = 0;
        uint32_t nxt = r0 + lane < r1 ? __ldg(p.adj + bi + r0 + lane) : 0u;  // next chunk, in flight
        for (int c0 = r0; c0 < r1 && found < need; c0 += 32) {
            const int x = c0 + lane;
            bool isT = false;
            uint32_t w = nxt, ejy = 0;
            nxt = c0 + 32 + lane < r1 ? __ldg(p.adj + bi + c0 + 32 + lane) : 0u;
            if (x < r1) isT = find(w, ejy);
            unsigned tb = __ballot_sync(kFull, isT);
            found += __popc(tb);
            read += (unsigned long long)min(32, r1 - c0);
            nt += (unsigned long long)__popc(tb);
            if (p.tdeg && __popc(tb) >= kLaneGather) {
                // L = 8 and many members in this chunk: each member lane
                // loads its own three 32-byte rows (two 16-byte loads each, all
                // in flight at once), then one reduce-scatter per row
                uint4 r[6];
                if (isT) {
                    const uint4 *rb = reinterpret_cast<const uint4 *>(p.tau_adj + (int64_t)ejy * 8);
                    const uint4 *rc = reinterpret_cast<const uint4 *>(p.tau_adj + (bi + x) * 8);
                    const uint4 *rd = reinterpret_cast<const uint4 *>(p.tdeg + (int64_t)(w & TG_IDMASK) * 8);
                    r[0] = __ldg(rb);
                    r[1] = __ldg(rb + 1);
                    r[2] = __ldg(rc);
                    r[3] = __ldg(rc + 1);
                    r[4] = __ldg(rd);
                    r[5] = __ldg(rd + 1);
                } else {
#pragma unroll
                    for (int q = 0; q < 6; ++q) r[q] = make_uint4(0u, 0u, 0u, 0u);
                }
                unsigned long long *dst[3] = {Bm, Cm, Dm};
#pragma unroll
                for (int row = 0; row < 3; ++row) {
                    uint32_t v[8] = {r[2 * row].x, r[2 * row].y, r[2 * row].z, r[2 * row].w,
                                     r[2 * row + 1].x, r[2 * row + 1].y, r[2 * row + 1].z, r[2 * row + 1].w};
                    int bidx = 0;
                    const uint32_t sum = warp_sum8_scatter(v, lane, &bidx);
                    if ((lane & 3) == 0) dst[row][a * 8 + bidx] += sum;
                }
                continue;
            }
            if (L < 8 && __popc(tb) >= kLaneGather) {
                // the same with scalar loads (rows of L < 8 counts)
                uint32_t v[8];
                int bidx = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = (isT && q < L) ? __ldg(p.tau_adj + (int64_t)ejy * L + q) : 0u;
                uint32_t sum = warp_sum8_scatter(v, lane, &bidx);
                if ((lane & 3) == 0 && bidx < L) Bm[a * L + bidx] += sum;
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = (isT && q < L) ? __ldg(p.tau_adj + (bi + x) * L + q) : 0u;
                sum = warp_sum8_scatter(v, lane, &bidx);
                if ((lane & 3) == 0 && bidx < L) Cm[a * L + bidx] += sum;
                {
                    const int32_t *ty = p.toff + (int64_t)(w & TG_IDMASK) * (L + 1);
                    int32_t prev = isT ? __ldg(ty) : 0;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int32_t nx = (isT && q < L) ? __ldg(ty + q + 1) : prev;
                        v[q] = (uint32_t)(nx - prev);
                        prev = nx;
                    }
                }
                sum = warp_sum8_scatter(v, lane, &bidx);
                if ((lane & 3) == 0 && bidx < L) Dm[a * L + bidx] += sum;
                continue;
            }
            while (tb) {
                // group grp takes the grp-th remaining member
                unsigned m = tb;
                for (int k = 0; k < grp; ++k) m &= m - 1u;
                const bool has = m != 0u;
                const int src = has ? __ffs(m) - 1 : 0;
                for (int k = 0; k < ng; ++k) tb &= tb - 1u;
                const uint32_t wy = __shfl_sync(kFull, w, src);
                const uint32_t ej = __shfl_sync(kFull, ejy, src);
                uint32_t vb = 0, vc = 0, vd = 0;
                if (has && b < L) {
                    const int32_t *ty = p.toff + (int64_t)(wy & TG_IDMASK) * (L + 1);
                    vb = __ldg(p.tau_adj + (int64_t)ej * L + b);
                    vc = __ldg(p.tau_adj + (bi + c0 + src) * L + b);
                    vd = (uint32_t)(__ldg(ty + b + 1) - __ldg(ty + b));
                }
                for (int o = gsz; o < 32; o <<= 1) {
                    vb += __shfl_xor_sync(kFull, vb, o);
                    vc += __shfl_xor_sync(kFull, vc, o);
                    vd += __shfl_xor_sync(kFull, vd, o);
                }
                if (grp == 0 && b < L) {
                    Bm[a * L + b] += vb;
                    Cm[a * L + b] += vc;
                    Dm[a * L + b] += vd;
                }
            }
        }
    }
}

constexpr int kEdgeMaxThreads = 512;
constexpr int kTsumThreads = 1024;

// One CTA per unit of edges sharing j (Gamma_j bitmap and edge-id map shared
// by the CTA), one warp per edge: T = Gamma_i n Gamma_j gives B, C, DT.
// kWrite: store them for k_cyc_finish (fewer registers, more warps in
// flight for the gathers); else finish the edge here.
template <bool kWrite>
__global__ void __launch_bounds__(kWrite ? kTsumThreads : kEdgeMaxThreads) k_cyc_edge(EdgeParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int L = p.L, L2 = L * L;
    size_t off = 0;
    unsigned long long *shist = reinterpret_cast<unsigned long long *>(smem);
    if (p.hist_smem) off += ((size_t)p.hist_len * 8 + 15) & ~(size_t)15;
    // per warp: B, C, DT, then (finishing here) the table of identity terms
    const size_t tbytes = ((size_t)3 * L2 * 8 + 15) & ~(size_t)15;
    const size_t wbytes = tbytes + (kWrite ? 0 : (size_t)XT_N * L2 * 8);
    unsigned long long *Bm = reinterpret_cast<unsigned long long *>(smem + off + warp * wbytes);
    unsigned long long *Cm = Bm + L2;
    unsigned long long *Dm = Cm + L2;
    long long *xt = reinterpret_cast<long long *>(smem + off + warp * wbytes + tbytes);
    off += (size_t)W * wbytes;
    unsigned long long *s_unit = reinterpret_cast<unsigned long long *>(smem + off);
    off += 16;
    uint32_t *bm = reinterpret_cast<uint32_t *>(smem + off);
    const int64_t bwords = (p.nbits + 31) >> 5;
    uint32_t *emap = p.emap + (int64_t)blockIdx.x * p.nbits;
    for (int64_t x = tid; x < bwords; x += blockDim.x) bm[x] = 0u;
    if (p.hist_smem)
        for (int64_t x = tid; x < p.hist_len; x += blockDim.x) shist[x] = 0;
    const int64_t *__restrict__ rowptr = p.rowptr;
    const uint32_t *__restrict__ adj = p.adj;
    int cur_j = -1;
    int64_t cur_bj = 0;
    int cur_dj = 0;
    unsigned long long wk_gamma = 0, wk_t = 0;

    for (;;) {
        __syncthreads();
        if (tid == 0) *s_unit = atomicAdd(p.queue, 1ull);
        __syncthreads();
        const unsigned long long item = *s_unit;
        if (item >= p.nunits) break;
        const uint32_t un = p.ulist ? p.ulist[item] : (uint32_t)item;
        const uint32_t p0 = p.ustart[un], p1 = p.ustart[un + 1];
        const int2 ab0 = p.edges[p.order[p0]];
        const int j = min(ab0.x, ab0.y);
        const int64_t bj = rowptr[j];
        const int dj = (int)(rowptr[j + 1] - bj);
        if (p.k == 4 && j != cur_j) {
            for (int x = tid; x < cur_dj; x += blockDim.x) {
                const uint32_t id = __ldg(adj + cur_bj + x) & TG_IDMASK;
                if ((int64_t)id < p.nbits) atomicAnd(&bm[id >> 5], ~(1u << (id & 31u)));
            }
            __syncthreads();
            for (int x = tid; x < dj; x += blockDim.x) {
                const uint32_t id = __ldg(adj + bj + x) & TG_IDMASK;
                if ((int64_t)id < p.nbits) {
                    atomicOr(&bm[id >> 5], 1u << (id & 31u));
                    emap[id] = (uint32_t)(bj + x);
                }
            }
            cur_j = j;
            cur_bj = bj;
            cur_dj = dj;
            __syncthreads();
        }
        for (uint32_t q = p0 + warp; q < p1; q += W) {
            const int64_t e = p.order[q];
            const int2 ab = p.edges[e];
            const int i = max(ab.x, ab.y);
            const int ti = p.ntype[i], tj = p.ntype[j];
            const int64_t bi = rowptr[i];
            const int32_t *toi = p.toff + (int64_t)i * (L + 1);
            const int32_t *toj = p.toff + (int64_t)j * (L + 1);
            const uint32_t *tn = p.tau + e * L;
            if (p.k == 4) {
                for (int x = lane; x < 3 * L2; x += 32) Bm[x] = 0ull;
                __syncwarp();
                // T = Gamma_i n Gamma_j: sums of tau_jy, tau_iy and d_y by types
                const uint32_t pj = ((uint32_t)tj << TG_TSHIFT) | (uint32_t)j;
                auto find = [&](uint32_t w, uint32_t &ejy) -> bool {
                    const uint32_t id = w & TG_IDMASK;
                    if ((int)id == j) return false;
                    if ((int64_t)id < p.nbits) {
                        if (!bm_test(bm, id)) return false;
                        ejy = __ldcg(emap + id);  // written for this j before the barrier
                        return true;
                    }
                    ejy = entry_to(rowptr, adj, p.toff, L, bj, dj, toj, pj, w);
                    return ejy != 0xffffffffu;
                };
                unsigned long long rd = 0, nt = 0;
                tsum_edge(p, e, bi, toi, find, Bm, Cm, Dm, rd, nt);
                if (lane == 0) {
                    wk_gamma += rd;
                    wk_t += nt;
                }
                __syncwarp();
            }
            if (kWrite) {
                // B, C, DT of this edge for the finishing kernel
                unsigned long long *dst = p.tsum + ((int64_t)q - p.qbase) * 3 * L2;
                for (int x = lane; x < 3 * L2; x += 32) dst[x] = Bm[x];
            } else {
                edge_finish(p, shist, e, i, j, ti, tj, toi, toj, tn, Bm, Cm, Dm, xt);
            }
            __syncwarp();  // this warp's matrices are cleared for the next edge
        }
    }
    if (p.hist_smem) {
        __syncthreads();
        for (int64_t x = tid; x < p.hist_len; x += blockDim.x)
            if (shist[x]) atomicAdd(p.hist + x, shist[x]);
    }
    if (p.work && lane == 0) {
        atomicAdd(p.work + 0, wk_gamma);
        atomicAdd(p.work + 3, wk_t);
    }
}

// T sums of light units (Gamma_j of at most TG_LIGHT_DEGREE entries): one warp
// per unit, Gamma_j in a per-warp hash map from node id to the edge id of
// (j, y); the unit's edges one after the other, no CTA barrier.
constexpr int kTsumLightWarps = 8;

__global__ void __launch_bounds__(kTsumLightWarps * 32) k_cyc_tsum_light(EdgeParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = p.L, L2 = L * L;
    const size_t wbytes = (((size_t)3 * L2 * 8 + 15) & ~(size_t)15) + (size_t)2 * 4 * (1 << TG_LIGHT_LG);
    unsigned long long *Bm = reinterpret_cast<unsigned long long *>(smem + warp * wbytes);
    unsigned long long *Cm = Bm + L2;
    unsigned long long *Dm = Cm + L2;
    uint32_t *hk = reinterpret_cast<uint32_t *>(smem + warp * wbytes + (((size_t)3 * L2 * 8 + 15) & ~(size_t)15));
    uint32_t *hv = hk + (1 << TG_LIGHT_LG);
    const int64_t *__restrict__ rowptr = p.rowptr;
    const uint32_t *__restrict__ adj = p.adj;
    unsigned long long wk_gamma = 0, wk_t = 0;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(p.queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= p.nunits) break;
        const uint32_t un = p.ulist[item];
        const uint32_t p0 = p.ustart[un], p1 = p.ustart[un + 1];
        const int2 ab0 = p.edges[p.order[p0]];
        const int j = min(ab0.x, ab0.y);
        const int64_t bj = rowptr[j];
        const int dj = (int)(rowptr[j + 1] - bj);
        for (int q = lane; q < (1 << TG_LIGHT_LG); q += 32) hk[q] = 0u;
        __syncwarp();
        for (int x = lane; x < dj; x += 32)
            hmap_put(hk, hv, TG_LIGHT_LG, __ldg(adj + bj + x) & TG_IDMASK, (uint32_t)(bj + x));
        __syncwarp();
        for (uint32_t q = p0; q < p1; ++q) {
            const int64_t e = p.order[q];
            const int2 ab = p.edges[e];
            const int i = max(ab.x, ab.y);
            const int64_t bi = rowptr[i];
            for (int x = lane; x < 3 * L2; x += 32) Bm[x] = 0ull;
            __syncwarp();
            auto find = [&](uint32_t w, uint32_t &ejy) -> bool {
                const uint32_t id = w & TG_IDMASK;
                if ((int)id == j) return false;
                ejy = hmap_get(hk, hv, TG_LIGHT_LG, id);
                return ejy != 0xffffffffu;
            };
            unsigned long long rd = 0, nt = 0;
            tsum_edge(p, e, bi, p.toff + (int64_t)i * (L + 1), find, Bm, Cm, Dm, rd, nt);
            __syncwarp();
            if (lane == 0) {
                wk_gamma += rd;
                wk_t += nt;
            }
            unsigned long long *dst = p.tsum + ((int64_t)q - p.qbase) * 3 * L2;
            for (int x = lane; x < 3 * L2; x += 32) dst[x] = Bm[x];
            __syncwarp();
        }
    }
    if (p.work && lane == 0) {
        atomicAdd(p.work + 0, wk_gamma);
        atomicAdd(p.work + 3, wk_t);
    }
}

// Warp per edge of the order positions [p.qbase, p.qbase + count): B, C, DT
// from k_cyc_edge<true> or k_cyc_tsum_light, then edge_finish.
__global__ void __launch_bounds__(256) k_cyc_finish(EdgeParams p, int64_t count) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = p.L, L2 = L * L;
    size_t off = 0;
    unsigned long long *shist = reinterpret_cast<unsigned long long *>(smem);
    if (p.hist_smem) off += ((size_t)p.hist_len * 8 + 15) & ~(size_t)15;
    const size_t tbytes = ((size_t)3 * L2 * 8 + 15) & ~(size_t)15;
    const size_t wbytes = tbytes + (size_t)XT_N * L2 * 8;
    unsigned long long *Bm = reinterpret_cast<unsigned long long *>(smem + off + warp * wbytes);
    long long *xt = reinterpret_cast<long long *>(smem + off + warp * wbytes + tbytes);
    if (p.hist_smem) {
        for (int64_t x = tid; x < p.hist_len; x += blockDim.x) shist[x] = 0;
        __syncthreads();
    }
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + tid) >> 5; r < count; r += nw) {
        const int64_t e = p.order[p.qbase + r];
        const int2 ab = p.edges[e];
        const int j = min(ab.x, ab.y), i = max(ab.x, ab.y);
        const unsigned long long *src = p.tsum + r * 3 * L2;
        for (int x = lane; x < 3 * L2; x += 32) Bm[x] = __ldg(src + x);
        __syncwarp();
        edge_finish(p, shist, e, i, j, p.ntype[i], p.ntype[j], p.toff + (int64_t)i * (L + 1),
                    p.toff + (int64_t)j * (L + 1), p.tau + e * L, Bm, Bm + L2, Bm + 2 * L2, xt);
        __syncwarp();
    }
    if (p.hist_smem) {
        __syncthreads();
        for (int64_t x = tid; x < p.hist_len; x += blockDim.x)
            if (shist[x]) atomicAdd(p.hist + x, shist[x]);
    }
}


int num_sms_e() {
    int dev = 0, sms = 0;
    (void)cudaGetDevice(&dev);
    (void)cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

int smem_optin_e() {
    int dev = 0, v = 0;
    (void)cudaGetDevice(&dev);
    (void)cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v > 0 ? v : 48 * 1024;
}

}  // namespace

namespace {
// tdeg[v 8 + t] = d_v^t (L = 8), rows of 32 bytes for 16-byte loads
__global__ void k_typed_degrees(const int32_t *toff, int64_t n, uint32_t *tdeg) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n * 8;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = x >> 3;
        const int t = (int)(x & 7);
        tdeg[x] = (uint32_t)(toff[v * 9 + t + 1] - toff[v * 9 + t]);
    }
}
}  // namespace

int tg_cyc_edges(const tg_graph *g, int k, int level, const uint32_t *order, int64_t count,
                 const tg_units &un, uint64_t *rows, int64_t width,
                 unsigned long long *hist, const uint32_t *tau, const uint32_t *tau_adj,
                 const uint32_t *theta,
                 const uint32_t *dsum, const unsigned long long *c4e,
                 const unsigned long long *k4e, unsigned long long *work, const tg_tune &t,
                 cudaStream_t s) {
    if (un.nunits == 0 || count <= 0) return TG_OK;
    const int L = g->L, L2 = L * L;
    if (g->max_degree >= ((int64_t)1 << 27)) return TG_EOVERFLOW;  // 32-lane uint32 sums
    EdgeParams p{};
    p.rowptr = g->rowptr;
    p.adj = g->adj;
    p.eid = g->eid;
    p.toff = g->toff;
    p.ntype = g->ntype;
    p.edges = g->edges;
    p.order = order;
    p.ustart = un.ustart.p;
    p.tau = tau;
    p.tau_adj = tau_adj;
    DevBuf<uint32_t> tdeg;
    if (L == 8 && k == 4 && tdeg.alloc((size_t)g->n * 8, s)) {
        k_typed_degrees<<<(unsigned)std::min<int64_t>((g->n * 8 + 255) / 256, 65535LL * 16), 256, 0, s>>>(
            g->toff, g->n, tdeg.p); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
        p.tdeg = tdeg.p;
    }
    p.theta = theta;
    p.dsum = dsum;
    p.c4e = c4e;
    p.k4e = k4e;
    p.L = L;
    p.P = L * (L + 1) / 2;
    p.k = k;
    p.level = level;
    p.rows = rows;
    p.width = width;
    p.hist = hist;
    p.hist_len = tg_global_len(L, k);
    p.off1 = tg_binom(L + 1, 2);
    p.off2 = p.off1 + tg_binom(L + 2, 3);
    p.off4 = p.off1 + 2 * tg_binom(L + 2, 3);
    p.n4 = tg_binom(L + 3, 4);
    p.work = work;
    const size_t avail = (size_t)smem_optin_e() - 1024;
    const size_t hist_bytes = ((size_t)p.hist_len * 8 + 15) & ~(size_t)15;
    const int hist_smem = (!rows && hist_bytes <= 48 * 1024) ? 1 : 0;
    // per warp: B, C, DT; the kernels that finish edges add the term table
    const size_t tbytes = ((size_t)3 * L2 * 8 + 15) & ~(size_t)15;
    const size_t xbytes = tbytes + (size_t)XT_N * L2 * 8;
    // B, C, DT through memory, in batches of work units whose sums fit in a
    // quarter of free memory; the fused kernel only when forced or when a
    // single unit would not fit
    const size_t row_bytes = (size_t)3 * L2 * 8;
    size_t free_b = 0, total_b = 0;
    TG_TRY_CUDA(cudaMemGetInfo(&free_b, &total_b));
    bool split = k == 4 && t.edge_pass != TG_EDGE_PASS_FUSED;
    int64_t qcap = std::min<int64_t>(count, (int64_t)(free_b / 4 / row_bytes));
    if (t.edge_batch > 0 && qcap > t.edge_batch) qcap = t.edge_batch;
    // batches [bu[x], bu[x + 1]) of units, with their heavy and light sub-lists
    std::vector<uint32_t> bu{0u, un.nunits}, bh{0u, un.nheavy}, bl{0u, un.nlight};
    if (split && qcap < count) {
        std::vector<uint32_t> us((size_t)un.nunits + 1), hv((size_t)un.nheavy), lv((size_t)un.nlight);
        TG_TRY_CUDA(cudaMemcpyAsync(us.data(), un.ustart.p, us.size() * 4, cudaMemcpyDeviceToHost, s));
        if (un.nheavy)
            TG_TRY_CUDA(cudaMemcpyAsync(hv.data(), un.heavy.p, hv.size() * 4, cudaMemcpyDeviceToHost, s));
        if (un.nlight)
            TG_TRY_CUDA(cudaMemcpyAsync(lv.data(), un.light.p, lv.size() * 4, cudaMemcpyDeviceToHost, s));
        TG_TRY_CUDA(cudaStreamSynchronize(s));
        bu.assign(1, 0u);
        for (uint32_t u0 = 0; u0 < un.nunits;) {
            uint32_t u1 = u0;
            while (u1 < un.nunits && (int64_t)us[u1 + 1] - us[u0] <= qcap) ++u1;
            if (u1 == u0) {  // one unit beyond the cap
                split = false;
                break;
            }
            bu.push_back(u1);
            u0 = u1;
        }
        if (split) {
            bh.clear();
            bl.clear();
            for (uint32_t x : bu) {
                bh.push_back((uint32_t)(std::lower_bound(hv.begin(), hv.end(), x) - hv.begin()));
                bl.push_back((uint32_t)(std::lower_bound(lv.begin(), lv.end(), x) - lv.begin()));
            }
        }
    }
    std::vector<uint32_t> ustart_h;
    if (split && bu.size() > 2) {
        ustart_h.resize(bu.size());
        for (size_t x = 0; x < bu.size(); ++x)
            TG_TRY_CUDA(cudaMemcpyAsync(&ustart_h[x], un.ustart.p + bu[x], 4, cudaMemcpyDeviceToHost, s));
        TG_TRY_CUDA(cudaStreamSynchronize(s));
    } else {
        ustart_h = {0u, (uint32_t)count};
    }
    int threads = t.cta_threads;
    if (threads > (split ? kTsumThreads : kEdgeMaxThreads)) threads = split ? kTsumThreads : kEdgeMaxThreads;
    if (threads < 32) threads = 32;
    p.hist_smem = split ? 0 : hist_smem;
    const size_t wbytes = split ? tbytes : xbytes;
    size_t fixed = (p.hist_smem ? hist_bytes : 0) + (size_t)(threads / 32) * wbytes + 16;
    while (fixed + 4096 > avail && threads > 32) {
        threads -= 32;
        fixed = (p.hist_smem ? hist_bytes : 0) + (size_t)(threads / 32) * wbytes + 16;
    }
    if (fixed + 16 > avail) return TG_EINVAL;
    int64_t nbits = k == 4 ? g->n_nonisolated : 0;
    if (t.bitmap_bits > 0 && nbits > t.bitmap_bits) nbits = t.bitmap_bits;
    const int64_t maxb = (int64_t)((avail - fixed) / 16) * 128;
    if (nbits > maxb) nbits = maxb;
    if (nbits < 0) nbits = 0;
    p.nbits = nbits;
    const size_t smem = fixed + ((((size_t)((nbits + 31) >> 5)) * 4 + 15) & ~(size_t)15);
    DevBuf<unsigned long long> queue, tsum;
    if (!queue.alloc(2, s)) return TG_ENOMEM;
    if (split && !tsum.alloc((size_t)(bu.size() > 2 ? qcap : count) * 3 * L2, s)) return TG_ENOMEM;
    p.tsum = tsum.p;
    const void *kfn = split ? (const void *)k_cyc_edge<true> : (const void *)k_cyc_edge<false>;
    TG_TRY(tg_allow_max_smem(kfn));
    int per_sm = 0;
    TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, smem));
    if (per_sm < 1) per_sm = 1;
    const int64_t hgrid_max = (int64_t)num_sms_e() * per_sm;
    DevBuf<uint32_t> emap;
    if (!emap.alloc((size_t)std::max<int64_t>(1, std::min<int64_t>(hgrid_max, split ? un.nheavy : un.nunits) * nbits), s))
        return TG_ENOMEM;
    p.emap = emap.p;
    if (!split) {
        // fused: every unit one CTA, Gamma_j bitmap, edges finished in place
        TG_TRY_CUDA(cudaMemsetAsync(queue.p, 0, 8, s));
        p.queue = queue.p;
        p.ulist = nullptr;
        p.nunits = un.nunits;
        int64_t grid = std::min<int64_t>(hgrid_max, p.nunits);
        if (t.grid_limit > 0 && grid > t.grid_limit) grid = t.grid_limit;
        if (grid < 1) grid = 1;
        k_cyc_edge<false><<<(unsigned)grid, threads, smem, s>>>(p);
        tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
        return TG_OK;
    }
    const size_t lw = (((size_t)3 * L2 * 8 + 15) & ~(size_t)15) + (size_t)2 * 4 * (1 << TG_LIGHT_LG);
    const size_t lsmem = (size_t)kTsumLightWarps * lw;
    TG_TRY(tg_allow_max_smem((const void *)k_cyc_tsum_light));
    int lper = 0;
    TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lper, k_cyc_tsum_light,
                                                              kTsumLightWarps * 32, lsmem));
    if (lper < 1) lper = 1;
    const size_t fsmem = (hist_smem ? hist_bytes : 0) + (256 / 32) * xbytes;
    TG_TRY(tg_allow_max_smem((const void *)k_cyc_finish));
    int fper = 0;
    TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fper, k_cyc_finish, 256, fsmem));
    if (fper < 1) fper = 1;
    for (size_t x = 0; x + 1 < bu.size(); ++x) {
        p.qbase = ustart_h[x];
        const int64_t nq = (int64_t)ustart_h[x + 1] - ustart_h[x];
        if (nq <= 0) continue;
        // heavy units: one CTA each, Gamma_j bitmap; B, C, DT to memory
        EdgeParams hp = p;
        hp.hist_smem = 0;
        hp.ulist = un.heavy.p + bh[x];
        hp.nunits = bh[x + 1] - bh[x];
        if (hp.nunits > 0) {
            TG_TRY_CUDA(cudaMemsetAsync(queue.p, 0, 8, s));
            hp.queue = queue.p;
            int64_t grid = std::min<int64_t>(hgrid_max, hp.nunits);
            if (t.grid_limit > 0 && grid > t.grid_limit) grid = t.grid_limit;
            if (grid < 1) grid = 1;
            k_cyc_edge<true><<<(unsigned)grid, threads, smem, s>>>(hp);
            tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
        }
        // light units: one warp each, Gamma_j in a per-warp hash map
        EdgeParams lp = p;
        lp.hist_smem = 0;
        lp.ulist = un.light.p + bl[x];
        lp.nunits = bl[x + 1] - bl[x];
        if (lp.nunits > 0) {
            TG_TRY_CUDA(cudaMemsetAsync(queue.p + 1, 0, 8, s));
            lp.queue = queue.p + 1;
            int64_t lgrid = (int64_t)num_sms_e() * lper;
            const int64_t need = ((int64_t)lp.nunits + kTsumLightWarps - 1) / kTsumLightWarps;
            if (lgrid > need) lgrid = need;
            if (t.grid_limit > 0 && lgrid > t.grid_limit) lgrid = t.grid_limit;
            k_cyc_tsum_light<<<(unsigned)lgrid, kTsumLightWarps * 32, lsmem, s>>>(lp); tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
        }
        // finishing pass: warp per edge
        EdgeParams fp = p;
        fp.hist_smem = hist_smem;
        int64_t fgrid = (int64_t)num_sms_e() * fper;
        if (fgrid > (nq + 7) / 8) fgrid = (nq + 7) / 8;
        if (t.grid_limit > 0 && fgrid > t.grid_limit) fgrid = t.grid_limit;
        if (fgrid < 1) fgrid = 1;
        k_cyc_finish<<<(unsigned)fgrid, 256, fsmem, s>>>(fp, nq); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    return TG_OK;
}
