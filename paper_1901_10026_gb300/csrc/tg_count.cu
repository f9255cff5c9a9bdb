// Per-edge typed graphlet counting (Alg. 1-3, the closed forms of Sec.
// "Combinatorial Relationships", Sec. "From Typed Orbits to Graphlets") and
// the global reduction of Sec. "Global Typed Graphlet Counts".
//
// One warp owns one edge (i, j) at a time; i is the endpoint with the larger
// new id, so d_i <= d_j.
//   Phase A/B (Alg. 1): classify Gamma_i \ {j} into T_ij / S_i and
//     Gamma_j \ {i} into T_ij / S_j, counting |T^t|, |S_i^t|, |S_j^t|.
//   Phase C (Alg. 2 and 3): for every w_k in S_i u S_j u T_ij and every w_r
//     in Gamma_{w_k}, classify w_r and update the enumerated orbits.  The
//     unmarked case (w_r in I, orbits g3 and g8) is not touched per w_r:
//     each w_k adds its typed degree vector d_{w_k}^{t'} (minus the entries
//     for i and j) once, and every marked w_r subtracts one.  This is the
//     same count as the per-w_r increments of Alg. 2-3.
//   Phase D: closed forms per type pair t <= t', then either the per-edge
//     row or warp-aggregated updates of a per-CTA histogram indexed by the
//     colex rank of the sorted type multiset.
// Membership of a neighbour w in Gamma_i or Gamma_j is a binary search inside
// the typed range Gamma_i^{phi(w)} (lists are sorted by (type, id)).
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "tg_device.cuh"

namespace {

using namespace tgd;

constexpr int kWarps = 8;
constexpr int kBlock = kWarps * 32;

// enumerated-orbit counter rows (per warp)
enum { C_G3 = 0, C_G6 = 1, C_G7 = 2, C_G8 = 3, C_G10 = 4, C_G12 = 5, C_NUM = 6 };

struct CountParams {
    const int64_t *rowptr;
    const uint32_t *adj;
    const int32_t *toff;
    const uint8_t *ntype;
    const int2 *edges;
    const uint32_t *order;  // processing order (edge ids); NULL -> e0 + item
    int64_t e0;
    int64_t count;
    int32_t L, P, k, level;
    unsigned long long *queue;
    uint64_t *rows;  // per-edge output, row (e - e0)
    int64_t width;
    unsigned long long *hist;  // undivided global sums
    int64_t hist_len;
    int32_t hist_smem;
    int64_t off1, off2, off4, n4;
};

__device__ __forceinline__ void hist_add(const CountParams &p, unsigned long long *shist,
                                         int64_t x, unsigned long long v) {
    if (!v) return;
    if (p.hist_smem)
        atomicAdd(shist + x, v);
    else
        atomicAdd(p.hist + x, v);
}

__global__ void __launch_bounds__(kBlock) k_count_warp(CountParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = p.L, P = p.P;
    size_t hist_bytes = p.hist_smem ? (((size_t)p.hist_len * 8 + 15) & ~(size_t)15) : 0;
    size_t wbytes = ((size_t)C_NUM * P * 4 + 3 * 16 * 4 + 32 * 4 + 15) & ~(size_t)15;
    unsigned long long *shist = reinterpret_cast<unsigned long long *>(smem);
    unsigned char *wb = smem + hist_bytes + warp * wbytes;
    int *cnt = reinterpret_cast<int *>(wb);
    unsigned *Tn = reinterpret_cast<unsigned *>(wb + (size_t)C_NUM * P * 4);
    unsigned *Si = Tn + 16;
    unsigned *Sj = Si + 16;
    int *pos2owner = reinterpret_cast<int *>(Sj + 16);

    if (p.hist_smem) {
        for (int64_t x = threadIdx.x; x < p.hist_len; x += blockDim.x) shist[x] = 0;
        __syncthreads();
    }
    const int64_t *__restrict__ rowptr = p.rowptr;
    const uint32_t *__restrict__ adj = p.adj;
    const int32_t *__restrict__ toff = p.toff;

    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(p.queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= (unsigned long long)p.count) break;
        const int64_t e = p.order ? p.order[item] : p.e0 + (int64_t)item;

        const int2 ab = p.edges[e];
        const int j = ab.x < ab.y ? ab.x : ab.y;  // larger degree
        const int i = ab.x < ab.y ? ab.y : ab.x;
        const int ti = p.ntype[i], tj = p.ntype[j];
        const int64_t bi = rowptr[i], bj = rowptr[j];
        const int di = (int)(rowptr[i + 1] - bi), dj = (int)(rowptr[j + 1] - bj);
        const int32_t *toi = toff + (int64_t)i * (L + 1);
        const int32_t *toj = toff + (int64_t)j * (L + 1);

        for (int x = lane; x < C_NUM * P; x += 32) cnt[x] = 0;
        if (lane < 16) {
            Tn[lane] = 0;
            Si[lane] = 0;
            Sj[lane] = 0;
        }
        __syncwarp();

        // ---- Alg. 1: T_ij and S_i from Gamma_i, S_j from Gamma_j ----------
        for (int x = lane; x < di; x += 32) {
            uint32_t w = __ldg(adj + bi + x);
            if ((int)(w & TG_IDMASK) == j) continue;
            bool inJ = contains(adj, bj, toj, w);
            atomicAdd(inJ ? &Tn[w >> TG_TSHIFT] : &Si[w >> TG_TSHIFT], 1u);
        }
        for (int x = lane; x < dj; x += 32) {
            uint32_t w = __ldg(adj + bj + x);
            if ((int)(w & TG_IDMASK) == i) continue;
            if (!contains(adj, bi, toi, w)) atomicAdd(&Sj[w >> TG_TSHIFT], 1u);
        }
        __syncwarp();

        // ---- Alg. 2 and 3 ------------------------------------------------
        if (p.k == 4) {
            for (int side = 0; side < 2; ++side) {
                const int64_t sb = side == 0 ? bi : bj;
                const int sd = side == 0 ? di : dj;
                for (int c0 = 0; c0 < sd; c0 += 32) {
                    const int x = c0 + lane;
                    bool act = x < sd;
                    uint32_t wk = act ? __ldg(adj + sb + x) : 0u;
                    const int kid = (int)(wk & TG_IDMASK), kt = (int)(wk >> TG_TSHIFT);
                    int cls = CLS_I;
                    if (act) {
                        if (side == 0) {
                            if (kid == j)
                                act = false;
                            else
                                cls = contains(adj, bj, toj, wk) ? CLS_T : CLS_SI;
                        } else {
                            if (kid == i || contains(adj, bi, toi, wk))
                                act = false;  // T members are enumerated from Gamma_i
                            else
                                cls = CLS_SJ;
                        }
                    }
                    int64_t kb = 0;
                    int dk = 0;
                    if (act) {
                        kb = rowptr[kid];
                        dk = (int)(rowptr[kid + 1] - kb);
                        const int32_t *tk = toff + (int64_t)kid * (L + 1);
                        const int gI = cls == CLS_T ? C_G8 : C_G3;
                        for (int t2 = 0; t2 < L; ++t2) {
                            int c = __ldg(tk + t2 + 1) - __ldg(tk + t2);
                            if ((cls & 1) && t2 == ti) --c;  // w_r = i
                            if ((cls & 2) && t2 == tj) --c;  // w_r = j
                            if (c) atomicAdd(&cnt[gI * P + pair_index(L, kt, t2)], c);
                        }
                    }
                    // flattened walk over the (up to 32) lists Gamma_{w_k}
                    int incl = dk;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        int y = __shfl_up_sync(kFull, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const int excl = incl - dk;
                    const int total = __shfl_sync(kFull, incl, 31);
                    int carry = 0;
                    for (int base = 0; base < total; base += 32) {
                        const int srel = excl - base;
                        const bool starts = dk > 0 && srel >= 0 && srel < 32;
                        const unsigned smask = __reduce_or_sync(kFull, starts ? (1u << srel) : 0u);
                        if (starts) pos2owner[srel] = lane;
                        __syncwarp();
                        const unsigned below =
                            smask & (lane == 31 ? kFull : ((2u << lane) - 1u));
                        const int owner = below ? pos2owner[31 - __clz(below)] : carry;
                        carry = __shfl_sync(kFull, owner, 31);
                        __syncwarp();
                        const int64_t ob = __shfl_sync(kFull, kb, owner);
                        const int oex = __shfl_sync(kFull, excl, owner);
                        const int ocls = __shfl_sync(kFull, cls, owner);
                        const int okt = __shfl_sync(kFull, kt, owner);
                        const int okid = __shfl_sync(kFull, kid, owner);
                        const int pos = base + lane;
                        if (pos < total) {
                            const uint32_t wr = __ldg(adj + ob + (pos - oex));
                            const int rid = (int)(wr & TG_IDMASK);
                            if (rid != i && rid != j) {
                                const int rcls = (contains(adj, bi, toi, wr) ? 1 : 0) |
                                                 (contains(adj, bj, toj, wr) ? 2 : 0);
                                if (rcls != CLS_I) {
                                    const int pr = pair_index(L, okt, (int)(wr >> TG_TSHIFT));
                                    atomicAdd(&cnt[(ocls == CLS_T ? C_G8 : C_G3) * P + pr], -1);
                                    if (ocls == CLS_SI) {
                                        if (rcls == CLS_SI && rid < okid)
                                            atomicAdd(&cnt[C_G7 * P + pr], 1);
                                    } else if (ocls == CLS_SJ) {
                                        if (rcls == CLS_SJ && rid < okid)
                                            atomicAdd(&cnt[C_G7 * P + pr], 1);
                                        else if (rcls == CLS_SI)
                                            atomicAdd(&cnt[C_G6 * P + pr], 1);
                                    } else {
                                        if (rcls == CLS_T) {
                                            if (rid < okid) atomicAdd(&cnt[C_G12 * P + pr], 1);
                                        } else {
                                            atomicAdd(&cnt[C_G10 * P + pr], 1);
                                        }
                                    }
                                }
                            }
                        }
                    }
                }
            }
            __syncwarp();
        }

        // ---- closed forms and output --------------------------------------
        if (p.rows) {
            uint64_t *row = p.rows + (e - p.e0) * p.width;
            for (int t = lane; t < L; t += 32) {
                row[t] = (uint64_t)Si[t] + Sj[t];
                row[L + t] = Tn[t];
            }
        } else {
            if (lane == 0) {
                int a = ti, b = tj;
                sort2(a, b);
                hist_add(p, shist, (int64_t)a + (int64_t)(b + 1) * b / 2, 1ull);
            }
            for (int t = lane; t < L; t += 32) {
                int a = ti, b = tj, c = t;
                sort2(a, b);
                sort2(b, c);
                sort2(a, b);
                const int64_t r = colex3(a, b, c);
                hist_add(p, shist, p.off1 + r, (unsigned long long)Si[t] + Sj[t]);
                hist_add(p, shist, p.off2 + r, (unsigned long long)Tn[t]);
            }
        }
        if (p.k == 4) {
            for (int pr = lane; pr < P; pr += 32) {
                int t, u;
                unpair(L, pr, t, u);
                const uint64_t sit = Si[t], siu = Si[u], sjt = Sj[t], sju = Sj[u];
                const uint64_t tt = Tn[t], tu = Tn[u];
                const uint64_t g3 = (uint64_t)(int64_t)cnt[C_G3 * P + pr];
                const uint64_t g6 = (uint64_t)(int64_t)cnt[C_G6 * P + pr];
                const uint64_t g7 = (uint64_t)(int64_t)cnt[C_G7 * P + pr];
                const uint64_t g8 = (uint64_t)(int64_t)cnt[C_G8 * P + pr];
                const uint64_t g10 = (uint64_t)(int64_t)cnt[C_G10 * P + pr];
                const uint64_t g12 = (uint64_t)(int64_t)cnt[C_G12 * P + pr];
                uint64_t g4, g5, g9, g11;
                closed_forms(t == u, sit, siu, sjt, sju, tt, tu, g6, g7, g10, g12, g4, g5, g9, g11);
                if (p.rows) {
                    uint64_t *row = p.rows + (e - p.e0) * p.width + 2 * L;
                    if (p.level == TG_ORBIT) {
                        row[0 * P + pr] = g3;
                        row[1 * P + pr] = g4;
                        row[2 * P + pr] = g5;
                        row[3 * P + pr] = g6;
                        row[4 * P + pr] = g7;
                        row[5 * P + pr] = g8;
                        row[6 * P + pr] = g9;
                        row[7 * P + pr] = g10;
                        row[8 * P + pr] = g11;
                        row[9 * P + pr] = g12;
                    } else {
                        row[0 * P + pr] = g3 + g4;
                        row[1 * P + pr] = g5;
                        row[2 * P + pr] = g6;
                        row[3 * P + pr] = g7 + g8 + g9;
                        row[4 * P + pr] = g10 + g11;
                        row[5 * P + pr] = g12;
                    }
                } else {
                    const uint64_t h[6] = {g3 + g4, g5, g6, g7 + g8 + g9, g10 + g11, g12};
                    if (h[0] | h[1] | h[2] | h[3] | h[4] | h[5]) {
                        int a = ti, b = tj, c = t, d = u;
                        sort2(a, b);
                        sort2(c, d);
                        sort2(a, c);
                        sort2(b, d);
                        sort2(b, c);
                        const int64_t r = colex4(a, b, c, d);
#pragma unroll
                        for (int q = 0; q < 6; ++q)
                            hist_add(p, shist, p.off4 + q * p.n4 + r, h[q]);
                    }
                }
            }
        }
        __syncwarp();
    }

    if (p.hist_smem) {
        __syncthreads();
        for (int64_t x = threadIdx.x; x < p.hist_len; x += blockDim.x)
            if (shist[x]) atomicAdd(p.hist + x, shist[x]);
    }
}

// ---------------------------------------------------------------------------
// CTA-per-edge counter with the mark table Psi of Alg. 1 held as a bitmap in
// shared memory over node ids [0, nbits).  The edges arrive grouped by their
// high-degree endpoint j, so the bits of Gamma_j stay set while a CTA works
// through consecutive edges of the same j; per edge only Gamma_i \ {j} is
// OR-ed in (the old bit tells T_ij from S_i) and taken out again afterwards.
// A per-edge open-addressing hash of Gamma_i in shared memory resolves a set
// bit into S_i / T_ij (found) or S_j (not found).  Nodes with id >= nbits and
// lists too long for the hash fall back to the sorted-range binary search.
// The w_k lists are walked by all warps of the CTA: each warp takes chunks of
// 32 w_k, compacts the active ones and walks the concatenation of their
// lists 32 entries at a time (owner of a position = number of list starts
// at or before it).
// ---------------------------------------------------------------------------
struct CtaParams {
    int64_t nbits;  // bitmap covers node ids [0, nbits)
    int32_t hmax;   // hash slots available (power of two)
};

struct EdgeCtx {
    const uint32_t *adj;
    const uint32_t *bm;
    const uint32_t *hk;
    int64_t nbits;
    int64_t bi, bj;
    const int32_t *toi, *toj;
    int i, j, lg, hash_ok;
};

// class of a Gamma_i member w (!= j): CLS_T or CLS_SI
__device__ __forceinline__ int class_of_i_member(const EdgeCtx &c, uint32_t w) {
    if (c.hash_ok) return hlookup(c.hk, c.lg, w & TG_IDMASK);
    return contains(c.adj, c.bj, c.toj, w) ? CLS_T : CLS_SI;
}

// class of any node w != i, j relative to the edge
__device__ __forceinline__ int classify(const EdgeCtx &c, uint32_t w) {
    const uint32_t id = w & TG_IDMASK;
    if ((int64_t)id < c.nbits) {
        if (!bm_test(c.bm, id)) return CLS_I;
        int ci = c.hash_ok ? hlookup(c.hk, c.lg, id)
                           : (contains(c.adj, c.bi, c.toi, w)
                                  ? (contains(c.adj, c.bj, c.toj, w) ? CLS_T : CLS_SI)
                                  : 0);
        return ci ? ci : CLS_SJ;
    }
    int ci = c.hash_ok ? hlookup(c.hk, c.lg, id)
                       : (contains(c.adj, c.bi, c.toi, w)
                              ? (contains(c.adj, c.bj, c.toj, w) ? CLS_T : CLS_SI)
                              : 0);
    if (ci) return ci;
    return contains(c.adj, c.bj, c.toj, w) ? CLS_SJ : CLS_I;
}

__device__ __forceinline__ void record_marked(int *cnt, int P, int ocls, int okid, int pr,
                                              int rcls, int rid) {
    atomicAdd(&cnt[(ocls == CLS_T ? C_G8 : C_G3) * P + pr], -1);
    if (ocls == CLS_SI) {
        if (rcls == CLS_SI && rid < okid) atomicAdd(&cnt[C_G7 * P + pr], 1);
    } else if (ocls == CLS_SJ) {
        if (rcls == CLS_SJ && rid < okid)
            atomicAdd(&cnt[C_G7 * P + pr], 1);
        else if (rcls == CLS_SI)
            atomicAdd(&cnt[C_G6 * P + pr], 1);
    } else {
        if (rcls == CLS_T) {
            if (rid < okid) atomicAdd(&cnt[C_G12 * P + pr], 1);
        } else {
            atomicAdd(&cnt[C_G10 * P + pr], 1);
        }
    }
}

// Orbit row incremented by a marked pair (w_k of class ocls, w_r of class
// rcls, lower = w_r < w_k), or -1: Alg. 2 (g7 inside one S-set with the
// symmetry break, g6 from the S_j pass) and Alg. 3 (g12 inside T with the
// symmetry break, g10 from T to S_i u S_j).
__device__ __forceinline__ int marked_orbit(int ocls, int rcls, bool lower) {
    if (ocls == CLS_SI) return (rcls == CLS_SI && lower) ? C_G7 : -1;
    if (ocls == CLS_SJ) {
        if (rcls == CLS_SJ) return lower ? C_G7 : -1;
        return rcls == CLS_SI ? C_G6 : -1;
    }
    if (rcls == CLS_T) return lower ? C_G12 : -1;
    return C_G10;
}

template <int U>
__global__ void __launch_bounds__(1024, 1) k_count_cta(CountParams p, CtaParams cp) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int L = p.L, P = p.P;
    const unsigned lanemask_le = lane == 31 ? kFull : ((2u << lane) - 1u);

    // shared-memory layout
    size_t off = 0;
    unsigned long long *shist = reinterpret_cast<unsigned long long *>(smem);
    if (p.hist_smem) off += ((size_t)p.hist_len * 8 + 15) & ~(size_t)15;
    const int64_t bwords = (cp.nbits + 31) >> 5;
    uint32_t *bm = reinterpret_cast<uint32_t *>(smem + off);
    off += (((size_t)bwords * 4) + 15) & ~(size_t)15;
    uint32_t *hk = reinterpret_cast<uint32_t *>(smem + off);
    off += (size_t)cp.hmax * 4;
    int *cnt_all = reinterpret_cast<int *>(smem + off);
    off += (((size_t)W * C_NUM * P * 4) + 15) & ~(size_t)15;
    unsigned *Tn = reinterpret_cast<unsigned *>(smem + off);
    unsigned *Si = Tn + 16;
    unsigned *Sj = Si + 16;
    unsigned long long *s_item = reinterpret_cast<unsigned long long *>(Sj + 16);
    int *cnt = cnt_all + warp * C_NUM * P;
    // per-warp staging of one chunk of w_k: 32 x (end, origin, entry, class)
    unsigned char *stage = smem + off + kMiscBytes + (size_t)warp * kStageBytes;
    int64_t *w_org = reinterpret_cast<int64_t *>(stage);
    int *w_end = reinterpret_cast<int *>(stage + 32 * 8);
    uint32_t *w_wk = reinterpret_cast<uint32_t *>(stage + 32 * 12);
    unsigned char *w_cls = stage + 32 * 16;

    for (int64_t x = tid; x < bwords; x += blockDim.x) bm[x] = 0u;
    for (int x = tid; x < cp.hmax; x += blockDim.x) hk[x] = kEmpty;
    if (p.hist_smem)
        for (int64_t x = tid; x < p.hist_len; x += blockDim.x) shist[x] = 0;

    const int64_t *__restrict__ rowptr = p.rowptr;
    const uint32_t *__restrict__ adj = p.adj;
    const int32_t *__restrict__ toff = p.toff;
    int cur_j = -1;
    int64_t cur_bj = 0;
    int cur_dj = 0;

    for (;;) {
        __syncthreads();
        if (tid == 0) *s_item = atomicAdd(p.queue, 1ull);
        __syncthreads();
        const unsigned long long item = *s_item;
        if (item >= (unsigned long long)p.count) break;
        const int64_t e = p.order ? p.order[item] : p.e0 + (int64_t)item;
        const int2 ab = p.edges[e];
        const int j = ab.x < ab.y ? ab.x : ab.y;
        const int i = ab.x < ab.y ? ab.y : ab.x;
        const int ti = p.ntype[i], tj = p.ntype[j];
        const int64_t bi = rowptr[i], bj = rowptr[j];
        const int di = (int)(rowptr[i + 1] - bi), dj = (int)(rowptr[j + 1] - bj);
        const int32_t *toi = toff + (int64_t)i * (L + 1);
        const int32_t *toj = toff + (int64_t)j * (L + 1);

        if (j != cur_j) {
            for (int x = tid; x < cur_dj; x += blockDim.x) {
                uint32_t id = __ldg(adj + cur_bj + x) & TG_IDMASK;
                if ((int64_t)id < cp.nbits) atomicAnd(&bm[id >> 5], ~(1u << (id & 31u)));
            }
            __syncthreads();
            for (int x = tid; x < dj; x += blockDim.x) {
                uint32_t id = __ldg(adj + bj + x) & TG_IDMASK;
                if ((int64_t)id < cp.nbits) atomicOr(&bm[id >> 5], 1u << (id & 31u));
            }
            cur_j = j;
            cur_bj = bj;
            cur_dj = dj;
        }
        for (int x = tid; x < W * C_NUM * P; x += blockDim.x) cnt_all[x] = 0;
        if (tid < 48) Tn[tid] = 0;
        int lg = 5;
        while ((1 << lg) < 2 * di) ++lg;
        const int hash_ok = (1 << lg) <= cp.hmax;
        __syncthreads();

        // ---- Alg. 1 on the bitmap: T_ij / S_i, marks for S_i -------------
        for (int x = tid; x < di; x += blockDim.x) {
            const uint32_t w = __ldg(adj + bi + x);
            const uint32_t id = w & TG_IDMASK;
            if ((int)id == j) continue;
            bool inJ;
            if ((int64_t)id < cp.nbits) {
                const uint32_t b = 1u << (id & 31u);
                inJ = (atomicOr(&bm[id >> 5], b) & b) != 0u;
            } else {
                inJ = contains(adj, bj, toj, w);
            }
            atomicAdd(inJ ? &Tn[w >> TG_TSHIFT] : &Si[w >> TG_TSHIFT], 1u);
            if (hash_ok) hinsert(hk, lg, id, inJ ? CLS_T : CLS_SI);
        }
        __syncthreads();
        if (tid < L) Sj[tid] = (unsigned)(__ldg(toj + tid + 1) - __ldg(toj + tid)) - Tn[tid] -
                               (tid == ti ? 1u : 0u);

        EdgeCtx c;
        c.adj = adj;
        c.bm = bm;
        c.hk = hk;
        c.nbits = cp.nbits;
        c.bi = bi;
        c.bj = bj;
        c.toi = toi;
        c.toj = toj;
        c.i = i;
        c.j = j;
        c.lg = lg;
        c.hash_ok = hash_ok;

        // ---- Alg. 2 and 3 -------------------------------------------------
        if (p.k == 4) {
            const int nch = (di + dj + 31) >> 5;
            for (int ch = warp; ch < nch; ch += W) {
                const int x = ch * 32 + lane;
                bool act = false;
                uint32_t wk = 0;
                int cls = CLS_I;
                if (x < di) {
                    wk = __ldg(adj + bi + x);
                    if ((int)(wk & TG_IDMASK) != j) {
                        act = true;
                        cls = class_of_i_member(c, wk);
                    }
                } else if (x < di + dj) {
                    wk = __ldg(adj + bj + (x - di));
                    const int kid = (int)(wk & TG_IDMASK);
                    if (kid != i) {
                        const int ci = hash_ok ? hlookup(hk, lg, (uint32_t)kid)
                                               : (contains(adj, bi, toi, wk) ? CLS_T : 0);
                        if (!ci) {
                            act = true;
                            cls = CLS_SJ;
                        }
                    }
                }
                int64_t kb = 0;
                int dk = 0;
                const int kid0 = (int)(wk & TG_IDMASK), kt0 = (int)(wk >> TG_TSHIFT);
                const int gI0 = cls == CLS_T ? C_G8 : C_G3;
                const int32_t *tk = toff + (int64_t)kid0 * (L + 1);
                if (act) {
                    kb = rowptr[kid0];
                    dk = (int)(rowptr[kid0 + 1] - kb);
                }
                // typed degree vector of w_k (minus i and j) into g3 / g8,
                // summed over the lanes that share (orbit, type of w_k)
                {
                    const int dkey = act ? (gI0 * 16 + kt0) : -1;
                    const unsigned dm = __match_any_sync(kFull, dkey);
                    const bool dlead = act && lane == __ffs(dm) - 1;
                    int prev = act ? __ldg(tk) : 0;
                    for (int t2 = 0; t2 < L; ++t2) {
                        int cc = 0;
                        if (act) {
                            const int nx = __ldg(tk + t2 + 1);
                            cc = nx - prev;
                            prev = nx;
                            if ((cls & 1) && t2 == ti) --cc;
                            if ((cls & 2) && t2 == tj) --cc;
                        }
                        const int sum = __reduce_add_sync(dm, cc);
                        if (dlead && sum) atomicAdd(&cnt[gI0 * P + pair_index(L, kt0, t2)], sum);
                    }
                }
                // Stage the active w_k of this chunk (in lane order) in the
                // warp's shared-memory slots: segment end in the flattened
                // walk, list origin, packed entry and class.  The walk below
                // then needs no warp-synchronous intrinsics.
                const unsigned am = __ballot_sync(kFull, act);
                const int na = __popc(am);
                if (na == 0) continue;
                int incl = act ? dk : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                const int total = __shfl_sync(kFull, incl, 31);
                if (act) {
                    const int r = __popc(am & ((1u << lane) - 1u));
                    w_end[r] = incl;
                    w_org[r] = kb - (incl - dk);
                    w_wk[r] = wk;
                    w_cls[r] = (unsigned char)cls;
                }
                __syncwarp();
                for (int base = 0; base < total; base += 32 * U) {
                    uint32_t wr[U], owk[U];
                    int ocl[U];
                    bool val[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int pos = base + 32 * u + lane;
                        val[u] = pos < total;
                        wr[u] = 0u;
                        owk[u] = 0u;
                        ocl[u] = 0;
                        if (val[u]) {
                            // owner: first staged segment whose end exceeds pos
                            int lo = 0, hi = na - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (w_end[mid] > pos)
                                    hi = mid;
                                else
                                    lo = mid + 1;
                            }
                            owk[u] = w_wk[lo];
                            ocl[u] = w_cls[lo];
                            wr[u] = __ldg(adj + (w_org[lo] + pos));
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        // counter updates of this position: key1 gets -1
                        // (g3 / g8 correction), key2 gets +1 (g6, g7, g10 or
                        // g12); -1 means none
                        int key1 = -1, key2 = -1;
                        if (val[u]) {
                            const int rid = (int)(wr[u] & TG_IDMASK);
                            if (rid != i && rid != j) {
                                const int rcls = classify(c, wr[u]);
                                if (rcls != CLS_I) {
                                    const int pr = pair_index(L, (int)(owk[u] >> TG_TSHIFT),
                                                              (int)(wr[u] >> TG_TSHIFT));
                                    key1 = (ocl[u] == CLS_T ? C_G8 : C_G3) * P + pr;
                                    const int row =
                                        marked_orbit(ocl[u], rcls, rid < (int)(owk[u] & TG_IDMASK));
                                    if (row >= 0) key2 = row * P + pr;
                                }
                            }
                        }
                        const unsigned m1 = __match_any_sync(kFull, key1);
                        if (key1 >= 0 && lane == __ffs(m1) - 1) atomicAdd(&cnt[key1], -__popc(m1));
                        const unsigned m2 = __match_any_sync(kFull, key2);
                        if (key2 >= 0 && lane == __ffs(m2) - 1) atomicAdd(&cnt[key2], __popc(m2));
                    }
                }
                __syncwarp();  // the slots are rewritten by the next chunk
            }
        }
        __syncthreads();
        // reduce the per-warp counters into warp 0's block
        for (int x = tid; x < C_NUM * P; x += blockDim.x) {
            int sacc = 0;
            for (int w = 0; w < W; ++w) sacc += cnt_all[w * C_NUM * P + x];
            cnt_all[x] = sacc;
        }
        __syncthreads();

        // ---- closed forms and output --------------------------------------
        if (p.rows) {
            uint64_t *row = p.rows + (e - p.e0) * p.width;
            for (int t = tid; t < L; t += blockDim.x) {
                row[t] = (uint64_t)Si[t] + Sj[t];
                row[L + t] = Tn[t];
            }
        } else {
            if (tid == 0) {
                int a = ti, b = tj;
                sort2(a, b);
                hist_add(p, shist, (int64_t)a + (int64_t)(b + 1) * b / 2, 1ull);
            }
            for (int t = tid; t < L; t += blockDim.x) {
                int a = ti, b = tj, cc = t;
                sort2(a, b);
                sort2(b, cc);
                sort2(a, b);
                const int64_t r = colex3(a, b, cc);
                hist_add(p, shist, p.off1 + r, (unsigned long long)Si[t] + Sj[t]);
                hist_add(p, shist, p.off2 + r, (unsigned long long)Tn[t]);
            }
        }
        if (p.k == 4) {
            for (int pr = tid; pr < P; pr += blockDim.x) {
                int t, u;
                unpair(L, pr, t, u);
                const uint64_t sit = Si[t], siu = Si[u], sjt = Sj[t], sju = Sj[u];
                const uint64_t tt = Tn[t], tu = Tn[u];
                const uint64_t g3 = (uint64_t)(int64_t)cnt_all[C_G3 * P + pr];
                const uint64_t g6 = (uint64_t)(int64_t)cnt_all[C_G6 * P + pr];
                const uint64_t g7 = (uint64_t)(int64_t)cnt_all[C_G7 * P + pr];
                const uint64_t g8 = (uint64_t)(int64_t)cnt_all[C_G8 * P + pr];
                const uint64_t g10 = (uint64_t)(int64_t)cnt_all[C_G10 * P + pr];
                const uint64_t g12 = (uint64_t)(int64_t)cnt_all[C_G12 * P + pr];
                uint64_t g4, g5, g9, g11;
                closed_forms(t == u, sit, siu, sjt, sju, tt, tu, g6, g7, g10, g12, g4, g5, g9, g11);
                if (p.rows) {
                    uint64_t *row = p.rows + (e - p.e0) * p.width + 2 * L;
                    if (p.level == TG_ORBIT) {
                        row[0 * P + pr] = g3;
                        row[1 * P + pr] = g4;
                        row[2 * P + pr] = g5;
                        row[3 * P + pr] = g6;
                        row[4 * P + pr] = g7;
                        row[5 * P + pr] = g8;
                        row[6 * P + pr] = g9;
                        row[7 * P + pr] = g10;
                        row[8 * P + pr] = g11;
                        row[9 * P + pr] = g12;
                    } else {
                        row[0 * P + pr] = g3 + g4;
                        row[1 * P + pr] = g5;
                        row[2 * P + pr] = g6;
                        row[3 * P + pr] = g7 + g8 + g9;
                        row[4 * P + pr] = g10 + g11;
                        row[5 * P + pr] = g12;
                    }
                } else {
                    const uint64_t h[6] = {g3 + g4, g5, g6, g7 + g8 + g9, g10 + g11, g12};
                    if (h[0] | h[1] | h[2] | h[3] | h[4] | h[5]) {
                        int a = ti, b = tj, cc = t, d = u;
                        sort2(a, b);
                        sort2(cc, d);
                        sort2(a, cc);
                        sort2(b, d);
                        sort2(b, cc);
                        const int64_t r = colex4(a, b, cc, d);
#pragma unroll
                        for (int q = 0; q < 6; ++q)
                            hist_add(p, shist, p.off4 + q * p.n4 + r, h[q]);
                    }
                }
            }
        }
        // ---- reset the marks of S_i and the hash ---------------------------
        for (int x = tid; x < di; x += blockDim.x) {
            const uint32_t w = __ldg(adj + bi + x);
            const uint32_t id = w & TG_IDMASK;
            if ((int)id == j || (int64_t)id >= cp.nbits) continue;
            if (class_of_i_member(c, w) == CLS_SI) atomicAnd(&bm[id >> 5], ~(1u << (id & 31u)));
        }
        __syncthreads();
        if (hash_ok)
            for (int x = tid; x < (1 << lg); x += blockDim.x) hk[x] = kEmpty;
    }

    if (p.hist_smem) {
        __syncthreads();
        for (int64_t x = tid; x < p.hist_len; x += blockDim.x)
            if (shist[x]) atomicAdd(p.hist + x, shist[x]);
    }
}

// |E(H)| per global entry: divide and check.
__global__ void k_finalize(const unsigned long long *sums, uint64_t *out, int64_t len,
                           int64_t off1, int64_t off2, int64_t off4, int64_t n4,
                           unsigned *err) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < len;
         x += (int64_t)gridDim.x * blockDim.x) {
        uint64_t d = 1;
        if (x >= off4) {
            const uint64_t eh[6] = {3, 3, 4, 4, 5, 6};
            d = eh[(x - off4) / n4];
        } else if (x >= off2) {
            d = 3;
        } else if (x >= off1) {
            d = 2;
        }
        uint64_t v = sums[x];
        if (v % d) atomicOr(err, TG_DERR_DIVISIBLE);
        out[x] = v / d;
    }
}

// s_v = sum of neighbour degrees (for the work model and the schedule).
__global__ void k_neighbor_degree_sum(const int64_t *rowptr, const uint32_t *adj, int64_t n,
                                      unsigned long long *s) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = wid; v < n; v += nw) {
        unsigned long long acc = 0;
        for (int64_t x = rowptr[v] + lane; x < rowptr[v + 1]; x += 32) {
            uint32_t w = adj[x] & TG_IDMASK;
            acc += (unsigned long long)(rowptr[w + 1] - rowptr[w]);
        }
        for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
        if (lane == 0) s[v] = acc;
    }
}

// Paper work model per edge: 2 d_i + d_j + sum_{w in S_i u S_j u T} d_w.
__global__ void k_work_model(const int64_t *rowptr, const uint32_t *adj, const int32_t *toff,
                             const int2 *edges, int64_t M, int32_t L,
                             const unsigned long long *s, unsigned long long *total,
                             unsigned long long *edge_cost) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long acc_total = 0;
    for (int64_t e = wid; e < M; e += nw) {
        const int2 ab = edges[e];
        const int j = ab.x < ab.y ? ab.x : ab.y;
        const int i = ab.x < ab.y ? ab.y : ab.x;
        const int64_t bi = rowptr[i], bj = rowptr[j];
        const int64_t di = rowptr[i + 1] - bi, dj = rowptr[j + 1] - bj;
        const int32_t *toj = toff + (int64_t)j * (L + 1);
        unsigned long long tsum = 0;
        for (int64_t x = lane; x < di; x += 32) {
            uint32_t w = adj[bi + x];
            int id = (int)(w & TG_IDMASK);
            if (id == j) continue;
            if (contains(adj, bj, toj, w)) tsum += (unsigned long long)(rowptr[id + 1] - rowptr[id]);
        }
        for (int o = 16; o; o >>= 1) tsum += __shfl_down_sync(kFull, tsum, o);
        if (lane == 0) {
            unsigned long long c = 2ull * di + dj + (s[i] - dj) + (s[j] - di) - tsum;
            if (edge_cost) edge_cost[e] = c;
            acc_total += c;
        }
    }
    if (lane == 0 && acc_total) atomicAdd(total, acc_total);
}

// Group key of an edge: (j, i) with j the high-degree endpoint (smaller new
// id), so the edges sharing j are contiguous and hubs come first.
__global__ void k_group_keys(const int2 *edges, int64_t e0, int64_t count, int nb, uint64_t *key,
                             uint32_t *val) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < count;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int2 ab = edges[e0 + x];
        const uint64_t j = (uint64_t)(ab.x < ab.y ? ab.x : ab.y);
        const uint64_t i = (uint64_t)(ab.x < ab.y ? ab.y : ab.x);
        key[x] = (j << nb) | i;
        val[x] = (uint32_t)(e0 + x);
    }
}

inline unsigned grid_for(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (unsigned)b;
}

}  // namespace

// ----------------------------------------------------------- schedule -----
// ------------------------------------------------------------- tuning -----
static std::mutex g_tune_mu;
static tg_tune g_tune = {TG_KERNEL_AUTO, 1024, 2, 4096, 0, 0, 0, 0, 0};

static tg_tune tune_now() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune;
}

extern "C" int tg_set_tune(const tg_tune *t) {
    tg_tune d = {TG_KERNEL_AUTO, 1024, 2, 4096, 0, 0, 0, 0, 0};
    if (t) {
        if (t->kernel < 0 || t->kernel > TG_KERNEL_CYCLES) return TG_EINVAL;
        if (t->cta_threads && (t->cta_threads < 32 || t->cta_threads > 1024 || t->cta_threads % 32))
            return TG_EINVAL;
        if (t->unroll && t->unroll != 1 && t->unroll != 2 && t->unroll != 4) return TG_EINVAL;
        if (t->hash_slots && (t->hash_slots < 32 || (t->hash_slots & (t->hash_slots - 1))))
            return TG_EINVAL;
        if (t->bitmap_bits < 0 || t->grid_limit < 0) return TG_EINVAL;
        if (t->edge_pass != TG_EDGE_PASS_AUTO && t->edge_pass != TG_EDGE_PASS_FUSED)
            return TG_EINVAL;
        if (t->edge_batch < 0) return TG_EINVAL;
        if (t->c4_bin_fill < 0 || t->c4_bin_fill > (1 << 20)) return TG_EINVAL;
        d.kernel = t->kernel;
        if (t->cta_threads) d.cta_threads = t->cta_threads;
        if (t->unroll) d.unroll = t->unroll;
        if (t->hash_slots) d.hash_slots = t->hash_slots;
        d.bitmap_bits = t->bitmap_bits;
        d.grid_limit = t->grid_limit;
        d.edge_pass = t->edge_pass;
        d.edge_batch = t->edge_batch;
        d.c4_bin_fill = t->c4_bin_fill;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune = d;
    return TG_OK;
}

extern "C" int tg_get_tune(tg_tune *t) {
    if (!t) return TG_EINVAL;
    *t = tune_now();
    return TG_OK;
}

// ---------------------------------------------------------- autotune -----
static int check_counts(const tg_graph *g, int k);

namespace {
struct TuneKey {
    int device, L, k, mbits, dbits;
    bool operator<(const TuneKey &o) const {
        return std::tie(device, L, k, mbits, dbits) < std::tie(o.device, o.L, o.k, o.mbits, o.dbits);
    }
};
std::mutex g_autotune_mu;
std::map<TuneKey, tg_tune> g_autotune_cache;

int bitlen(int64_t x) {
    int b = 0;
    while (x > 0) ++b, x >>= 1;
    return b;
}
}  // namespace

extern "C" int tg_autotune_reset(void) {
    std::lock_guard<std::mutex> lk(g_autotune_mu);
    g_autotune_cache.clear();
    return TG_OK;
}

extern "C" int tg_autotune(const tg_graph *g, int32_t k, tg_tune *best, void *stream) {
    TG_TRY(check_counts(g, k));
    const TuneKey key{g->device, g->L, k, bitlen(g->M), bitlen(g->max_degree)};
    {
        std::lock_guard<std::mutex> lk(g_autotune_mu);
        auto it = g_autotune_cache.find(key);
        if (it != g_autotune_cache.end()) {
            TG_TRY(tg_set_tune(&it->second));
            if (best) *best = it->second;
            return TG_OK;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const tg_tune before = tune_now();
    DevBuf<uint64_t> out;
    if (!out.alloc(tg_global_len(g->L, k), s)) return TG_ENOMEM;
    cudaEvent_t ev[2];
    TG_TRY_CUDA(cudaEventCreate(&ev[0]));
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return TG_ECUDA;
    }
    // one count under candidate c, in milliseconds
    auto timed = [&](const tg_tune &c, float &ms) -> int {
        TG_TRY(tg_set_tune(&c));
        TG_TRY_CUDA(cudaEventRecord(ev[0], s));
        TG_TRY(tg_count_global(g, k, out.p, s));
        TG_TRY_CUDA(cudaEventRecord(ev[1], s));
        TG_TRY_CUDA(cudaEventSynchronize(ev[1]));
        TG_TRY_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        return TG_OK;
    };
    tg_tune cur = before;
    cur.kernel = TG_KERNEL_CYCLES;
    float cur_ms = 0.f;
    int rc = timed(cur, cur_ms);  // warm-up: schedule, pools, module loads
    if (rc == TG_OK) rc = timed(cur, cur_ms);
    struct Dim {
        int32_t tg_tune::*field;
        std::vector<int32_t> values;
        bool k4_only;
    };
    const Dim dims[] = {{&tg_tune::unroll, {2, 4}, false},
                        {&tg_tune::c4_bin_fill, {8, 32, 128}, true},
                        {&tg_tune::edge_pass, {TG_EDGE_PASS_AUTO, TG_EDGE_PASS_FUSED}, true},
                        {&tg_tune::hash_slots, {4096, 32}, false}};
    for (const Dim &d : dims) {
        if (rc != TG_OK || (d.k4_only && k != 4)) continue;
        tg_tune base = cur;
        for (int32_t v : d.values) {
            if (rc != TG_OK) break;
            // c4_bin_fill 0 means 32: do not time the default twice
            const int32_t now = (d.field == &tg_tune::c4_bin_fill && base.*d.field == 0) ? 32 : base.*d.field;
            if (v == now) continue;
            tg_tune c = base;
            c.*d.field = v;
            float ms = 0.f;
            rc = timed(c, ms);
            if (rc == TG_OK && ms < 0.98f * cur_ms) cur = c, cur_ms = ms;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc != TG_OK) {
        tg_set_tune(&before);
        return rc;
    }
    TG_TRY(tg_set_tune(&cur));
    {
        std::lock_guard<std::mutex> lk(g_autotune_mu);
        g_autotune_cache[key] = cur;
    }
    if (best) *best = cur;
    return TG_OK;
}

// ----------------------------------------------------------- schedule -----
struct tg_sched {
    uint32_t *order = nullptr;          // M edge ids grouped by high-degree endpoint
    unsigned long long *s = nullptr;    // n neighbour-degree sums
    int64_t M = 0, n = 0;
};

void tg_sched_free(tg_graph *g) {
    if (!g->sched) return;
    (void)cudaDeviceSynchronize();
    tg_dfree(g->sched->order, 0, nullptr);
    tg_dfree(g->sched->s, 0, nullptr);
    (void)cudaDeviceSynchronize();
    delete g->sched;
    g->sched = nullptr;
}

void tg_sched_free_on(tg_graph *g, cudaStream_t s) {
    if (!g->sched) return;
    tg_dfree(g->sched->order, 0, s);
    tg_dfree(g->sched->s, 0, s);
    delete g->sched;
    g->sched = nullptr;
}

// Edge ids [e0, e0 + count) sorted by (j, i); *out owns count entries.
static int grouped_order(const tg_graph *g, int64_t e0, int64_t count, cudaStream_t s,
                         DevBuf<uint32_t> &out) {
    if (!out.alloc(count > 0 ? count : 1, s)) return TG_ENOMEM;
    if (count <= 0) return TG_OK;
    DevBuf<uint64_t> k1, k2;
    DevBuf<uint32_t> v2;
    if (!k1.alloc(count, s) || !k2.alloc(count, s) || !v2.alloc(count, s)) return TG_ENOMEM;
    const int nb = tg_bitlen((uint64_t)(g->n > 1 ? g->n - 1 : 1));
    k_group_keys<<<grid_for(count), 256, 0, s>>>(g->edges, e0, count, nb, k1.p, out.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    uint64_t *rk = nullptr;
    uint32_t *rv = nullptr;
    TG_TRY(tg_radix_sort_kv(k1.p, k2.p, out.p, v2.p, count, 2 * nb, s, &rk, &rv));
    if (rv != out.p) TG_TRY_CUDA(cudaMemcpyAsync(out.p, rv, count * 4, cudaMemcpyDeviceToDevice, s));
    return TG_OK;
}

static int get_sched(const tg_graph *g, cudaStream_t s, tg_sched **out) {
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->sched) {
        *out = g->sched;
        return TG_OK;
    }
    DevBuf<uint32_t> order;
    TG_TRY(grouped_order(g, 0, g->M, s, order));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    tg_sched *sc = new (std::nothrow) tg_sched();
    if (!sc) return TG_ENOMEM;
    sc->M = g->M;
    sc->n = g->n;
    sc->order = order.release();
    g->sched = sc;
    *out = sc;
    return TG_OK;
}

// The neighbour-degree sums of the schedule, made on first use (only the
// work model reads them).
static int sched_sums(const tg_graph *g, tg_sched *sc, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g->mu);
    if (sc->s) return TG_OK;
    DevBuf<unsigned long long> sv;
    if (!sv.alloc(g->n, s)) return TG_ENOMEM;
    k_neighbor_degree_sum<<<grid_for(g->n * 32), 256, 0, s>>>(g->rowptr, g->adj, g->n, sv.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    sc->s = sv.release();
    return TG_OK;
}

// ------------------------------------------------------------ launches ----

static int max_smem_optin() {
    int dev = 0, v = 0;
    (void)cudaGetDevice(&dev);
    (void)cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v > 0 ? v : 48 * 1024;
}

static size_t warp_smem_bytes(int P) {
    return ((size_t)C_NUM * P * 4 + 3 * 16 * 4 + 32 * 4 + 15) & ~(size_t)15;
}

static void fill_params(CountParams &p, const tg_graph *g, int k, int level,
                        const uint32_t *order, int64_t e0, int64_t count, uint64_t *rows,
                        int64_t width, unsigned long long *hist, unsigned long long *queue) {
    const int L = g->L;
    p = CountParams{};
    p.rowptr = g->rowptr;
    p.adj = g->adj;
    p.toff = g->toff;
    p.ntype = g->ntype;
    p.edges = g->edges;
    p.order = order;
    p.e0 = e0;
    p.count = count;
    p.L = L;
    p.P = L * (L + 1) / 2;
    p.k = k;
    p.level = level;
    p.queue = queue;
    p.rows = rows;
    p.width = width;
    p.hist = hist;
    p.hist_len = tg_global_len(L, k);
    p.off1 = tg_binom(L + 1, 2);
    p.off2 = p.off1 + tg_binom(L + 2, 3);
    p.off4 = p.off1 + 2 * tg_binom(L + 2, 3);
    p.n4 = tg_binom(L + 3, 4);
    const size_t hist_bytes = ((size_t)p.hist_len * 8 + 15) & ~(size_t)15;
    p.hist_smem = (!rows && hist_bytes <= 48 * 1024) ? 1 : 0;
}

static int launch_warp(const CountParams &p, cudaStream_t s) {
    const size_t hist_bytes = p.hist_smem ? (((size_t)p.hist_len * 8 + 15) & ~(size_t)15) : 0;
    const size_t smem = hist_bytes + kWarps * warp_smem_bytes(p.P);
    TG_TRY(tg_allow_max_smem((const void *)k_count_warp));
    int per_sm = 0;
    TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_warp, kBlock, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)tg_num_sms() * per_sm;
    const int64_t need = (p.count + kWarps - 1) / kWarps;
    if (grid > need) grid = need;
    const int gl = tune_now().grid_limit;
    if (gl > 0 && grid > gl) grid = gl;
    k_count_warp<<<(unsigned)grid, kBlock, smem, s>>>(p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    return TG_OK;
}

// Shared-memory plan of the CTA kernel; false if even a minimal plan does not fit.
static bool plan_cta(const tg_graph *g, const CountParams &p, const tg_tune &t, int threads,
                     CtaParams &cp, size_t &smem) {
    const int W = threads / 32;
    const size_t hist_bytes = p.hist_smem ? (((size_t)p.hist_len * 8 + 15) & ~(size_t)15) : 0;
    const size_t cnt_bytes = (((size_t)W * C_NUM * p.P * 4) + 15) & ~(size_t)15;
    const size_t misc = kMiscBytes + (size_t)W * kStageBytes;
    int hmax = t.hash_slots;
    const size_t avail = (size_t)max_smem_optin();
    size_t fixed = hist_bytes + cnt_bytes + misc + (size_t)hmax * 4;
    while (fixed + 4096 > avail && hmax > 32) {
        hmax >>= 1;
        fixed = hist_bytes + cnt_bytes + misc + (size_t)hmax * 4;
    }
    if (fixed + 16 > avail) return false;
    int64_t bits = g->n_nonisolated;
    if (t.bitmap_bits > 0 && bits > t.bitmap_bits) bits = t.bitmap_bits;
    const int64_t max_bits = (int64_t)((avail - fixed - 16) / 16) * 128;  // 16-byte granules
    if (bits > max_bits) bits = max_bits;
    if (bits < 0) bits = 0;
    cp.nbits = bits;
    cp.hmax = hmax;
    smem = hist_bytes + ((((size_t)((bits + 31) >> 5)) * 4 + 15) & ~(size_t)15) + (size_t)hmax * 4 +
           cnt_bytes + misc;
    return true;
}

template <int U>
static int launch_cta_u(const CountParams &p, const CtaParams &cp, int threads, size_t smem,
                        cudaStream_t s) {
    TG_TRY(tg_allow_max_smem((const void *)k_count_cta<U>));
    int per_sm = 0;
    TG_TRY_CUDA(
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_cta<U>, threads, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)tg_num_sms() * per_sm;
    if (grid > p.count) grid = p.count;
    const int gl = tune_now().grid_limit;
    if (gl > 0 && grid > gl) grid = gl;
    k_count_cta<U><<<(unsigned)grid, threads, smem, s>>>(p, cp); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    return TG_OK;
}

// Launch the counting kernel over `count` edges (order[item] or e0 + item);
// full_order is the grouped order of the whole graph.
static int launch_count(const tg_graph *g, int k, int level, const uint32_t *full_order,
                        const uint32_t *order, int64_t e0, int64_t count, uint64_t *rows,
                        int64_t width, unsigned long long *hist, cudaStream_t s) {
    if (count <= 0) return TG_OK;
    {
        const tg_tune t0 = tune_now();
        if ((t0.kernel == TG_KERNEL_AUTO || t0.kernel == TG_KERNEL_REUSE ||
             t0.kernel == TG_KERNEL_CYCLES) &&
            order)
            return tg_reuse_count(g, k, level, full_order, order, count, rows, width, hist, t0, s);
    }
    DevBuf<unsigned long long> queue;
    if (!queue.alloc(1, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(queue.p, 0, 8, s));
    CountParams p;
    fill_params(p, g, k, level, order, e0, count, rows, width, hist, queue.p);
    const tg_tune t = tune_now();
    if (t.kernel == TG_KERNEL_WARP_SEARCH) return launch_warp(p, s);
    CtaParams cp;
    size_t smem = 0;
    const int threads = t.cta_threads;
    if (!plan_cta(g, p, t, threads, cp, smem)) return launch_warp(p, s);
    switch (t.unroll) {
        case 1: return launch_cta_u<1>(p, cp, threads, smem, s);
        case 4: return launch_cta_u<4>(p, cp, threads, smem, s);
        default: return launch_cta_u<2>(p, cp, threads, smem, s);
    }
}

static int check_counts(const tg_graph *g, int k) {
    if (!g) return TG_EINVAL;
    if (k != 3 && k != 4) return TG_EINVAL;
    // 32-bit per-edge enumerated counters: every one is bounded by 2M; the
    // flattened walk indexes up to 32 * Delta entries.
    if (2 * g->M >= ((int64_t)1 << 31) || 32 * g->max_degree >= ((int64_t)1 << 31))
        return TG_EOVERFLOW;
    return TG_OK;
}

static int sums_impl(const tg_graph *g, int k, int64_t e0, int64_t e1,
                     unsigned long long *dsums, cudaStream_t s) {
    const int64_t len = tg_global_len(g->L, k);
    TG_TRY_CUDA(cudaMemsetAsync(dsums, 0, len * 8, s));
    tg_sched *sc = nullptr;
    TG_TRY(get_sched(g, s, &sc));
    if (e0 == 0 && e1 == g->M)
        return launch_count(g, k, TG_GRAPHLET, sc->order, sc->order, 0, g->M, nullptr, 0, dsums,
                            s);
    DevBuf<uint32_t> order;
    TG_TRY(grouped_order(g, e0, e1 - e0, s, order));
    return launch_count(g, k, TG_GRAPHLET, sc->order, order.p, 0, e1 - e0, nullptr, 0, dsums, s);
}
extern "C" int tg_count_global(const tg_graph *g, int32_t k, uint64_t *out, void *stream) {
    TG_TRY(check_counts(g, k));
    if (!out) return TG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int L = g->L;
    const int64_t len = tg_global_len(L, k);
    DevBuf<unsigned long long> sums;
    DevBuf<unsigned> err;
    if (!sums.alloc(len, s) || !err.alloc(1, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(err.p, 0, 4, s));
    TG_TRY(sums_impl(g, k, 0, g->M, sums.p, s));
    const bool dev_out = tg_is_device_ptr(out);
    DevBuf<uint64_t> tmp;
    uint64_t *dst = out;
    if (!dev_out) {
        if (!tmp.alloc(len, s)) return TG_ENOMEM;
        dst = tmp.p;
    }
    const int64_t off1 = tg_binom(L + 1, 2), n3 = tg_binom(L + 2, 3);
    k_finalize<<<grid_for(len), 256, 0, s>>>(sums.p, dst, len, off1, off1 + n3, off1 + 2 * n3,
                                             tg_binom(L + 3, 4), err.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    unsigned herr = 0;
    TG_TRY_CUDA(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, s));
    if (!dev_out) TG_TRY_CUDA(cudaMemcpyAsync(out, dst, len * 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    if (herr) return TG_EINTERNAL;
    return TG_OK;
}

extern "C" int tg_count_range(const tg_graph *g, int32_t k, int64_t e0, int64_t e1,
                              uint64_t *sums, void *stream) {
    TG_TRY(check_counts(g, k));
    if (!sums || e0 < 0 || e1 < e0 || e1 > g->M) return TG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t len = tg_global_len(g->L, k);
    if (tg_is_device_ptr(sums)) {
        TG_TRY(sums_impl(g, k, e0, e1, reinterpret_cast<unsigned long long *>(sums), s));
        TG_TRY_CUDA(cudaStreamSynchronize(s));
        return TG_OK;
    }
    DevBuf<unsigned long long> d;
    if (!d.alloc(len, s)) return TG_ENOMEM;
    TG_TRY(sums_impl(g, k, e0, e1, d.p, s));
    TG_TRY_CUDA(cudaMemcpyAsync(sums, d.p, len * 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}

namespace {

// Per order position: the work of its edge in the per-edge pass, d_i + 8
// (d_i the smaller degree: the Gamma_i scan), for the cost-balanced slices.
__global__ void k_order_cost(const uint32_t *order, const int2 *edges, const int64_t *rowptr,
                             int64_t M, int64_t *cost) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q <= M;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (q == M) {
            cost[q] = 0;
            continue;
        }
        const int2 ab = edges[order[q]];
        const int i = max(ab.x, ab.y);
        cost[q] = rowptr[i + 1] - rowptr[i] + 8;
    }
}

// The first position whose exclusive prefix reaches total * r / parts, for
// r = first .. first + 1 (out[0], out[1]).
__global__ void k_split_points(const int64_t *prefix, int64_t M, int32_t first, int32_t parts,
                               int64_t *out) {
    const int r = first + (int)threadIdx.x;
    if (threadIdx.x > 1) return;
    const int64_t total = prefix[M];
    const int64_t want = (int64_t)((__int128)total * r / parts);
    int64_t lo = 0, hi = M;  // first q with prefix[q] >= want
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (prefix[mid] < want)
            lo = mid + 1;
        else
            hi = mid;
    }
    out[threadIdx.x] = r >= parts ? M : lo;
}

}  // namespace

extern "C" int tg_count_shard(const tg_graph *g, int32_t k, int32_t shard, int32_t nshards,
                              uint64_t *sums, void *stream) {
    TG_TRY(check_counts(g, k));
    if (!sums || nshards < 1 || shard < 0 || shard >= nshards) return TG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t len = tg_global_len(g->L, k);
    DevBuf<unsigned long long> d;
    unsigned long long *dsums = reinterpret_cast<unsigned long long *>(sums);
    const bool dev_out = tg_is_device_ptr(sums);
    if (!dev_out) {
        if (!d.alloc(len, s)) return TG_ENOMEM;
        dsums = d.p;
    }
    if (nshards == 1) {
        TG_TRY(sums_impl(g, k, 0, g->M, dsums, s));
    } else {
        TG_TRY_CUDA(cudaMemsetAsync(dsums, 0, len * 8, s));
        tg_sched *sc = nullptr;
        TG_TRY(get_sched(g, s, &sc));
        const int64_t M = g->M;
        int64_t q[2] = {0, 0};
        if (M > 0) {
            DevBuf<int64_t> cost, pre, qs;
            if (!cost.alloc(M + 1, s) || !pre.alloc(M + 1, s) || !qs.alloc(2, s)) return TG_ENOMEM;
            k_order_cost<<<grid_for(M + 1), 256, 0, s>>>(sc->order, g->edges, g->rowptr, M, cost.p); tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
            TG_TRY(tg_scan_i64(cost.p, pre.p, M + 1, s));
            k_split_points<<<1, 32, 0, s>>>(pre.p, M, shard, nshards, qs.p); tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
            TG_TRY_CUDA(cudaMemcpyAsync(q, qs.p, 16, cudaMemcpyDeviceToHost, s));
            TG_TRY_CUDA(cudaStreamSynchronize(s));
        }
        const tg_tune t = tune_now();
        if (t.kernel == TG_KERNEL_AUTO || t.kernel == TG_KERNEL_CYCLES) {
            // a slice of the edges, and a share of the whole-graph enumerations
            tg_part part;
            part.index = shard;
            part.count = nshards;
            if (k == 4)
                TG_TRY(tg_reuse_count(g, k, TG_GRAPHLET, sc->order, sc->order + q[0], q[1] - q[0],
                                      nullptr, 0, dsums, t, s, part));
            else if (q[1] > q[0])
                TG_TRY(tg_reuse_count(g, k, TG_GRAPHLET, sc->order, sc->order + q[0], q[1] - q[0],
                                      nullptr, 0, dsums, t, s));
        } else if (q[1] > q[0]) {
            // the per-edge kernels need nothing beyond the slice's edges
            TG_TRY(launch_count(g, k, TG_GRAPHLET, sc->order, sc->order + q[0], 0, q[1] - q[0],
                                nullptr, 0, dsums, s));
        }
    }
    if (!dev_out) TG_TRY_CUDA(cudaMemcpyAsync(sums, dsums, len * 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}

extern "C" int tg_count_per_edge(const tg_graph *g, int32_t k, int32_t level, uint64_t *rows,
                                 void *stream) {
    TG_TRY(check_counts(g, k));
    if (!rows || (level != TG_GRAPHLET && level != TG_ORBIT)) return TG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t width = tg_slots(g->L, k, level);
    if (g->M == 0) return TG_OK;
    tg_sched *sc = nullptr;
    TG_TRY(get_sched(g, s, &sc));
    if (tg_is_device_ptr(rows)) {
        TG_TRY(launch_count(g, k, level, sc->order, sc->order, 0, g->M, rows, width, nullptr, s));
        TG_TRY_CUDA(cudaStreamSynchronize(s));
        return TG_OK;
    }
    DevBuf<uint64_t> d;
    if (!d.alloc((size_t)g->M * width, s)) return TG_ENOMEM;
    TG_TRY(launch_count(g, k, level, sc->order, sc->order, 0, g->M, d.p, width, nullptr, s));
    TG_TRY_CUDA(cudaMemcpyAsync(rows, d.p, (size_t)g->M * width * 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}

int tg_rows_device(const tg_graph *g, int k, int level, uint64_t *rows, cudaStream_t s) {
    TG_TRY(check_counts(g, k));
    if (g->M == 0) return TG_OK;
    tg_sched *sc = nullptr;
    TG_TRY(get_sched(g, s, &sc));
    return launch_count(g, k, level, sc->order, sc->order, 0, g->M, rows,
                        tg_slots(g->L, k, level), nullptr, s);
}

extern "C" int tg_work_model(const tg_graph *g, uint64_t *entries, void *stream) {
    if (!g || !entries) return TG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    *entries = 0;
    if (g->M == 0) return TG_OK;
    tg_sched *sc = nullptr;
    TG_TRY(get_sched(g, s, &sc));
    TG_TRY(sched_sums(g, sc, s));
    DevBuf<unsigned long long> tot;
    if (!tot.alloc(1, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(tot.p, 0, 8, s));
    k_work_model<<<grid_for(g->M * 32), 256, 0, s>>>(g->rowptr, g->adj, g->toff, g->edges, g->M,
                                                     g->L, sc->s, tot.p, nullptr); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    unsigned long long h = 0;
    TG_TRY_CUDA(cudaMemcpyAsync(&h, tot.p, 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    *entries = h;
    return TG_OK;
}
