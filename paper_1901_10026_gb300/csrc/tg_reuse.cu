// Per-edge typed graphlet counts from Alg. 1's typed triangle counts.
//
// Alg. 1 gives, for every edge (a, b), the typed triangle counts
// tau_ab[t] = |Gamma_a^t n Gamma_b^t| (Def. "Typed Triangle Nodes").  For an
// edge (i, j) with d_i <= d_j, Alg. 2 and 3 classify the neighbours w_r of
// every w_k in S_i u S_j u T_ij.  For w_k adjacent to i or j, the part of
// Gamma_{w_k} inside Gamma_i (or Gamma_j) is exactly tau of the edge
// (i, w_k) (or (j, w_k)), so every count of Alg. 2-3 is fixed by tau, the
// typed degrees and two explicit enumerations:
//   Q[a][b]  = ordered pairs (y in T^a, z in T^b) that are adjacent (4-cliques)
//   S6[a][b] = pairs (x in S_i^a, w in Gamma_x n Gamma_j \ {i}, type b)
//              (4-cycles plus the S_i-T edges)
// both enumerated from the small side Gamma_i.  With ordered L x L matrices
// (first index: type of the member of the first set)
//   B  = sum_{y in T} tau_jy,  C = sum_{y in T} tau_iy,  DT = sum_{y in T} d_y,
//   Theta_v[a][b] = sum_{w in Gamma_v^a} tau_vw[b],  D_v[a][b] = sum d_w^b,
// the identities
//   TSj = B - Q - [b = phi_i] |T^a|          (y in T, z in S_j adjacent)
//   TSi = C - Q - [b = phi_j] |T^a|
//   SSj = Theta_j - B - [a = phi_i] tau_ij   (x in S_j, z in S_j u T)
//   SSi = Theta_i - C - [a = phi_j] tau_ij
//   DSj = D_j - DT - [a = phi_i] d_i,   DSi = D_i - DT - [a = phi_j] d_j
//   SjSj = SSj - TSj^T,  SiSi = SSi - TSi^T,  G6 = S6 - TSi^T
//   Y = DSi - [b = phi_i]|S_i^a| - SSi - G6 + DSj - [b = phi_j]|S_j^a| - SSj - G6^T
//   Z = DT - ([b = phi_i] + [b = phi_j]) |T^a| - Q - TSi - TSj
// give the enumerated orbits of Alg. 2-3 (sym(X){a,b} = X[a][b] + X[b][a] for
// a != b, X[a][a] for a = b):
//   g12 = sym(Q)/2, g10 = sym(TSi + TSj), g7 = sym(SiSi + SjSj)/2,
//   g6 = sym(G6), g3 = sym(Y), g8 = sym(Z);
// g4, g5, g9, g11 then follow from Sec. "Combinatorial Relationships" as in
// the paper.  The counts equal those of Alg. 1-3 exactly; the work drops from
// sum over w in S_i u S_j u T of d_w to the small side's enumerations.
#include <mutex>
#include <new>

#include "tg_device.cuh"

using namespace tgd;

namespace {

constexpr int kTauUnit = 256;  // edges per work unit of the tau kernel
constexpr int kTCap = 1024;    // T members kept in shared memory for probing
constexpr int kProbeFactor = 4;

// ---------------------------------------------------------------- units ----
// Work units of a grouped order (edges sorted by their high-degree end j): a
// unit is a run of edges sharing j.  A CTA rebuilds its Gamma_j bitmap when it
// takes a unit of another j, so a group is cut by cost, not by count: with
// c_e = d_i + kUnitEdgeCost per edge and C_j the group's total, the units hold
// about max(C_j / kUnitSplit, kUnitMinCost) each.  A hub's list is then built
// about kUnitSplit times, and its heavy edges (first in the group) are spread
// over as many units instead of filling one.
constexpr int kUnitSplit = 8;
constexpr int64_t kUnitEdgeCost = 16;
constexpr int64_t kUnitMinCost = 8192;

__global__ void k_group_bounds(const uint32_t *order, const int2 *edges, const int64_t *rowptr,
                               int64_t count, uint32_t *gs, uint32_t *ge, int64_t *cost) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < count;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int2 ab = edges[order[p]];
        const int j = min(ab.x, ab.y), i = max(ab.x, ab.y);
        if (p == 0 || min(edges[order[p - 1]].x, edges[order[p - 1]].y) != j) gs[j] = (uint32_t)p;
        if (p == count - 1 || min(edges[order[p + 1]].x, edges[order[p + 1]].y) != j)
            ge[j] = (uint32_t)(p + 1);
        cost[p] = (rowptr[i + 1] - rowptr[i]) + kUnitEdgeCost;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) cost[count] = 0;
}

// cum: exclusive prefix of the edge costs (count + 1 entries)
__global__ void k_unit_flags(const uint32_t *order, const int2 *edges, int64_t count,
                             const uint32_t *gs, const uint32_t *ge, const int64_t *cum,
                             uint32_t *flag) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < count;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int2 ab = edges[order[p]];
        const int j = min(ab.x, ab.y);
        const uint32_t g0 = gs[j];
        if ((uint32_t)p == g0) {
            flag[p] = 1u;
            continue;
        }
        const int64_t base = cum[g0];
        const int64_t ucost = max((cum[ge[j]] - base) / kUnitSplit, kUnitMinCost);
        flag[p] = (cum[p] - base) / ucost != (cum[p - 1] - base) / ucost ? 1u : 0u;
    }
}

__global__ void k_unit_starts(const uint32_t *flag, const uint32_t *pos, int64_t count,
                              uint32_t *ustart, uint32_t nunits) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < count;
         p += (int64_t)gridDim.x * blockDim.x)
        if (flag[p]) ustart[pos[p]] = (uint32_t)p;
    if (blockIdx.x == 0 && threadIdx.x == 0) ustart[nunits] = (uint32_t)count;
}

// flag[u] = unit u's j has at most TG_LIGHT_DEGREE neighbours
__global__ void k_unit_class(const uint32_t *order, const int2 *edges, const int64_t *rowptr,
                             const uint32_t *ustart, uint32_t nunits, uint32_t *flag) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nunits;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int2 ab = edges[order[ustart[u]]];
        const int j = min(ab.x, ab.y);
        flag[u] = (rowptr[j + 1] - rowptr[j]) <= TG_LIGHT_DEGREE ? 1u : 0u;
    }
}

__global__ void k_unit_lists(const uint32_t *flag, const uint32_t *pos, uint32_t nunits,
                             uint32_t *light, uint32_t *heavy) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nunits;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (flag[u])
            light[pos[u]] = (uint32_t)u;
        else
            heavy[u - pos[u]] = (uint32_t)u;
    }
}

// ------------------------------------------------------------ tau (Alg. 1) --
// One CTA per unit (edges sharing j); Gamma_j is a shared-memory bitmap that
// stays set while the CTA's units keep the same j; one warp per edge counts
// Gamma_i \ {j} against it by type.
// Bits [lo, hi) of a 32-bit word, the range clamped to the word.
__device__ __forceinline__ uint32_t word_bits(int lo, int hi) {
    lo = lo < 0 ? 0 : lo;
    hi = hi > 32 ? 32 : hi;
    if (lo >= hi) return 0u;
    const uint32_t up = hi == 32 ? 0xffffffffu : ((1u << hi) - 1u);
    return up & ~((1u << lo) - 1u);
}

constexpr int kTauUnroll = 8;       // chunks of 32 entries in flight per warp
constexpr int kTauThreads = 1024;   // one CTA per SM holds the bitmap: 32 warps share it

__global__ void __launch_bounds__(kTauThreads) k_tau(const int64_t *rowptr, const uint32_t *adj,
                                             const int32_t *toff, const uint8_t *ntype,
                                             const int2 *edges,
                                             const uint32_t *order, const uint32_t *ustart,
                                             const uint32_t *ulist, uint32_t nunits, int32_t L,
                                             int64_t nbits, unsigned long long *queue,
                                             uint32_t *tau) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int64_t bwords = (nbits + 31) >> 5;
    uint32_t *bm = reinterpret_cast<uint32_t *>(smem);
    unsigned long long *s_unit =
        reinterpret_cast<unsigned long long *>(smem + ((bwords * 4 + 15) & ~(int64_t)15));
    for (int64_t x = tid; x < bwords; x += blockDim.x) bm[x] = 0u;
    int cur_j = -1;
    int64_t cur_bj = 0;
    int cur_dj = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) *s_unit = atomicAdd(queue, 1ull);
        __syncthreads();
        const unsigned long long item = *s_unit;
        if (item >= nunits) break;
        const uint32_t u = ulist[item];
        const uint32_t p0 = ustart[u], p1 = ustart[u + 1];
        const int2 ab0 = edges[order[p0]];
        const int j = min(ab0.x, ab0.y);
        const int64_t bj = rowptr[j];
        const int dj = (int)(rowptr[j + 1] - bj);
        const int32_t *toj = toff + (int64_t)j * (L + 1);
        const uint32_t pj = ((uint32_t)ntype[j] << TG_TSHIFT) | (uint32_t)j;
        if (j != cur_j) {
            for (int x = tid; x < cur_dj; x += blockDim.x) {
                const uint32_t id = __ldg(adj + cur_bj + x) & TG_IDMASK;
                if ((int64_t)id < nbits) atomicAnd(&bm[id >> 5], ~(1u << (id & 31u)));
            }
            __syncthreads();
            for (int x = tid; x < dj; x += blockDim.x) {
                const uint32_t id = __ldg(adj + bj + x) & TG_IDMASK;
                if ((int64_t)id < nbits) atomicOr(&bm[id >> 5], 1u << (id & 31u));
            }
            cur_j = j;
            cur_bj = bj;
            cur_dj = dj;
            __syncthreads();
        }
        for (uint32_t p = p0 + warp; p < p1; p += W) {
            const uint32_t e = order[p];
            const int2 ab = edges[e];
            const int i = max(ab.x, ab.y);
            const int64_t bi = rowptr[i];
            const int di = (int)(rowptr[i + 1] - bi);
            // lane t < L keeps the count of type t: Gamma_i is sorted by type, so
            // the hits of type t are the ballot's bits in t's position range
            const int32_t *toi = toff + (int64_t)i * (L + 1);
            const int ts0 = lane < L ? __ldg(toi + lane) : 0, ts1 = lane < L ? __ldg(toi + lane + 1) : 0;
            unsigned mine = 0;
            // kTauUnroll chunks of 32 entries in flight per warp
            for (int c0 = 0; c0 < di; c0 += 32 * kTauUnroll) {
                uint32_t wv[kTauUnroll];
#pragma unroll
                for (int u = 0; u < kTauUnroll; ++u) {
                    const int x = c0 + 32 * u + lane;
                    wv[u] = x < di ? __ldg(adj + bi + x) : 0xffffffffu;
                }
#pragma unroll
                for (int u = 0; u < kTauUnroll; ++u) {
                    bool hit = false;
                    const uint32_t w = wv[u];
                    if (w != 0xffffffffu) {
                        const uint32_t id = w & TG_IDMASK;
                        if ((int)id != j)
                            hit = (int64_t)id < nbits ? bm_test(bm, id)
                                                      : adjacent(rowptr, adj, toff, L, bj, dj, toj, pj, w);
                    }
                    const unsigned hm = __ballot_sync(kFull, hit);
                    const int cb = c0 + 32 * u;
                    if (lane < L) mine += __popc(hm & word_bits(ts0 - cb, ts1 - cb));
                }
            }
            if (lane < L) tau[(int64_t)e * L + lane] = mine;
        }
    }
}

// tau_adj[p L + b] = tau[eid[p] L + b]: the triangle counts of every
// adjacency entry's edge, one thread per count.
__global__ void k_tau_adj(const uint32_t *eid, const uint32_t *tau, int64_t entries, int32_t L,
                          uint32_t *tau_adj) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < entries * L;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = x / L;
        tau_adj[x] = __ldg(tau + (int64_t)__ldg(eid + q) * L + (x - q * L));
    }
}

// Light units: one warp per unit, Gamma_j (at most TG_LIGHT_DEGREE entries)
// in a per-warp hash set, the unit's edges one after the other; no CTA barrier.
constexpr int kLightWarps = 8;

__global__ void __launch_bounds__(kLightWarps * 32) k_tau_light(
    const int64_t *rowptr, const uint32_t *adj, const int32_t *toff, const int2 *edges,
    const uint32_t *order,
    const uint32_t *ustart, const uint32_t *ulist, uint32_t nlist, int32_t L,
    unsigned long long *queue, uint32_t *tau) {
    __shared__ uint32_t keys[kLightWarps][1 << TG_LIGHT_LG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *hk = keys[warp];
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= nlist) break;
        const uint32_t u = ulist[item];
        const uint32_t p0 = ustart[u], p1 = ustart[u + 1];
        const int2 ab0 = edges[order[p0]];
        const int j = min(ab0.x, ab0.y);
        const int64_t bj = rowptr[j];
        const int dj = (int)(rowptr[j + 1] - bj);
        for (int q = lane; q < (1 << TG_LIGHT_LG); q += 32) hk[q] = 0u;
        __syncwarp();
        for (int x = lane; x < dj; x += 32) hset_put(hk, TG_LIGHT_LG, __ldg(adj + bj + x) & TG_IDMASK);
        __syncwarp();
        for (uint32_t p = p0; p < p1; ++p) {
            const uint32_t e = order[p];
            const int2 ab = edges[e];
            const int i = max(ab.x, ab.y);
            const int64_t bi = rowptr[i];
            const int di = (int)(rowptr[i + 1] - bi);
            // lane t < L keeps the count of type t (hits in t's position range)
            const int32_t *toi = toff + (int64_t)i * (L + 1);
            const int ts0 = lane < L ? __ldg(toi + lane) : 0, ts1 = lane < L ? __ldg(toi + lane + 1) : 0;
            unsigned mine = 0;
            for (int c0 = 0; c0 < di; c0 += 32) {
                const int x = c0 + lane;
                bool hit = false;
                if (x < di) {
                    const uint32_t id = __ldg(adj + bi + x) & TG_IDMASK;
                    hit = (int)id != j && hset_has(hk, TG_LIGHT_LG, id);
                }
                const unsigned hm = __ballot_sync(kFull, hit);
                if (lane < L) mine += __popc(hm & word_bits(ts0 - c0, ts1 - c0));
            }
            if (lane < L) tau[(int64_t)e * L + lane] = mine;
        }
        __syncwarp();
    }
}

// --------------------------------------------------- per-node aggregates ----
// Theta_v[a][b] = sum over w in Gamma_v^a of tau_vw[b]; D_v[a][b] = sum of
// d_w^b.  Nodes of degree up to dsmall: one thread per node, its 2 L^2 sums in
// a private column of shared memory (k_node_aggr_small).  Larger nodes: their
// typed ranges are cut into chunks of at most kAggrChunk entries, one warp per
// chunk, whose sums are added to the (zeroed) rows (k_node_aggr).
constexpr int kAggrSmall = 64;        // degree bound of the one-thread nodes
constexpr int kAggrSmallMaxL = 8;     // types up to which they are used
constexpr int kAggrSmallThreads = 128;
constexpr int kAggrChunk = 2048;

// chunks of node v's typed ranges (0 for a node left to the one-thread kernel)
__global__ void k_aggr_chunks(const int64_t *rowptr, const int32_t *toff, int64_t n, int32_t L,
                              int dsmall, uint32_t *nch) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c = 0;
        if (rowptr[v + 1] - rowptr[v] > dsmall) {
            const int32_t *tv = toff + v * (L + 1);
            for (int a = 0; a < L; ++a) c += (uint32_t)((tv[a + 1] - tv[a] + kAggrChunk - 1) / kAggrChunk);
        }
        nch[v] = c;
    }
}

__global__ void __launch_bounds__(kAggrSmallThreads)
    k_node_aggr_small(const int64_t *rowptr, const uint32_t *adj, const uint32_t *eid,
                      const int32_t *toff, const uint32_t *tau, int64_t n, int32_t L,
                      int dsmall, uint32_t *theta, uint32_t *dsum) {
    extern __shared__ uint32_t col[];  // [2 L^2][blockDim.x]
    const int tid = threadIdx.x, bd = blockDim.x;
    const int L2 = L * L;
    for (int64_t v = blockIdx.x * (int64_t)bd + tid; v < n; v += (int64_t)gridDim.x * bd) {
        const int64_t rb = rowptr[v], re = rowptr[v + 1];
        if (re - rb > dsmall) continue;  // a warp of k_node_aggr takes it
        for (int q = 0; q < 2 * L2; ++q) col[q * bd + tid] = 0u;
        for (int64_t x = rb; x < re; ++x) {
            const uint32_t wu = __ldg(adj + x);
            const int a = (int)(wu >> TG_TSHIFT);
            const uint32_t *tw = tau + (int64_t)__ldg(eid + x) * L;
            const int32_t *ow = toff + (int64_t)(wu & TG_IDMASK) * (L + 1);
            int prev = __ldg(ow);
            for (int b = 0; b < L; ++b) {
                const int nx = __ldg(ow + b + 1);
                col[(a * L + b) * bd + tid] += __ldg(tw + b);
                col[(L2 + a * L + b) * bd + tid] += (uint32_t)(nx - prev);
                prev = nx;
            }
        }
        for (int q = 0; q < L2; ++q) {
            theta[v * L2 + q] = col[q * bd + tid];
            dsum[v * L2 + q] = col[(L2 + q) * bd + tid];
        }
    }
}

__global__ void k_node_aggr(const int64_t *rowptr, const uint32_t *adj, const uint32_t *eid,
                            const int32_t *toff, const uint32_t *tau, int64_t n, int32_t L,
                            const uint32_t *nch, const uint32_t *cpos, uint32_t *theta,
                            uint32_t *dsum) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t items = (int64_t)cpos[n - 1] + nch[n - 1];
    for (int64_t it = wid; it < items; it += nw) {
        int64_t lo = 0, hi = n - 1;  // the last node whose first chunk is <= it
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if ((int64_t)cpos[mid] <= it)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int64_t v = lo;
        int64_t r = it - cpos[v];
        const int64_t rb = rowptr[v];
        const int32_t *tv = toff + v * (L + 1);
        int a = 0, s0 = 0, s1 = 0;
        for (; a < L; ++a) {
            s0 = __ldg(tv + a);
            s1 = __ldg(tv + a + 1);
            const int64_t ch = (s1 - s0 + kAggrChunk - 1) / kAggrChunk;
            if (r < ch) break;
            r -= ch;
        }
        const int c0 = s0 + (int)r * kAggrChunk, c1 = min(s1, c0 + kAggrChunk);
        uint32_t at[TG_MAX_TYPES], ad[TG_MAX_TYPES];
#pragma unroll
        for (int b = 0; b < TG_MAX_TYPES; ++b) {
            at[b] = 0;
            ad[b] = 0;
        }
        for (int x = c0 + lane; x < c1; x += 32) {
            const uint32_t w = __ldg(adj + rb + x) & TG_IDMASK;
            const uint32_t *tw = tau + (int64_t)__ldg(eid + rb + x) * L;
            const int32_t *ow = toff + (int64_t)w * (L + 1);
            int prev = __ldg(ow);
#pragma unroll
            for (int b = 0; b < TG_MAX_TYPES; ++b) {
                if (b < L) {
                    at[b] += __ldg(tw + b);
                    const int nx = __ldg(ow + b + 1);
                    ad[b] += (uint32_t)(nx - prev);
                    prev = nx;
                }
            }
        }
#pragma unroll
        for (int b = 0; b < TG_MAX_TYPES; ++b) {
            if (b < L) {
                const uint32_t st = __reduce_add_sync(kFull, at[b]);
                const uint32_t sd = __reduce_add_sync(kFull, ad[b]);
                if (lane == 0) {
                    if (st) atomicAdd(theta + (v * L + a) * L + b, st);
                    if (sd) atomicAdd(dsum + (v * L + a) * L + b, sd);
                }
            }
        }
    }
}

// ------------------------------------------------------ per-edge counts ----
struct ReuseParams {
    const int64_t *rowptr;
    const uint32_t *adj;
    const uint32_t *eid;
    const int32_t *toff;
    const uint8_t *ntype;
    const int2 *edges;
    const uint32_t *order;
    const uint32_t *tau;
    const uint32_t *theta;
    const uint32_t *dsum;
    int64_t count;
    int32_t L, P, k, level;
    int64_t nbits;
    int32_t hmax;
    unsigned long long *queue;
    uint64_t *rows;
    int64_t width;
    unsigned long long *hist;
    int64_t hist_len;
    int32_t hist_smem;
    int64_t off1, off2, off4, n4;
    unsigned long long *work;  // [Gamma_i entries, walked entries, probe pairs, T members]
};

__device__ __forceinline__ void hadd(const ReuseParams &p, unsigned long long *shist, int64_t x,
                                     unsigned long long v) {
    if (!v) return;
    if (p.hist_smem)
        atomicAdd(shist + x, v);
    else
        atomicAdd(p.hist + x, v);
}

// matrices (L x L, uint64) accumulated during the walk
enum { MB = 0, MC = 1, MDT = 2, MQ = 3, MS6 = 4, NMAT = 5 };
// derived matrices (int64)
enum { XTSJ = 0, XTSI, XSSJ, XSSI, XDSJ, XDSI, XSJSJ, XSISI, XG6, XY, XZ, NX };

template <int U>
__global__ void __launch_bounds__(1024, 1) k_count_reuse(ReuseParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int L = p.L, P = p.P, L2 = L * L;

    size_t off = 0;
    unsigned long long *shist = reinterpret_cast<unsigned long long *>(smem);
    if (p.hist_smem) off += ((size_t)p.hist_len * 8 + 15) & ~(size_t)15;
    unsigned long long *mat = reinterpret_cast<unsigned long long *>(smem + off);
    off += (size_t)NMAT * L2 * 8;
    long long *xm = reinterpret_cast<long long *>(smem + off);
    off += (size_t)NX * L2 * 8;
    const int64_t bwords = (p.nbits + 31) >> 5;
    uint32_t *bm = reinterpret_cast<uint32_t *>(smem + off);
    off += ((size_t)bwords * 4 + 15) & ~(size_t)15;
    uint32_t *hk = reinterpret_cast<uint32_t *>(smem + off);
    off += (size_t)p.hmax * 4;
    uint32_t *tlist = reinterpret_cast<uint32_t *>(smem + off);
    off += (size_t)kTCap * 4;
    unsigned *Tn = reinterpret_cast<unsigned *>(smem + off);
    unsigned *Si = Tn + 16;
    unsigned *Sj = Si + 16;
    unsigned long long *s_item = reinterpret_cast<unsigned long long *>(Sj + 16);
    unsigned *s_ntl = reinterpret_cast<unsigned *>(s_item + 1);
    // CTA-level staging of one tile of Gamma_i (blockDim entries each)
    unsigned char *stg = smem + off + kMiscBytes;
    const size_t nb = blockDim.x;
    int64_t *o_end = reinterpret_cast<int64_t *>(stg);
    int64_t *o_org = o_end + nb;
    int64_t *p_kb = o_org + nb;
    uint64_t *wsum = reinterpret_cast<uint64_t *>(p_kb + nb);  // 33 entries
    uint32_t *o_wk = reinterpret_cast<uint32_t *>(wsum + 34);
    uint32_t *p_wk = o_wk + nb;
    unsigned char *o_cls = reinterpret_cast<unsigned char *>(p_wk + nb);

    for (int64_t x = tid; x < bwords; x += blockDim.x) bm[x] = 0u;
    for (int x = tid; x < p.hmax; x += blockDim.x) hk[x] = kEmpty;
    if (p.hist_smem)
        for (int64_t x = tid; x < p.hist_len; x += blockDim.x) shist[x] = 0;

    const int64_t *__restrict__ rowptr = p.rowptr;
    const uint32_t *__restrict__ adj = p.adj;
    const int32_t *__restrict__ toff = p.toff;
    int cur_j = -1;
    int64_t cur_bj = 0;
    int cur_dj = 0;
    unsigned long long wk_gamma = 0, wk_walk = 0, wk_probe = 0, wk_tmem = 0;  // thread 0

    for (;;) {
        __syncthreads();
        if (tid == 0) *s_item = atomicAdd(p.queue, 1ull);
        __syncthreads();
        const unsigned long long item = *s_item;
        if (item >= (unsigned long long)p.count) break;
        const int64_t e = p.order[item];
        const int2 ab = p.edges[e];
        const int j = min(ab.x, ab.y), i = max(ab.x, ab.y);
        const int ti = p.ntype[i], tj = p.ntype[j];
        const int64_t bi = rowptr[i], bj = rowptr[j];
        const int di = (int)(rowptr[i + 1] - bi), dj = (int)(rowptr[j + 1] - bj);
        const int32_t *toi = toff + (int64_t)i * (L + 1);
        const int32_t *toj = toff + (int64_t)j * (L + 1);

        if (j != cur_j) {
            for (int x = tid; x < cur_dj; x += blockDim.x) {
                const uint32_t id = __ldg(adj + cur_bj + x) & TG_IDMASK;
                if ((int64_t)id < p.nbits) atomicAnd(&bm[id >> 5], ~(1u << (id & 31u)));
            }
            __syncthreads();
            for (int x = tid; x < dj; x += blockDim.x) {
                const uint32_t id = __ldg(adj + bj + x) & TG_IDMASK;
                if ((int64_t)id < p.nbits) atomicOr(&bm[id >> 5], 1u << (id & 31u));
            }
            cur_j = j;
            cur_bj = bj;
            cur_dj = dj;
        }
        for (int x = tid; x < NMAT * L2; x += blockDim.x) mat[x] = 0ull;
        if (tid < 48) Tn[tid] = 0;
        if (tid == 0) *s_ntl = 0;
        int lg = 5;
        while ((1 << lg) < 2 * di) ++lg;
        const int hash_ok = (1 << lg) <= p.hmax;
        __syncthreads();

        // ---- Alg. 1 on the bitmap: classes of Gamma_i, list of T ----------
        for (int x = tid; x < di; x += blockDim.x) {
            const uint32_t w = __ldg(adj + bi + x);
            const uint32_t id = w & TG_IDMASK;
            if ((int)id == j) continue;
            const bool inJ =
                (int64_t)id < p.nbits ? bm_test(bm, id) : contains(adj, bj, toj, w);
            if (inJ) {
                atomicAdd(&Tn[w >> TG_TSHIFT], 1u);
                const unsigned k = atomicAdd(s_ntl, 1u);
                if (k < (unsigned)kTCap) tlist[k] = w;
            } else {
                atomicAdd(&Si[w >> TG_TSHIFT], 1u);
            }
            if (hash_ok) hinsert(hk, lg, id, inJ ? CLS_T : CLS_SI);
        }
        __syncthreads();
        if (tid < L)
            Sj[tid] = (unsigned)(__ldg(toj + tid + 1) - __ldg(toj + tid)) - Tn[tid] -
                      (tid == ti ? 1u : 0u);
        const unsigned ntl = *s_ntl;
        const bool tl_ok = ntl <= (unsigned)kTCap;
        if (tid == 0) {
            wk_gamma += (unsigned long long)di;
            wk_tmem += ntl;
        }

        if (p.k == 4) {
            // Gamma_i in tiles of one member per thread.  Per tile: T members
            // add their tau / degree rows; a block scan stages the members
            // whose lists are walked (S_i for 4-cycles, short-list T for
            // 4-cliques) and those that probe the T list instead; then every
            // thread of the CTA takes positions of the concatenated lists.
            for (int tile = 0; tile < di; tile += (int)blockDim.x) {
                const int x = tile + tid;
                uint32_t wk = 0;
                int cls = CLS_I;
                if (x < di) {
                    wk = __ldg(adj + bi + x);
                    if ((int)(wk & TG_IDMASK) != j) {
                        const uint32_t id = wk & TG_IDMASK;
                        cls = hash_ok ? hlookup(hk, lg, id)
                                      : (contains(adj, bj, toj, wk) ? CLS_T : CLS_SI);
                    }
                }
                const int kid = (int)(wk & TG_IDMASK), kt = (int)(wk >> TG_TSHIFT);
                int64_t kb = 0;
                int dk = 0;
                if (cls != CLS_I) {
                    kb = rowptr[kid];
                    dk = (int)(rowptr[kid + 1] - kb);
                }
                const bool isT = cls == CLS_T;
                {
                    const unsigned tm = __match_any_sync(kFull, isT ? kt : -1);
                    const bool lead = isT && lane == __ffs(tm) - 1;
                    const uint32_t *tiy = p.tau;
                    const uint32_t *tjy = p.tau;
                    const int32_t *ty = toff + (int64_t)kid * (L + 1);
                    if (isT) {
                        tiy = p.tau + (int64_t)__ldg(p.eid + bi + x) * L;
                        const int pj = find_pos(adj, bj, toj, wk);
                        tjy = p.tau + (int64_t)__ldg(p.eid + bj + (pj < 0 ? 0 : pj)) * L;
                    }
                    int prev = isT ? __ldg(ty) : 0;
                    for (int b2 = 0; b2 < L; ++b2) {
                        uint32_t vb = 0, vc = 0, vd = 0;
                        if (isT) {
                            vb = __ldg(tjy + b2);
                            vc = __ldg(tiy + b2);
                            const int nx = __ldg(ty + b2 + 1);
                            vd = (uint32_t)(nx - prev);
                            prev = nx;
                        }
                        const uint32_t sb = __reduce_add_sync(tm, vb);
                        const uint32_t sc = __reduce_add_sync(tm, vc);
                        const uint32_t sd = __reduce_add_sync(tm, vd);
                        if (lead) {
                            const int m = kt * L + b2;
                            if (sb) atomicAdd(&mat[MB * L2 + m], (unsigned long long)sb);
                            if (sc) atomicAdd(&mat[MC * L2 + m], (unsigned long long)sc);
                            if (sd) atomicAdd(&mat[MDT * L2 + m], (unsigned long long)sd);
                        }
                    }
                }
                const bool probe = isT && tl_ok && dk > kProbeFactor * (int)ntl;
                const bool scan = (cls == CLS_SI) || (isT && !probe);
                // block scan of (scan count, probe count, walked length)
                const uint64_t packed = ((uint64_t)scan << 52) | ((uint64_t)probe << 41) |
                                        (uint64_t)(scan ? dk : 0);
                uint64_t incl = packed;
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
                    if (lane < W) wsum[lane] = y - y0;  // exclusive warp offsets
                    if (lane == W - 1) wsum[32] = y;    // tile total
                }
                __syncthreads();
                incl += wsum[warp];
                const uint64_t tot = wsum[32];
                const uint64_t mlen = ((uint64_t)1 << 41) - 1, mcnt = (1u << 11) - 1;
                const int nscan = (int)(tot >> 52), nprobe = (int)((tot >> 41) & mcnt);
                const int64_t total = (int64_t)(tot & mlen);
                if (scan) {
                    const int r = (int)((incl >> 52) - 1);
                    const int64_t end = (int64_t)(incl & mlen);
                    o_end[r] = end;
                    o_org[r] = kb - (end - dk);
                    o_wk[r] = wk;
                    o_cls[r] = (unsigned char)cls;
                }
                if (probe) {
                    const int r = (int)(((incl >> 41) & mcnt) - 1);
                    p_wk[r] = wk;
                    p_kb[r] = kb;
                }
                if (tid == 0) {
                    wk_walk += (unsigned long long)total;
                    wk_probe += (unsigned long long)nprobe * ntl;
                }
                __syncthreads();
                // walk the concatenated lists of the staged members
                for (int64_t base = 0; base < total; base += (int64_t)blockDim.x * U) {
                    uint32_t wr[U], owk[U];
                    int ocl[U];
                    bool val[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int64_t pos = base + (int64_t)u * blockDim.x + tid;
                        val[u] = pos < total;
                        wr[u] = 0u;
                        owk[u] = 0u;
                        ocl[u] = 0;
                        if (val[u]) {
                            int lo = 0, hi = nscan - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (o_end[mid] > pos)
                                    hi = mid;
                                else
                                    lo = mid + 1;
                            }
                            owk[u] = o_wk[lo];
                            ocl[u] = o_cls[lo];
                            wr[u] = __ldg(adj + (o_org[lo] + pos));
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        int key = -1;
                        if (val[u]) {
                            const uint32_t rid = wr[u] & TG_IDMASK;
                            const bool inJ = (int64_t)rid < p.nbits
                                                 ? bm_test(bm, rid)
                                                 : contains(adj, bj, toj, wr[u]);
                            if (inJ && (int)rid != i) {
                                const int m = (int)(owk[u] >> TG_TSHIFT) * L +
                                              (int)(wr[u] >> TG_TSHIFT);
                                if (ocl[u] == CLS_SI) {
                                    key = MS6 * L2 + m;  // 4-cycle or S_i-T edge
                                } else {
                                    const int rc = hash_ok
                                                       ? hlookup(hk, lg, rid)
                                                       : (contains(adj, bi, toi, wr[u]) ? CLS_T : 0);
                                    if (rc == CLS_T) key = MQ * L2 + m;  // 4-clique
                                }
                            }
                        }
                        const unsigned mm = __match_any_sync(kFull, key);
                        if (key >= 0 && lane == __ffs(mm) - 1)
                            atomicAdd(&mat[key], (unsigned long long)__popc(mm));
                    }
                }
                // probe pairs (y, z): y a long-list T member, z another T member
                const int64_t npairs = (int64_t)nprobe * ntl;
                for (int64_t q0 = 0; q0 < npairs; q0 += blockDim.x) {
                    const int64_t q = q0 + tid;
                    int key = -1;
                    if (q < npairs) {
                        const int yi = (int)(q / ntl), zi = (int)(q % ntl);
                        const uint32_t y = p_wk[yi], z = tlist[zi];
                        if (z != y) {
                            const int32_t *yto = toff + (int64_t)(y & TG_IDMASK) * (L + 1);
                            if (find_pos(adj, p_kb[yi], yto, z) >= 0)
                                key = MQ * L2 + (int)(y >> TG_TSHIFT) * L + (int)(z >> TG_TSHIFT);
                        }
                    }
                    const unsigned mm = __match_any_sync(kFull, key);
                    if (key >= 0 && lane == __ffs(mm) - 1)
                        atomicAdd(&mat[key], (unsigned long long)__popc(mm));
                }
                __syncthreads();  // staged members are rewritten by the next tile
            }
        }
        __syncthreads();

        // ---- identities (see the file header) -----------------------------
        const uint32_t *thi = p.theta + (int64_t)i * L2, *thj = p.theta + (int64_t)j * L2;
        const uint32_t *dvi = p.dsum + (int64_t)i * L2, *dvj = p.dsum + (int64_t)j * L2;
        if (p.k == 4) {
            for (int m = tid; m < L2; m += blockDim.x) {
                const int a = m / L, b = m % L;
                const long long Bm = (long long)mat[MB * L2 + m], Cm = (long long)mat[MC * L2 + m];
                const long long Qm = (long long)mat[MQ * L2 + m], DT = (long long)mat[MDT * L2 + m];
                const long long di_b = __ldg(toi + b + 1) - __ldg(toi + b);
                const long long dj_b = __ldg(toj + b + 1) - __ldg(toj + b);
                xm[XTSJ * L2 + m] = Bm - Qm - (b == ti ? (long long)Tn[a] : 0);
                xm[XTSI * L2 + m] = Cm - Qm - (b == tj ? (long long)Tn[a] : 0);
                xm[XSSJ * L2 + m] = (long long)__ldg(thj + m) - Bm - (a == ti ? (long long)Tn[b] : 0);
                xm[XSSI * L2 + m] = (long long)__ldg(thi + m) - Cm - (a == tj ? (long long)Tn[b] : 0);
                xm[XDSJ * L2 + m] = (long long)__ldg(dvj + m) - DT - (a == ti ? di_b : 0);
                xm[XDSI * L2 + m] = (long long)__ldg(dvi + m) - DT - (a == tj ? dj_b : 0);
            }
            __syncthreads();
            for (int m = tid; m < L2; m += blockDim.x) {
                const int a = m / L, b = m % L, mt = b * L + a;
                const long long g6 = (long long)mat[MS6 * L2 + m] - xm[XTSI * L2 + mt];
                const long long g6t = (long long)mat[MS6 * L2 + mt] - xm[XTSI * L2 + m];
                xm[XSJSJ * L2 + m] = xm[XSSJ * L2 + m] - xm[XTSJ * L2 + mt];
                xm[XSISI * L2 + m] = xm[XSSI * L2 + m] - xm[XTSI * L2 + mt];
                xm[XG6 * L2 + m] = g6;
                xm[XY * L2 + m] = xm[XDSI * L2 + m] - (b == ti ? (long long)Si[a] : 0) -
                                  xm[XSSI * L2 + m] - g6 + xm[XDSJ * L2 + m] -
                                  (b == tj ? (long long)Sj[a] : 0) - xm[XSSJ * L2 + m] - g6t;
                xm[XZ * L2 + m] = (long long)mat[MDT * L2 + m] -
                                  (long long)Tn[a] * ((b == ti) + (b == tj)) -
                                  (long long)mat[MQ * L2 + m] - xm[XTSI * L2 + m] -
                                  xm[XTSJ * L2 + m];
            }
            __syncthreads();
        }

        // ---- closed forms and output --------------------------------------
        if (p.rows) {
            uint64_t *row = p.rows + e * p.width;
            for (int t = tid; t < L; t += blockDim.x) {
                row[t] = (uint64_t)Si[t] + Sj[t];
                row[L + t] = Tn[t];
            }
        } else {
            if (tid == 0) {
                int a = ti, b = tj;
                sort2(a, b);
                hadd(p, shist, (int64_t)a + (int64_t)(b + 1) * b / 2, 1ull);
            }
            for (int t = tid; t < L; t += blockDim.x) {
                int a = ti, b = tj, cc = t;
                sort2(a, b);
                sort2(b, cc);
                sort2(a, b);
                const int64_t r = colex3(a, b, cc);
                hadd(p, shist, p.off1 + r, (unsigned long long)Si[t] + Sj[t]);
                hadd(p, shist, p.off2 + r, (unsigned long long)Tn[t]);
            }
        }
        if (p.k == 4) {
            for (int pr = tid; pr < P; pr += blockDim.x) {
                int t, u;
                unpair(L, pr, t, u);
                const int m = t * L + u, mt = u * L + t;
                auto sym = [&](int X) -> long long {
                    return t == u ? xm[X * L2 + m] : xm[X * L2 + m] + xm[X * L2 + mt];
                };
                const long long q2 = t == u ? (long long)mat[MQ * L2 + m]
                                            : (long long)mat[MQ * L2 + m] + (long long)mat[MQ * L2 + mt];
                const uint64_t g12 = (uint64_t)(q2 / 2);
                const uint64_t g10 = (uint64_t)(sym(XTSI) + sym(XTSJ));
                const uint64_t g7 = (uint64_t)((sym(XSISI) + sym(XSJSJ)) / 2);
                const uint64_t g6 = (uint64_t)sym(XG6);
                const uint64_t g3 = (uint64_t)sym(XY);
                const uint64_t g8 = (uint64_t)sym(XZ);
                const uint64_t sit = Si[t], siu = Si[u], sjt = Sj[t], sju = Sj[u];
                const uint64_t tt = Tn[t], tu = Tn[u];
                uint64_t g4, g5, g9, g11;
                if (t == u) {
                    g4 = sit * sjt - g6;
                    g5 = c2(sit) + c2(sjt) - g7;
                    g9 = tt * (sit + sjt) - g10;
                    g11 = c2(tt) - g12;
                } else {
                    g4 = sit * sju + siu * sjt - g6;
                    g5 = sit * siu + sjt * sju - g7;
                    g9 = tt * (siu + sju) + tu * (sit + sjt) - g10;
                    g11 = tt * tu - g12;
                }
                if (p.rows) {
                    uint64_t *row = p.rows + e * p.width + 2 * L;
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
                        for (int q = 0; q < 6; ++q) hadd(p, shist, p.off4 + q * p.n4 + r, h[q]);
                    }
                }
            }
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
    if (tid == 0 && p.work) {
        atomicAdd(p.work + 0, wk_gamma);
        atomicAdd(p.work + 1, wk_walk);
        atomicAdd(p.work + 2, wk_probe);
        atomicAdd(p.work + 3, wk_tmem);
    }
}

// Events and work counters of the calling thread's last call (see
// tg_last_timing).  One set per host thread, so counts run concurrently from
// several threads (the serving loop's workers) neither reset nor mix each
// other's counters.
inline unsigned grid_r(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (unsigned)b;
}

struct LastTiming {
    bool ready = false;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    unsigned long long *work = nullptr;  // device, kWorkCounters counters
    uint64_t edges = 0;
    ~LastTiming() {
        for (auto &e : ev)
            if (e) (void)cudaEventDestroy(e);
        if (work) (void)cudaFree(work);
    }
};
thread_local LastTiming g_last;
constexpr int kWorkCounters = 8;

int timing_begin(cudaStream_t s, unsigned long long **work) {
    if (!g_last.ev[0]) {
        for (auto &e : g_last.ev) TG_TRY_CUDA(cudaEventCreate(&e));
        TG_TRY_CUDA(cudaMalloc(&g_last.work, kWorkCounters * sizeof(unsigned long long)));
    }
    g_last.ready = false;
    TG_TRY_CUDA(cudaMemsetAsync(g_last.work, 0, kWorkCounters * sizeof(unsigned long long), s));
    *work = g_last.work;
    return TG_OK;
}

// Work units of the grouped order (see k_unit_flags), split by class.
int edge_units(const tg_graph *g, const uint32_t *ord, int64_t cnt, cudaStream_t s,
               tg_units &un) {
    DevBuf<uint32_t> flag, pos, gs, ge;
    DevBuf<int64_t> cost, cum;
    if (!flag.alloc(cnt, s) || !pos.alloc(cnt, s) || !gs.alloc(g->n, s) || !ge.alloc(g->n, s) ||
        !cost.alloc(cnt + 1, s) || !cum.alloc(cnt + 1, s))
        return TG_ENOMEM;
    k_group_bounds<<<grid_r(cnt), 256, 0, s>>>(ord, g->edges, g->rowptr, cnt, gs.p, ge.p, cost.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    TG_TRY(tg_scan_i64(cost.p, cum.p, cnt + 1, s));
    k_unit_flags<<<grid_r(cnt), 256, 0, s>>>(ord, g->edges, cnt, gs.p, ge.p, cum.p, flag.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    TG_TRY(tg_scan_u32(flag.p, pos.p, cnt, s));
    uint32_t lastp = 0, lastf = 0;
    TG_TRY_CUDA(cudaMemcpyAsync(&lastp, pos.p + cnt - 1, 4, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaMemcpyAsync(&lastf, flag.p + cnt - 1, 4, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    un.nunits = lastp + lastf;
    if (!un.ustart.alloc((size_t)un.nunits + 1, s)) return TG_ENOMEM;
    k_unit_starts<<<grid_r(cnt), 256, 0, s>>>(flag.p, pos.p, cnt, un.ustart.p, un.nunits); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    // classes: light (one warp each) and heavy (one CTA each)
    DevBuf<uint32_t> cflag, cpos;
    if (!cflag.alloc(un.nunits, s) || !cpos.alloc(un.nunits, s) ||
        !un.light.alloc(un.nunits, s) || !un.heavy.alloc(un.nunits, s))
        return TG_ENOMEM;
    k_unit_class<<<grid_r(un.nunits), 256, 0, s>>>(ord, g->edges, g->rowptr, un.ustart.p, un.nunits,
                                                   cflag.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    TG_TRY(tg_scan_u32(cflag.p, cpos.p, un.nunits, s));
    k_unit_lists<<<grid_r(un.nunits), 256, 0, s>>>(cflag.p, cpos.p, un.nunits, un.light.p,
                                                   un.heavy.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    TG_TRY_CUDA(cudaMemcpyAsync(&lastp, cpos.p + un.nunits - 1, 4, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaMemcpyAsync(&lastf, cflag.p + un.nunits - 1, 4, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    un.nlight = lastp + lastf;
    un.nheavy = un.nunits - un.nlight;
    return TG_OK;
}




template <int U>
int launch_reuse_u(const ReuseParams &p, int threads, size_t smem, int grid_limit,
                   cudaStream_t s) {
    TG_TRY(tg_allow_max_smem((const void *)k_count_reuse<U>));
    int per_sm = 0;
    TG_TRY_CUDA(
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_reuse<U>, threads, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)tg_num_sms() * per_sm;
    if (grid > p.count) grid = p.count;
    if (grid_limit > 0 && grid > grid_limit) grid = grid_limit;
    if (grid < 1) grid = 1;
    k_count_reuse<U><<<(unsigned)grid, threads, smem, s>>>(p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    return TG_OK;
}

}  // namespace

// Runs Alg. 1 for every edge (tau), the per-node sums, then the per-edge
// counts for the edges order[0..count) (grouped by their high-degree end).
int tg_reuse_count(const tg_graph *g, int k, int level, const uint32_t *full_order,
                   const uint32_t *order, int64_t count, uint64_t *rows, int64_t width,
                   unsigned long long *hist, const tg_tune &t, cudaStream_t s,
                   const tg_part &part) {
    if (count <= 0 && part.count <= 1) return TG_OK;  // a share of a split count still enumerates
    const int L = g->L, L2 = L * L;
    const int64_t M = g->M, n = g->n;
    unsigned long long *work = nullptr;
    TG_TRY(timing_begin(s, &work));
    // tau for every edge of the graph (the identities need tau of edges
    // outside the counted range as well)
    DevBuf<uint32_t> tau, theta, dsum;
    tg_units un;
    if (!tau.alloc((size_t)M * L, s)) return TG_ENOMEM;
    {
        // tau of every edge, in the grouped order of the whole graph
        const uint32_t *ord = full_order;
        TG_TRY(edge_units(g, ord, M, s, un));
        DevBuf<unsigned long long> q;
        if (!q.alloc(2, s)) return TG_ENOMEM;
        TG_TRY_CUDA(cudaMemsetAsync(q.p, 0, 16, s));
        TG_TRY_CUDA(cudaEventRecord(g_last.ev[0], s));
        if (un.nheavy > 0) {
            const size_t avail = (size_t)tg_smem_optin();
            int64_t nbits = g->n_nonisolated;
            if (t.bitmap_bits > 0 && nbits > t.bitmap_bits) nbits = t.bitmap_bits;
            const int64_t maxb = (int64_t)((avail - 64) / 16) * 128;
            if (nbits > maxb) nbits = maxb;
            const size_t smem = ((((size_t)((nbits + 31) >> 5)) * 4 + 15) & ~(size_t)15) + 16;
            TG_TRY(tg_allow_max_smem((const void *)k_tau));
            int per_sm = 0;
            TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tau, kTauThreads, smem));
            if (per_sm < 1) per_sm = 1;
            int64_t grid = (int64_t)tg_num_sms() * per_sm;
            if (grid > (int64_t)un.nheavy) grid = un.nheavy;
            if (grid < 1) grid = 1;
            k_tau<<<(unsigned)grid, kTauThreads, smem, s>>>(g->rowptr, g->adj, g->toff, g->ntype, g->edges, ord,
                                                    un.ustart.p, un.heavy.p, un.nheavy, L, nbits,
                                                    q.p, tau.p); tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
        }
        if (un.nlight > 0) {
            int per_sm = 0;
            TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tau_light,
                                                                      kLightWarps * 32, 0));
            if (per_sm < 1) per_sm = 1;
            int64_t grid = (int64_t)tg_num_sms() * per_sm;
            const int64_t need = ((int64_t)un.nlight + kLightWarps - 1) / kLightWarps;
            if (grid > need) grid = need;
            k_tau_light<<<(unsigned)grid, kLightWarps * 32, 0, s>>>(
                g->rowptr, g->adj, g->toff, g->edges, ord, un.ustart.p, un.light.p, un.nlight, L,
                q.p + 1, tau.p); tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
        }
    }
    TG_TRY_CUDA(cudaEventRecord(g_last.ev[1], s));
    if (k == 4) {
        if (!theta.alloc((size_t)n * L2, s) || !dsum.alloc((size_t)n * L2, s)) return TG_ENOMEM;
        const int dsmall = L <= kAggrSmallMaxL ? kAggrSmall : -1;
        // rows of the chunked nodes start at zero
        TG_TRY_CUDA(cudaMemsetAsync(theta.p, 0, (size_t)n * L2 * 4, s));
        TG_TRY_CUDA(cudaMemsetAsync(dsum.p, 0, (size_t)n * L2 * 4, s));
        if (dsmall >= 0) {
            const size_t asmem = (size_t)2 * L2 * kAggrSmallThreads * 4;
            TG_TRY(tg_allow_max_smem((const void *)k_node_aggr_small));
            int per = 0;
            TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_node_aggr_small,
                                                                      kAggrSmallThreads, asmem));
            const int64_t ag = std::min<int64_t>((int64_t)tg_num_sms() * (per > 0 ? per : 1),
                                                 (n + kAggrSmallThreads - 1) / kAggrSmallThreads);
            k_node_aggr_small<<<(unsigned)std::max<int64_t>(ag, 1), kAggrSmallThreads, asmem, s>>>(
                g->rowptr, g->adj, g->eid, g->toff, tau.p, n, L, dsmall, theta.p, dsum.p); tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
        }
        DevBuf<uint32_t> nch, cpos;
        if (n > 0) {
            if (!nch.alloc(n, s) || !cpos.alloc(n, s)) return TG_ENOMEM;
            k_aggr_chunks<<<grid_r(n), 256, 0, s>>>(g->rowptr, g->toff, n, L, dsmall, nch.p); tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
            TG_TRY(tg_scan_u32(nch.p, cpos.p, n, s));
            int per = 0;
            TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_node_aggr, 256, 0));
            k_node_aggr<<<(unsigned)((int64_t)tg_num_sms() * (per > 0 ? per : 1)), 256, 0, s>>>(
                g->rowptr, g->adj, g->eid, g->toff, tau.p, n, L, nch.p, cpos.p, theta.p, dsum.p); tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
        }
    }
    TG_TRY_CUDA(cudaEventRecord(g_last.ev[2], s));
    if (t.kernel == TG_KERNEL_CYCLES || t.kernel == TG_KERNEL_AUTO) {
        // 4-cycles and 4-cliques per edge from whole-graph enumerations, then
        // the per-edge identities (tg_cycles.cu)
        DevBuf<unsigned long long> c4e, k4e, g4c, g4k;
        // whole-graph global sums: the 4-cycle and 4-clique terms come from
        // their type-multiset totals instead of per-edge counters
        // (a share of a split count: the part's own enumeration totals)
        const bool split_part = part.count > 1;
        if (split_part && (k != 4 || !hist || rows)) return TG_EINVAL;
        const bool fast =
            k == 4 && hist && !rows && (split_part || (order == full_order && count == M));
        if (fast) {
            const int64_t n4 = tg_binom(L + 3, 4);
            if (!g4c.alloc(n4, s) || !g4k.alloc(n4, s)) return TG_ENOMEM;
            TG_TRY_CUDA(cudaMemsetAsync(g4c.p, 0, n4 * 8, s));
            TG_TRY_CUDA(cudaMemsetAsync(g4k.p, 0, n4 * 8, s));
            TG_TRY(tg_cyc_cycles(g, nullptr, g4c.p, work, t, part, s));
        } else if (k == 4) {
            const int P = L * (L + 1) / 2;
            if (!c4e.alloc((size_t)M * L2, s) || !k4e.alloc((size_t)M * P, s)) return TG_ENOMEM;
            TG_TRY_CUDA(cudaMemsetAsync(c4e.p, 0, (size_t)M * L2 * 8, s));
            TG_TRY_CUDA(cudaMemsetAsync(k4e.p, 0, (size_t)M * P * 8, s));
            TG_TRY(tg_cyc_cycles(g, c4e.p, nullptr, work, t, tg_part(), s));
        }
        TG_TRY_CUDA(cudaEventRecord(g_last.ev[3], s));
        if (k == 4) TG_TRY(tg_cyc_cliques(g, k4e.p, g4k.p, work, t, fast ? part : tg_part(), s));
        TG_TRY_CUDA(cudaEventRecord(g_last.ev[4], s));
        tg_units un2;
        tg_units *ue = &un;
        if (order != full_order || count != M) {
            if (count > 0) TG_TRY(edge_units(g, order, count, s, un2));
            ue = &un2;
        }
        // triangle counts per adjacency entry, for the per-edge pass's reads
        DevBuf<uint32_t> tau_adj;
        if (k == 4 && count > 0) {
            if (!tau_adj.alloc((size_t)2 * M * L, s)) return TG_ENOMEM;
            k_tau_adj<<<grid_r(2 * M * L), 256, 0, s>>>(g->eid, tau.p, 2 * M, L, tau_adj.p); tg_note_launch();
            TG_TRY_CUDA(cudaGetLastError());
        }
        TG_TRY(tg_cyc_edges(g, k, level, order, count, *ue, rows, width, hist, tau.p, tau_adj.p,
                            theta.p, dsum.p, c4e.p, k4e.p, work, t, s));
        if (fast) TG_TRY(tg_cyc_correct(hist, L, g4c.p, g4k.p, s));
        TG_TRY_CUDA(cudaEventRecord(g_last.ev[5], s));
        g_last.edges = (uint64_t)count;
        g_last.ready = true;
        return TG_OK;
    }
    TG_TRY_CUDA(cudaEventRecord(g_last.ev[3], s));
    TG_TRY_CUDA(cudaEventRecord(g_last.ev[4], s));
    DevBuf<unsigned long long> queue;
    if (!queue.alloc(1, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(queue.p, 0, 8, s));
    ReuseParams p{};
    p.work = work;
    p.rowptr = g->rowptr;
    p.adj = g->adj;
    p.eid = g->eid;
    p.toff = g->toff;
    p.ntype = g->ntype;
    p.edges = g->edges;
    p.order = order;
    p.tau = tau.p;
    p.theta = theta.p;
    p.dsum = dsum.p;
    p.count = count;
    p.L = L;
    p.P = L * (L + 1) / 2;
    p.k = k;
    p.level = level;
    p.queue = queue.p;
    p.rows = rows;
    p.width = width;
    p.hist = hist;
    p.hist_len = tg_global_len(L, k);
    p.off1 = tg_binom(L + 1, 2);
    p.off2 = p.off1 + tg_binom(L + 2, 3);
    p.off4 = p.off1 + 2 * tg_binom(L + 2, 3);
    p.n4 = tg_binom(L + 3, 4);
    const int threads = t.cta_threads;
    const size_t hist_bytes = ((size_t)p.hist_len * 8 + 15) & ~(size_t)15;
    p.hist_smem = (!rows && hist_bytes <= 48 * 1024) ? 1 : 0;
    const size_t stage_bytes = (size_t)threads * (3 * 8 + 2 * 4 + 1) + 34 * 8 + 16;
    const size_t fixed = (p.hist_smem ? hist_bytes : 0) + (size_t)(NMAT + NX) * L2 * 8 +
                         (size_t)kTCap * 4 + kMiscBytes + stage_bytes;
    const size_t avail = (size_t)tg_smem_optin();
    int hmax = t.hash_slots;
    while (fixed + (size_t)hmax * 4 + 4096 > avail && hmax > 32) hmax >>= 1;
    if (fixed + (size_t)hmax * 4 + 16 > avail) return TG_EINVAL;
    int64_t nbits = g->n_nonisolated;
    if (t.bitmap_bits > 0 && nbits > t.bitmap_bits) nbits = t.bitmap_bits;
    const int64_t maxb = (int64_t)((avail - fixed - (size_t)hmax * 4 - 16) / 16) * 128;
    if (nbits > maxb) nbits = maxb;
    if (nbits < 0) nbits = 0;
    p.nbits = nbits;
    p.hmax = hmax;
    const size_t smem = fixed + ((((size_t)((nbits + 31) >> 5)) * 4 + 15) & ~(size_t)15) +
                        (size_t)hmax * 4;
    int r;
    switch (t.unroll) {
        case 1: r = launch_reuse_u<1>(p, threads, smem, t.grid_limit, s); break;
        case 4: r = launch_reuse_u<4>(p, threads, smem, t.grid_limit, s); break;
        default: r = launch_reuse_u<2>(p, threads, smem, t.grid_limit, s); break;
    }
    if (r != TG_OK) return r;
    TG_TRY_CUDA(cudaEventRecord(g_last.ev[5], s));
    g_last.edges = (uint64_t)count;
    g_last.ready = true;
    return TG_OK;
}

extern "C" int tg_last_timing(tg_timing *out) {
    if (!out) return TG_EINVAL;
    if (!g_last.ready) return TG_ENOTFOUND;
    TG_TRY_CUDA(cudaEventSynchronize(g_last.ev[5]));
    float ms[5] = {0, 0, 0, 0, 0};
    for (int q = 0; q < 5; ++q)
        TG_TRY_CUDA(cudaEventElapsedTime(&ms[q], g_last.ev[q], g_last.ev[q + 1]));
    unsigned long long w[kWorkCounters] = {};
    TG_TRY_CUDA(cudaMemcpy(w, g_last.work, sizeof(w), cudaMemcpyDeviceToHost));
    out->tau_ms = ms[0];
    out->aggregate_ms = ms[1];
    out->cycles_ms = ms[2];
    out->cliques_ms = ms[3];
    out->count_ms = ms[4];
    out->edges = g_last.edges;
    out->gamma_entries = w[0];
    out->walked_entries = w[1];
    out->probe_pairs = w[2];
    out->t_members = w[3];
    out->wedges = w[4];
    out->clique_tests = w[5];
    out->cliques = w[6];
    return TG_OK;
}
