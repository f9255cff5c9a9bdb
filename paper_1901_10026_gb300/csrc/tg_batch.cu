// Batched counting: many graphs in one persistent launch.
//
// Every (graph, edge) pair of the batch is one work item.  Items are ordered
// by an estimate of their Alg. 2-3 work (heaviest first, a degree-binned
// queue) and taken by warps from a shared atomic counter; a warp finds its
// item's graph by binary search over the per-graph item offsets and runs
// Alg. 1-3 and the closed forms for that edge (one warp per edge, membership
// by binary search in the (type, id)-sorted lists, the I-class orbits through
// typed degrees).  Per-edge mode writes each graph's rows; global mode adds
// into per-graph undivided sums that a second kernel divides by |E(H)|.
// The plan (descriptors, queue, scratch) is built once; runs are replayed
// from a captured CUDA graph.
//
// Union path: the graphs of one type count L also form one disjoint union
// (node ids offset per graph, built once per plan with the library's CSR
// builder), counted per edge by the whole-graph path of the single-graph
// calls (Alg. 1's triangle counts reused through the identities, 4-cycles
// and 4-cliques enumerated once); the union's canonical edge order keeps each
// graph's edges together and in the graph's own canonical order, so a
// graph's rows are one block of the union's rows, copied out per graph
// (per-edge modes) or summed per graph into its undivided sums (global mode).
// The tuner times both paths and keeps the faster.
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "tg_device.cuh"

using namespace tgd;

namespace {

enum { B3 = 0, B6 = 1, B7 = 2, B8 = 3, B10 = 4, B12 = 5, BN = 6 };

struct BatchGraph {
    const int32_t *new2old;      // for the union inputs
    int64_t n, M;
    const int64_t *rowptr;
    const uint32_t *adj;
    const int32_t *toff;
    const uint8_t *ntype;
    const int2 *edges;
    uint64_t *rows;              // per-edge output (per-edge modes)
    unsigned long long *sums;    // undivided sums (global mode)
    uint64_t *out;               // final global output (global mode)
    int64_t width;
    int32_t L, P;
    int64_t off1, off2, off4, n4, glen;
};

struct BatchParams {
    const BatchGraph *gs;
    const int64_t *eoff;  // G + 1 item offsets
    const uint32_t *order;
    int32_t G;
    int64_t count;
    int32_t k, level, global;
    int32_t Pmax;
    unsigned long long *queue;
};

__device__ __forceinline__ int find_graph(const int64_t *eoff, int G, int64_t item) {
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(eoff + mid) <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void k_batch_warp(BatchParams bp) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t wbytes = ((size_t)BN * bp.Pmax * 4 + 3 * 16 * 4 + 32 * 4 + 15) & ~(size_t)15;
    unsigned char *wb = smem + warp * wbytes;
    int *cnt = reinterpret_cast<int *>(wb);
    unsigned *Tn = reinterpret_cast<unsigned *>(wb + (size_t)BN * bp.Pmax * 4);
    unsigned *Si = Tn + 16;
    unsigned *Sj = Si + 16;
    int *pos2owner = reinterpret_cast<int *>(Sj + 16);

    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(bp.queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= (unsigned long long)bp.count) break;
        const int64_t gi = bp.order ? (int64_t)bp.order[item] : (int64_t)item;
        const int gidx = find_graph(bp.eoff, bp.G, gi);
        const BatchGraph &G = bp.gs[gidx];
        const int64_t e = gi - __ldg(bp.eoff + gidx);
        const int L = G.L, P = G.P;
        const int64_t *__restrict__ rowptr = G.rowptr;
        const uint32_t *__restrict__ adj = G.adj;
        const int32_t *__restrict__ toff = G.toff;
        const int2 ab = G.edges[e];
        const int j = min(ab.x, ab.y), i = max(ab.x, ab.y);
        const int ti = G.ntype[i], tj = G.ntype[j];
        const int64_t bi = rowptr[i], bj = rowptr[j];
        const int di = (int)(rowptr[i + 1] - bi), dj = (int)(rowptr[j + 1] - bj);
        const int32_t *toi = toff + (int64_t)i * (L + 1);
        const int32_t *toj = toff + (int64_t)j * (L + 1);

        for (int x = lane; x < BN * P; x += 32) cnt[x] = 0;
        if (lane < 16) {
            Tn[lane] = 0;
            Si[lane] = 0;
            Sj[lane] = 0;
        }
        __syncwarp();
        // Alg. 1
        for (int x = lane; x < di; x += 32) {
            const uint32_t w = __ldg(adj + bi + x);
            if ((int)(w & TG_IDMASK) == j) continue;
            atomicAdd(contains(adj, bj, toj, w) ? &Tn[w >> TG_TSHIFT] : &Si[w >> TG_TSHIFT], 1u);
        }
        for (int x = lane; x < dj; x += 32) {
            const uint32_t w = __ldg(adj + bj + x);
            if ((int)(w & TG_IDMASK) == i) continue;
            if (!contains(adj, bi, toi, w)) atomicAdd(&Sj[w >> TG_TSHIFT], 1u);
        }
        __syncwarp();
        // Alg. 2 and 3 over the flattened lists of 32 w_k at a time
        if (bp.k == 4) {
            for (int side = 0; side < 2; ++side) {
                const int64_t sb = side == 0 ? bi : bj;
                const int sd = side == 0 ? di : dj;
                for (int c0 = 0; c0 < sd; c0 += 32) {
                    const int x = c0 + lane;
                    bool act = x < sd;
                    const uint32_t wk = act ? __ldg(adj + sb + x) : 0u;
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
                                act = false;
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
                        const int gI = cls == CLS_T ? B8 : B3;
                        for (int t2 = 0; t2 < L; ++t2) {
                            int c = __ldg(tk + t2 + 1) - __ldg(tk + t2);
                            if ((cls & 1) && t2 == ti) --c;
                            if ((cls & 2) && t2 == tj) --c;
                            if (c) atomicAdd(&cnt[gI * P + pair_index(L, kt, t2)], c);
                        }
                    }
                    int incl = dk;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(kFull, incl, o);
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
                        const unsigned below = smask & (lane == 31 ? kFull : ((2u << lane) - 1u));
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
                                const int rc = (contains(adj, bi, toi, wr) ? 1 : 0) |
                                               (contains(adj, bj, toj, wr) ? 2 : 0);
                                if (rc != CLS_I) {
                                    const int pr = pair_index(L, okt, (int)(wr >> TG_TSHIFT));
                                    atomicAdd(&cnt[(ocls == CLS_T ? B8 : B3) * P + pr], -1);
                                    if (ocls == CLS_SI) {
                                        if (rc == CLS_SI && rid < okid) atomicAdd(&cnt[B7 * P + pr], 1);
                                    } else if (ocls == CLS_SJ) {
                                        if (rc == CLS_SJ && rid < okid)
                                            atomicAdd(&cnt[B7 * P + pr], 1);
                                        else if (rc == CLS_SI)
                                            atomicAdd(&cnt[B6 * P + pr], 1);
                                    } else {
                                        if (rc == CLS_T) {
                                            if (rid < okid) atomicAdd(&cnt[B12 * P + pr], 1);
                                        } else {
                                            atomicAdd(&cnt[B10 * P + pr], 1);
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
        // closed forms, then the row or the graph's sums
        if (!bp.global) {
            uint64_t *row = G.rows + e * G.width;
            for (int t = lane; t < L; t += 32) {
                row[t] = (uint64_t)Si[t] + Sj[t];
                row[L + t] = Tn[t];
            }
        } else {
            if (lane == 0) {
                int a = ti, b = tj;
                sort2(a, b);
                atomicAdd(G.sums + a + (b + 1) * b / 2, 1ull);
            }
            for (int t = lane; t < L; t += 32) {
                int a = ti, b = tj, c = t;
                sort2(a, b);
                sort2(b, c);
                sort2(a, b);
                const int64_t r = colex3(a, b, c);
                if (Si[t] + Sj[t]) atomicAdd(G.sums + G.off1 + r, (unsigned long long)Si[t] + Sj[t]);
                if (Tn[t]) atomicAdd(G.sums + G.off2 + r, (unsigned long long)Tn[t]);
            }
        }
        if (bp.k == 4) {
            for (int pr = lane; pr < P; pr += 32) {
                int t, u;
                unpair(L, pr, t, u);
                const uint64_t sit = Si[t], siu = Si[u], sjt = Sj[t], sju = Sj[u];
                const uint64_t tt = Tn[t], tu = Tn[u];
                const uint64_t g3 = (uint64_t)(int64_t)cnt[B3 * P + pr];
                const uint64_t g6 = (uint64_t)(int64_t)cnt[B6 * P + pr];
                const uint64_t g7 = (uint64_t)(int64_t)cnt[B7 * P + pr];
                const uint64_t g8 = (uint64_t)(int64_t)cnt[B8 * P + pr];
                const uint64_t g10 = (uint64_t)(int64_t)cnt[B10 * P + pr];
                const uint64_t g12 = (uint64_t)(int64_t)cnt[B12 * P + pr];
                uint64_t g4, g5, g9, g11;
                closed_forms(t == u, sit, siu, sjt, sju, tt, tu, g6, g7, g10, g12, g4, g5, g9, g11);
                if (!bp.global) {
                    uint64_t *row = G.rows + e * G.width + 2 * L;
                    if (bp.level == TG_ORBIT) {
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
                            if (h[q]) atomicAdd(G.sums + G.off4 + q * G.n4 + r, (unsigned long long)h[q]);
                    }
                }
            }
        }
        __syncwarp();
    }
}

// One block row per graph: divide its sums by |E(H)| into its output.
__global__ void k_batch_finalize(const BatchGraph *gs, int32_t G, unsigned *err) {
    const int g = blockIdx.y;
    if (g >= G) return;
    const BatchGraph &B = gs[g];
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < B.glen;
         x += (int64_t)gridDim.x * blockDim.x) {
        uint64_t d = 1;
        if (x >= B.off4) {
            const int64_t q = (x - B.off4) / B.n4;
            d = q < 2 ? 3 : (q < 4 ? 4 : (q == 4 ? 5 : 6));
        } else if (x >= B.off2) {
            d = 3;
        } else if (x >= B.off1) {
            d = 2;
        }
        const uint64_t v = B.sums[x];
        if (v % d) atomicOr(err, 1u);
        B.out[x] = v / d;
    }
}

// Work estimate of item (graph, edge) for the queue order: d_i + d_j plus
// the degree sum of the neighbours of the smaller side (a cheap proxy of the
// Alg. 2-3 walk).
__global__ void k_batch_keys(const BatchGraph *gs, const int64_t *eoff, int32_t G, int64_t count,
                             uint64_t *key, uint32_t *val) {
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < count;
         it += (int64_t)gridDim.x * blockDim.x) {
        const int g = find_graph(eoff, G, it);
        const BatchGraph &B = gs[g];
        const int2 ab = B.edges[it - eoff[g]];
        const int64_t da = B.rowptr[ab.x + 1] - B.rowptr[ab.x];
        const int64_t db = B.rowptr[ab.y + 1] - B.rowptr[ab.y];
        const uint64_t c = (uint64_t)(da * db + da + db);
        const int lb = 64 - __clzll((long long)(c | 1ull));
        uint64_t bucket = (uint64_t)lb * 8ull + ((lb > 3) ? ((c >> (lb - 4)) & 7ull) : 0ull);
        if (bucket > 1023) bucket = 1023;
        key[it] = 1023ull - bucket;
        val[it] = (uint32_t)it;
    }
}


// Inputs of the union of one type-count group: block m copies graph
// members[m]'s canonical edges (original ids offset by noff[m]) to
// src/dst[eoff[m] ..] and its node types to types[noff[m] ..].
__global__ void k_union_inputs(const BatchGraph *gs, const int32_t *members, const int64_t *eoff,
                               const int64_t *noff, int32_t *src, int32_t *dst, uint8_t *types) {
    const int m = blockIdx.x;
    const BatchGraph &B = gs[members[m]];
    const int64_t e0 = eoff[m], n0 = noff[m];
    for (int64_t e = threadIdx.x; e < B.M; e += blockDim.x) {
        const int2 ab = B.edges[e];
        src[e0 + e] = (int32_t)(n0 + B.new2old[ab.x]);
        dst[e0 + e] = (int32_t)(n0 + B.new2old[ab.y]);
    }
    for (int64_t x = threadIdx.x; x < B.n; x += blockDim.x) types[n0 + B.new2old[x]] = B.ntype[x];
}

// Per-edge modes: graph members[m]'s block of the union rows to its output.
__global__ void k_union_scatter(const uint64_t *stage, int64_t width, const BatchGraph *gs,
                                const int32_t *members, const int64_t *eoff) {
    const int m = blockIdx.x;
    const BatchGraph &B = gs[members[m]];
    const uint64_t *src = stage + eoff[m] * width;
    const int64_t words = B.M * width;
    for (int64_t x = threadIdx.x; x < words; x += blockDim.x) B.rows[x] = src[x];
}

// Global mode: graph members[m]'s undivided sums from its block of the union's
// per-edge graphlet rows (k = 3: [h1: L][h2: L]; k = 4: then six blocks of P
// type pairs), each row entry added under the sorted type multiset of the
// edge's endpoints and the slot's types, plus one per edge in the edge block.
// One CTA per graph owns its sums: a shared histogram, then plain stores.
__global__ void k_union_sums(const uint64_t *stage, int64_t width, const int2 *uedges,
                             const uint8_t *untype, const BatchGraph *gs, const int32_t *members,
                             const int64_t *eoff, int k) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *h = reinterpret_cast<unsigned long long *>(smem);
    const int m = blockIdx.x;
    const BatchGraph &B = gs[members[m]];
    const int L = B.L, P = B.P;
    for (int64_t x = threadIdx.x; x < B.glen; x += blockDim.x) h[x] = 0ull;
    __syncthreads();
    const int64_t e0 = eoff[m], ne = eoff[m + 1] - e0;
    for (int64_t q = threadIdx.x; q < ne * width; q += blockDim.x) {
        const int64_t e = e0 + q / width;
        const int sl = (int)(q % width);
        const int2 ab = uedges[e];
        const int ti = untype[ab.x], tj = untype[ab.y];
        if (sl == 0) {
            int a = ti, b = tj;
            sort2(a, b);
            atomicAdd(h + (int64_t)a + (int64_t)(b + 1) * b / 2, 1ull);
        }
        const uint64_t v = stage[e * width + sl];
        if (!v) continue;
        int64_t idx;
        if (sl < 2 * L) {
            int a = ti, b = tj, c = sl % L;
            sort2(a, b);
            sort2(b, c);
            sort2(a, b);
            idx = (sl < L ? B.off1 : B.off2) + colex3(a, b, c);
        } else {
            const int r = sl - 2 * L, blk = r / P;
            int t, u;
            unpair(L, r % P, t, u);
            int a = ti, b = tj, c = t, d = u;
            sort2(a, b);
            sort2(c, d);
            sort2(a, c);
            sort2(b, d);
            sort2(b, c);
            idx = B.off4 + blk * B.n4 + colex4(a, b, c, d);
        }
        atomicAdd(h + idx, (unsigned long long)v);
    }
    (void)k;
    __syncthreads();
    for (int64_t x = threadIdx.x; x < B.glen; x += blockDim.x) B.sums[x] = h[x];
}

}  // namespace

struct UnionGroup {
    int32_t L = 0;
    int32_t nm = 0;             // member graphs
    tg_graph *U = nullptr;      // their disjoint union
    int32_t *d_members = nullptr;
    int64_t *d_eoff = nullptr;  // nm + 1 edge offsets in the union
    int64_t width = 0;          // row width of the union count
};

struct tg_batch {
    int32_t G = 0, k = 4, mode = TG_BATCH_GLOBAL, Pmax = 1;
    int64_t count = 0;
    BatchGraph *d_gs = nullptr;
    int64_t *d_eoff = nullptr;
    uint32_t *d_order = nullptr;
    unsigned long long *d_queue = nullptr;
    unsigned long long *d_sums = nullptr;
    int64_t sums_len = 0;
    unsigned *d_err = nullptr;
    int warps = 8;
    int ordered = 1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool no_graph = false;  // enqueue the launches directly instead of replaying a graph
    std::vector<UnionGroup> groups;  // union path (empty when not built)
    uint64_t *d_stage = nullptr;     // union rows of the largest group
    size_t stage_words = 0;
    bool use_union = false;
    std::mutex mu;
};

static void batch_release(tg_batch *b) {
    if (!b) return;
    (void)cudaDeviceSynchronize();
    if (b->exec) (void)cudaGraphExecDestroy(b->exec);
    if (b->graph) (void)cudaGraphDestroy(b->graph);
    tg_dfree(b->d_gs, 0, nullptr);
    tg_dfree(b->d_eoff, 0, nullptr);
    tg_dfree(b->d_order, 0, nullptr);
    tg_dfree(b->d_queue, 0, nullptr);
    tg_dfree(b->d_sums, 0, nullptr);
    tg_dfree(b->d_err, 0, nullptr);
    for (UnionGroup &u : b->groups) {
        tg_free_graph(u.U);
        tg_dfree(u.d_members, 0, nullptr);
        tg_dfree(u.d_eoff, 0, nullptr);
    }
    tg_dfree(b->d_stage, 0, nullptr);
    (void)cudaDeviceSynchronize();
    delete b;
}

// Launch shape of the persistent kernel for the plan's current warps per CTA
// (attribute and occupancy queries stay outside stream capture).
static int batch_config(tg_batch *b, int64_t *grid, size_t *smem) {
    const int threads = b->warps * 32;
    const size_t wbytes = ((size_t)BN * b->Pmax * 4 + 3 * 16 * 4 + 32 * 4 + 15) & ~(size_t)15;
    *smem = (size_t)b->warps * wbytes;
    TG_TRY(tg_allow_max_smem((const void *)k_batch_warp));
    int per_sm = 0;
    TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_warp, threads, *smem));
    if (per_sm < 1) per_sm = 1;
    int64_t gr = (int64_t)tg_num_sms() * per_sm;
    const int64_t need = (b->count + b->warps - 1) / b->warps;
    if (gr > need) gr = need;
    *grid = gr < 1 ? 1 : gr;
    return TG_OK;
}

// Enqueue one run (reset, persistent count, finalize) on stream s.  `note`:
// count the launches (false while capturing: a replay counts them).
static int batch_enqueue(tg_batch *b, cudaStream_t s, int64_t grid, size_t smem, bool note = true) {
    TG_TRY_CUDA(cudaMemsetAsync(b->d_queue, 0, 8, s));
    if (b->mode == TG_BATCH_GLOBAL) {
        TG_TRY_CUDA(cudaMemsetAsync(b->d_sums, 0, (size_t)b->sums_len * 8, s));
        TG_TRY_CUDA(cudaMemsetAsync(b->d_err, 0, 4, s));
    }
    if (b->count > 0) {
        BatchParams p{};
        p.gs = b->d_gs;
        p.eoff = b->d_eoff;
        p.order = b->ordered ? b->d_order : nullptr;
        p.G = b->G;
        p.count = b->count;
        p.k = b->k;
        p.level = b->mode == TG_BATCH_PER_EDGE_ORBIT ? TG_ORBIT : TG_GRAPHLET;
        p.global = b->mode == TG_BATCH_GLOBAL;
        p.Pmax = b->Pmax;
        p.queue = b->d_queue;
        k_batch_warp<<<(unsigned)grid, b->warps * 32, smem, s>>>(p);
        if (note) tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    if (b->mode == TG_BATCH_GLOBAL && b->G > 0) {
        dim3 grid(4, (unsigned)b->G);
        k_batch_finalize<<<grid, 256, 0, s>>>(b->d_gs, b->G, b->d_err);
        if (note) tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    return TG_OK;
}

static int batch_capture(tg_batch *b, cudaStream_t s) {
    if (b->exec) {
        (void)cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        (void)cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    int64_t grid = 1;
    size_t smem = 0;
    TG_TRY(batch_config(b, &grid, &smem));
    cudaStream_t cs = nullptr;
    TG_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    int r = TG_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        r = TG_ECUDA;
    } else {
        const int r2 = batch_enqueue(b, cs, grid, smem, false);
        const cudaError_t e = cudaStreamEndCapture(cs, &b->graph);
        if (r2 != TG_OK) r = r2;
        else if (e != cudaSuccess) r = TG_ECUDA;
        else if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) r = TG_ECUDA;
    }
    (void)cudaStreamDestroy(cs);
    (void)cudaGetLastError();
    (void)s;
    return r;
}

// Build the union of each type-count group (host vectors hg: descriptors as
// copied to b->d_gs).  Any failure leaves the plan without the union path.
static int build_union(tg_batch *b, tg_graph *const *gs, const std::vector<BatchGraph> &hg,
                       cudaStream_t s) {
    std::vector<std::vector<int32_t>> byL(TG_MAX_TYPES + 1);
    for (int g = 0; g < b->G; ++g) byL[hg[g].L].push_back(g);
    const int level = b->mode == TG_BATCH_PER_EDGE_ORBIT ? TG_ORBIT : TG_GRAPHLET;
    for (int L = 1; L <= TG_MAX_TYPES; ++L) {
        const std::vector<int32_t> &mem = byL[L];
        if (mem.empty()) continue;
        UnionGroup u;
        u.L = L;
        u.nm = (int32_t)mem.size();
        std::vector<int64_t> eoff(mem.size() + 1, 0), noff(mem.size() + 1, 0);
        for (size_t q = 0; q < mem.size(); ++q) {
            eoff[q + 1] = eoff[q] + gs[mem[q]]->M;
            noff[q + 1] = noff[q] + gs[mem[q]]->n;
        }
        if (noff.back() > TG_MAX_NODES || eoff.back() >= ((int64_t)1 << 31)) return TG_EOVERFLOW;
        u.width = tg_slots(L, b->k, level);
        u.d_members = (int32_t *)tg_dalloc(mem.size() * 4, s);
        u.d_eoff = (int64_t *)tg_dalloc((mem.size() + 1) * 8, s);
        if (!u.d_members || !u.d_eoff) {
            tg_dfree(u.d_members, 0, s);
            tg_dfree(u.d_eoff, 0, s);
            return TG_ENOMEM;
        }
        b->groups.push_back(u);  // released with the plan from here on
        TG_TRY_CUDA(cudaMemcpyAsync(u.d_members, mem.data(), mem.size() * 4, cudaMemcpyHostToDevice, s));
        TG_TRY_CUDA(cudaMemcpyAsync(u.d_eoff, eoff.data(), (mem.size() + 1) * 8, cudaMemcpyHostToDevice, s));
        DevBuf<int64_t> dnoff;
        DevBuf<int32_t> src, dst;
        DevBuf<uint8_t> types;
        if (!dnoff.alloc(mem.size() + 1, s) || !src.alloc(std::max<int64_t>(1, eoff.back()), s) ||
            !dst.alloc(std::max<int64_t>(1, eoff.back()), s) || !types.alloc(noff.back(), s))
            return TG_ENOMEM;
        TG_TRY_CUDA(cudaMemcpyAsync(dnoff.p, noff.data(), (mem.size() + 1) * 8, cudaMemcpyHostToDevice, s));
        k_union_inputs<<<(unsigned)mem.size(), 256, 0, s>>>(b->d_gs, u.d_members, u.d_eoff, dnoff.p,
                                                            src.p, dst.p, types.p); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
        tg_graph *U = nullptr;
        TG_TRY(tg_build_csr(noff.back(), eoff.back(), src.p, dst.p, types.p, L, TG_INPUT_DEVICE, s, &U));
        b->groups.back().U = U;
        if (U->M != eoff.back()) return TG_EINTERNAL;  // graphs of a union never share an edge
        b->stage_words = std::max(b->stage_words, (size_t)U->M * (size_t)u.width);
    }
    b->d_stage = (uint64_t *)tg_dalloc(std::max<size_t>(1, b->stage_words) * 8, s);
    if (!b->d_stage) return TG_ENOMEM;
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}

// One run through the unions: per group the whole-graph per-edge count, then
// the rows out per graph, or (global mode) the per-graph sums and the division.
static int union_run(tg_batch *b, cudaStream_t s) {
    const int level = b->mode == TG_BATCH_PER_EDGE_ORBIT ? TG_ORBIT : TG_GRAPHLET;
    for (const UnionGroup &u : b->groups) {
        if (u.U->M > 0) TG_TRY(tg_rows_device(u.U, b->k, level, b->d_stage, s));
        if (b->mode == TG_BATCH_GLOBAL) {
            const size_t smem = (size_t)tg_global_len(u.L, b->k) * 8;
            TG_TRY(tg_allow_max_smem((const void *)k_union_sums));
            k_union_sums<<<(unsigned)u.nm, 512, smem, s>>>(b->d_stage, u.width, u.U->edges, u.U->ntype,
                                                           b->d_gs, u.d_members, u.d_eoff, b->k);
        } else {
            k_union_scatter<<<(unsigned)u.nm, 512, 0, s>>>(b->d_stage, u.width, b->d_gs, u.d_members,
                                                           u.d_eoff);
        }
        tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    if (b->mode == TG_BATCH_GLOBAL && b->G > 0) {
        TG_TRY_CUDA(cudaMemsetAsync(b->d_err, 0, 4, s));
        dim3 grid(4, (unsigned)b->G);
        k_batch_finalize<<<grid, 256, 0, s>>>(b->d_gs, b->G, b->d_err); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    return TG_OK;
}

extern "C" int tg_batch_create(int32_t G, tg_graph *const *gs, int32_t k, int32_t mode,
                               uint64_t *const *outs, const tg_tune *tune, void *stream,
                               tg_batch **out) {
    if (!out || G < 0 || (G > 0 && (!gs || !outs)) || (k != 3 && k != 4)) return TG_EINVAL;
    if (mode != TG_BATCH_GLOBAL && mode != TG_BATCH_PER_EDGE_GRAPHLET &&
        mode != TG_BATCH_PER_EDGE_ORBIT)
        return TG_EINVAL;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    tg_batch *b = new (std::nothrow) tg_batch();
    if (!b) return TG_ENOMEM;
    b->G = G;
    b->k = k;
    b->mode = mode;
    if (tune && tune->cta_threads >= 32 && tune->cta_threads <= 1024 && tune->cta_threads % 32 == 0)
        b->warps = tune->cta_threads / 32;
    std::vector<BatchGraph> hg((size_t)G);
    std::vector<int64_t> eoff((size_t)G + 1, 0);
    std::vector<int64_t> soff((size_t)G, 0);
    int64_t sums = 0;
    int Lmax = 1;
    for (int g = 0; g < G; ++g) {
        const tg_graph *x = gs[g];
        if (!x || !outs[g]) {
            delete b;
            return TG_EINVAL;
        }
        if (2 * x->M >= ((int64_t)1 << 31) || 32 * x->max_degree >= ((int64_t)1 << 31)) {
            delete b;
            return TG_EOVERFLOW;
        }
        if (!tg_is_device_ptr(outs[g])) {
            delete b;
            return TG_EINVAL;  // the persistent launch writes device memory only
        }
        BatchGraph &B = hg[g];
        const int L = x->L;
        B.new2old = x->new2old;
        B.n = x->n;
        B.M = x->M;
        B.rowptr = x->rowptr;
        B.adj = x->adj;
        B.toff = x->toff;
        B.ntype = x->ntype;
        B.edges = x->edges;
        B.L = L;
        B.P = L * (L + 1) / 2;
        B.off1 = tg_binom(L + 1, 2);
        B.off2 = B.off1 + tg_binom(L + 2, 3);
        B.off4 = B.off1 + 2 * tg_binom(L + 2, 3);
        B.n4 = tg_binom(L + 3, 4);
        B.glen = tg_global_len(L, k);
        if (mode == TG_BATCH_GLOBAL) {
            B.out = outs[g];
            soff[g] = sums;
            sums += B.glen;
        } else {
            B.rows = outs[g];
            B.width = tg_slots(L, k, mode == TG_BATCH_PER_EDGE_ORBIT ? TG_ORBIT : TG_GRAPHLET);
        }
        Lmax = std::max(Lmax, L);
        eoff[g + 1] = eoff[g] + x->M;
    }
    b->count = eoff[G];
    b->Pmax = Lmax * (Lmax + 1) / 2;
    if (b->count >= (int64_t)UINT32_MAX) {
        delete b;
        return TG_EOVERFLOW;
    }
    b->sums_len = sums;
    auto fail = [&](int r) {
        batch_release(b);
        return r;
    };
    b->d_gs = (BatchGraph *)tg_dalloc(sizeof(BatchGraph) * (size_t)(G > 0 ? G : 1), s);
    b->d_eoff = (int64_t *)tg_dalloc(sizeof(int64_t) * (size_t)(G + 1), s);
    b->d_order = (uint32_t *)tg_dalloc(sizeof(uint32_t) * (size_t)(b->count > 0 ? b->count : 1), s);
    b->d_queue = (unsigned long long *)tg_dalloc(8, s);
    b->d_err = (unsigned *)tg_dalloc(4, s);
    b->d_sums = (unsigned long long *)tg_dalloc((size_t)(sums > 0 ? sums : 1) * 8, s);
    if (!b->d_gs || !b->d_eoff || !b->d_order || !b->d_queue || !b->d_err || !b->d_sums)
        return fail(TG_ENOMEM);
    if (mode == TG_BATCH_GLOBAL)
        for (int g = 0; g < G; ++g) hg[g].sums = b->d_sums + soff[g];
    if (G > 0) {
        if (cudaMemcpyAsync(b->d_gs, hg.data(), sizeof(BatchGraph) * G, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(b->d_eoff, eoff.data(), sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice,
                            s) != cudaSuccess)
            return fail(TG_ECUDA);
    }
    if (b->count > 0) {
        DevBuf<uint64_t> k1, k2;
        DevBuf<uint32_t> v2;
        if (!k1.alloc(b->count, s) || !k2.alloc(b->count, s) || !v2.alloc(b->count, s))
            return fail(TG_ENOMEM);
        const int64_t blocks = std::min<int64_t>((b->count + 255) / 256, 65535LL * 16);
        k_batch_keys<<<(unsigned)blocks, 256, 0, s>>>(b->d_gs, b->d_eoff, G, b->count, k1.p,
                                                      b->d_order); tg_note_launch();
        if (cudaGetLastError() != cudaSuccess) return fail(TG_ECUDA);
        uint64_t *rk = nullptr;
        uint32_t *rv = nullptr;
        int r = tg_radix_sort_kv(k1.p, k2.p, b->d_order, v2.p, b->count, 10, s, &rk, &rv);
        if (r != TG_OK) return fail(r);
        if (rv != b->d_order &&
            cudaMemcpyAsync(b->d_order, rv, b->count * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(TG_ECUDA);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(TG_ECUDA);
    // union path: built unless the tuning asks for the persistent warp kernel
    const int kern = tune ? tune->kernel : TG_KERNEL_AUTO;
    if (kern != TG_KERNEL_WARP_SEARCH && G > 0) {
        const int ur = build_union(b, gs, hg, s);
        if (ur != TG_OK && kern == TG_KERNEL_CYCLES) return fail(ur);  // the union was asked for
        if (ur == TG_OK) {
            b->use_union = true;
        } else {
            (void)cudaGetLastError();
            (void)cudaStreamSynchronize(s);
            for (UnionGroup &u : b->groups) {
                tg_free_graph(u.U);
                tg_dfree(u.d_members, 0, s);
                tg_dfree(u.d_eoff, 0, s);
            }
            b->groups.clear();
            tg_dfree(b->d_stage, 0, s);
            b->d_stage = nullptr;
            (void)cudaStreamSynchronize(s);
        }
    }
    *out = b;
    return TG_OK;
}

extern "C" int tg_batch_run(tg_batch *b, void *stream) {
    if (!b) return TG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(b->mu);
    // the union path; else a replay of the captured graph, and when a capture
    // cannot be made (or the plan asks for none) the same launches directly
    if (!b->use_union && !b->exec && !b->no_graph && batch_capture(b, s) != TG_OK)
        b->no_graph = true;
    if (b->use_union) {
        TG_TRY(union_run(b, s));
    } else if (b->exec && !b->no_graph) {
        TG_TRY_CUDA(cudaGraphLaunch(b->exec, s));
        if (b->count > 0) tg_note_launch();                      // persistent count kernel
        if (b->mode == TG_BATCH_GLOBAL && b->G > 0) tg_note_launch();  // finalize
    } else {
        int64_t grid = 1;
        size_t smem = 0;
        TG_TRY(batch_config(b, &grid, &smem));
        TG_TRY(batch_enqueue(b, s, grid, smem));
    }
    if (b->mode == TG_BATCH_GLOBAL) {
        unsigned herr = 0;
        TG_TRY_CUDA(cudaMemcpyAsync(&herr, b->d_err, 4, cudaMemcpyDeviceToHost, s));
        TG_TRY_CUDA(cudaStreamSynchronize(s));
        if (herr) return TG_EINTERNAL;
    } else {
        TG_TRY_CUDA(cudaStreamSynchronize(s));
    }
    return TG_OK;
}

extern "C" int tg_batch_tune(tg_batch *b, void *stream, int32_t *best_threads) {
    if (!b) return TG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(b->mu);
    cudaEvent_t e0, e1;
    TG_TRY_CUDA(cudaEventCreate(&e0));
    TG_TRY_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bw = b->warps, bo = b->ordered;
    const int cand_w[3] = {4, 8, 16};
    int r = TG_OK;
    for (int o = 1; o >= 0 && r == TG_OK; --o)
        for (int c = 0; c < 3 && r == TG_OK; ++c) {
            b->warps = cand_w[c];
            b->ordered = o;
            int64_t grid = 1;
            size_t smem = 0;
            r = batch_config(b, &grid, &smem);
            if (r != TG_OK) break;
            r = batch_enqueue(b, s, grid, smem);  // warm
            if (r != TG_OK) break;
            if (cudaEventRecord(e0, s) != cudaSuccess) { r = TG_ECUDA; break; }
            r = batch_enqueue(b, s, grid, smem);
            if (r != TG_OK) break;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                r = TG_ECUDA;
                break;
            }
            float ms = 0;
            (void)cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bw = b->warps;
                bo = o;
            }
        }
    // the union path, when the plan has one
    bool uni = false;
    if (r == TG_OK && !b->groups.empty()) {
        r = union_run(b, s);  // warm
        if (r == TG_OK && cudaEventRecord(e0, s) != cudaSuccess) r = TG_ECUDA;
        if (r == TG_OK) r = union_run(b, s);
        if (r == TG_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
            r = TG_ECUDA;
        if (r == TG_OK) {
            float ms = 0;
            (void)cudaEventElapsedTime(&ms, e0, e1);
            uni = ms < best;
        }
    }
    (void)cudaEventDestroy(e0);
    (void)cudaEventDestroy(e1);
    b->warps = bw;
    b->ordered = bo;
    b->use_union = uni;
    if (r != TG_OK) return r;
    // the chosen configuration as a graph (runs enqueue directly if it fails)
    if (!uni && !b->no_graph && batch_capture(b, s) != TG_OK) b->no_graph = true;
    if (best_threads) *best_threads = uni ? 0 : bw * 32 * (bo ? 1 : -1);
    return TG_OK;
}

extern "C" int tg_batch_destroy(tg_batch *b) {
    batch_release(b);
    return TG_OK;
}

extern "C" int tg_count_batch(int32_t G, tg_graph *const *gs, int32_t k, int32_t mode,
                              uint64_t *const *outs, const tg_tune *tune, void *stream) {
    tg_batch *b = nullptr;
    TG_TRY(tg_batch_create(G, gs, k, mode, outs, tune, stream, &b));
    int r = tune ? TG_OK : tg_batch_tune(b, stream, nullptr);
    b->no_graph = true;  // one run: a graph would only add the capture
    if (r == TG_OK) r = tg_batch_run(b, stream);
    tg_batch_destroy(b);
    return r;
}
