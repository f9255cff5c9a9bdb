// Typed CSR builder (graph model of Def. "Heterogeneous network" and the
// typed neighbourhoods Gamma_i^t of Def. "Typed Neighborhood").
//
// Pipeline, all on the device with this library's own kernels:
//   1. canonical keys lo*n + hi for every non-loop input pair (validation of
//      ids and types on the way);
//   2. radix sort + unique -> the canonical edge list in original ids;
//   3. degrees, then a relabel by degree (descending, ties by original id),
//      so high-degree nodes get small ids and, for an edge, the endpoint with
//      the larger new id never has the larger degree (the d_i <= d_j
//      orientation of Thm. "3-node time complexity");
//   4. one radix sort of the 2M directed entries keyed (src, type, dst) gives
//      every adjacency list sorted by (type, id); entries are stored packed
//      as (type << 28) | id;
//   5. per-node type offsets toff[v][t] (start of Gamma_v^t inside row v).
#include <stdlib.h>

#include "tg_internal.cuh"

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > (int64_t)1 << 30) b = (int64_t)1 << 30;
    return (unsigned)b;
}

__global__ void k_check_types(const uint8_t *type, int64_t n, int32_t L, unsigned *err) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (type[v] >= L) atomicOr(err, TG_DERR_INPUT);
}

__global__ void k_canon_keys(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                             uint64_t *key, unsigned *err) {
    const uint64_t sentinel = (uint64_t)n * (uint64_t)n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = src[e], b = dst[e];
        uint64_t k = sentinel;
        if (a < 0 || a >= n || b < 0 || b >= n) {
            atomicOr(err, TG_DERR_INPUT);
        } else if (a != b) {
            int64_t lo = a < b ? a : b, hi = a < b ? b : a;
            k = (uint64_t)lo * (uint64_t)n + (uint64_t)hi;
        }
        key[e] = k;
    }
}

__global__ void k_unique_flags(const uint64_t *key, int64_t m, uint64_t sentinel,
                               uint32_t *flag) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        flag[e] = (key[e] != sentinel && (e == 0 || key[e] != key[e - 1])) ? 1u : 0u;
}

__global__ void k_compact_edges(const uint64_t *key, const uint32_t *flag, const uint32_t *pos,
                                int64_t m, int64_t n, int32_t *lo, int32_t *hi, int32_t *deg) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const bool keep = flag[e] != 0;
        uint64_t k = keep ? key[e] : 0ull;
        int32_t a = (int32_t)(k / (uint64_t)n), b = (int32_t)(k % (uint64_t)n);
        if (keep) {
            lo[pos[e]] = a;
            hi[pos[e]] = b;
            atomicAdd(&deg[b], 1);
        }
        // the keys are sorted, so the lanes holding one lower end a are
        // adjacent: one add of their number per a (a hub's edges no longer
        // queue on one counter)
        const unsigned peers = __match_any_sync(__activemask(), keep ? a : -1);
        if (keep && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&deg[a], __popc(peers));
    }
}

__global__ void k_max_deg(const int32_t *deg, int64_t n, unsigned long long *mx,
                          unsigned long long *nonisolated) {
    unsigned long long local = 0, cnt = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long d = (unsigned long long)deg[v];
        local = d > local ? d : local;
        cnt += d > 0;
    }
    for (int o = 16; o; o >>= 1) {
        unsigned long long y = __shfl_down_sync(0xffffffffu, local, o);
        local = y > local ? y : local;
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(mx, local);
        atomicAdd(nonisolated, cnt);
    }
}

__global__ void k_relabel_keys(const int32_t *deg, int64_t n, int64_t maxdeg, int idbits,
                               uint64_t *key) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        key[v] = ((uint64_t)(maxdeg - deg[v]) << idbits) | (uint64_t)v;
}

__global__ void k_apply_relabel(const uint64_t *key, int64_t n, uint64_t idmask,
                                const int32_t *deg, const uint8_t *type, int32_t *new2old,
                                int32_t *old2new, int64_t *ndeg, uint8_t *ntype) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = (int32_t)(key[p] & idmask);
        new2old[p] = v;
        old2new[v] = (int32_t)p;
        ndeg[p] = deg[v];
        ntype[p] = type[v];
    }
}

// Directed entries keyed (src << (tb + nb)) | (type(dst) << nb) | dst.
__global__ void k_directed_keys(const int32_t *lo, const int32_t *hi, int64_t M,
                                const int32_t *old2new, const uint8_t *ntype, int nb, int tb,
                                uint64_t *key, uint32_t *val, int2 *edges) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < M;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t a = (uint64_t)old2new[lo[e]], b = (uint64_t)old2new[hi[e]];
        key[2 * e] = (a << (tb + nb)) | ((uint64_t)ntype[b] << nb) | b;
        key[2 * e + 1] = (b << (tb + nb)) | ((uint64_t)ntype[a] << nb) | a;
        val[2 * e] = (uint32_t)e;
        val[2 * e + 1] = (uint32_t)e;
        edges[e] = make_int2((int)a, (int)b);
    }
}

// Packs the sorted entries and records the type boundaries of each row.
__global__ void k_fill_adj(const uint64_t *key, const uint32_t *val, int64_t total, int nb,
                           int tb, int32_t L, const int64_t *rowptr, uint32_t *adj,
                           uint32_t *eid, int32_t *toff) {
    const uint64_t nmask = ((uint64_t)1 << nb) - 1, tmask = ((uint64_t)1 << tb) - 1;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = key[x];
        int64_t v = (int64_t)(k >> (tb + nb));
        int32_t t = (int32_t)((k >> nb) & tmask);
        uint32_t id = (uint32_t)(k & nmask);
        adj[x] = ((uint32_t)t << TG_TSHIFT) | id;
        eid[x] = val[x];
        int64_t r0 = rowptr[v], r1 = rowptr[v + 1];
        int32_t tp = -1;
        if (x > r0) tp = (int32_t)((key[x - 1] >> nb) & tmask);
        int32_t *to = toff + v * (L + 1);
        for (int32_t q = tp + 1; q <= t; ++q) to[q] = (int32_t)(x - r0);
        if (x == r1 - 1)
            for (int32_t q = t + 1; q <= L; ++q) to[q] = (int32_t)(r1 - r0);
    }
}

int build_impl(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
               const uint8_t *type, int32_t L, uint32_t flags, cudaStream_t s, tg_graph **out) {
    if (!out) return TG_EINVAL;
    *out = nullptr;
    if (n < 1 || n > TG_MAX_NODES || m < 0 || m >= ((int64_t)1 << 31) || L < 1 ||
        L > TG_MAX_TYPES)
        return TG_EINVAL;
    if (m > 0 && (!src || !dst)) return TG_EINVAL;
    if (!type) return TG_EINVAL;
    const bool on_dev = (flags & TG_INPUT_DEVICE) != 0;

    DevBuf<unsigned> err;
    if (!err.alloc(4, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(err.p, 0, 4 * sizeof(unsigned), s));

    // Inputs on the device.
    DevBuf<int32_t> dsrc, ddst;
    DevBuf<uint8_t> dtype;
    const int32_t *psrc = src, *pdst = dst;
    const uint8_t *ptype = type;
    if (!on_dev) {
        if (!dsrc.alloc(m, s) || !ddst.alloc(m, s) || !dtype.alloc(n, s)) return TG_ENOMEM;
        if (m > 0) {
            TG_TRY_CUDA(cudaMemcpyAsync(dsrc.p, src, m * 4, cudaMemcpyHostToDevice, s));
            TG_TRY_CUDA(cudaMemcpyAsync(ddst.p, dst, m * 4, cudaMemcpyHostToDevice, s));
        }
        TG_TRY_CUDA(cudaMemcpyAsync(dtype.p, type, n, cudaMemcpyHostToDevice, s));
        psrc = dsrc.p;
        pdst = ddst.p;
        ptype = dtype.p;
    }
    k_check_types<<<grid_for(n), kThreads, 0, s>>>(ptype, n, L, err.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());

    // 1-2. canonical keys, sort, unique.
    DevBuf<uint64_t> k1, k2;
    if (!k1.alloc(m, s) || !k2.alloc(m, s)) return TG_ENOMEM;
    const uint64_t sentinel = (uint64_t)n * (uint64_t)n;
    uint64_t *sorted = k1.p;
    if (m > 0) {
        k_canon_keys<<<grid_for(m), kThreads, 0, s>>>(psrc, pdst, m, n, k1.p, err.p); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
        TG_TRY(tg_radix_sort_u64(k1.p, k2.p, m, tg_bitlen(sentinel), s, &sorted));
    }
    DevBuf<uint32_t> flag, pos;
    if (!flag.alloc(m, s) || !pos.alloc(m, s)) return TG_ENOMEM;
    uint32_t last[2] = {0, 0};
    if (m > 0) {
        k_unique_flags<<<grid_for(m), kThreads, 0, s>>>(sorted, m, sentinel, flag.p); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
        TG_TRY(tg_scan_u32(flag.p, pos.p, m, s));
        TG_TRY_CUDA(cudaMemcpyAsync(&last[0], pos.p + (m - 1), 4, cudaMemcpyDeviceToHost, s));
        TG_TRY_CUDA(cudaMemcpyAsync(&last[1], flag.p + (m - 1), 4, cudaMemcpyDeviceToHost, s));
    }
    unsigned herr = 0;
    TG_TRY_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    if (herr & TG_DERR_INPUT) return TG_EINVAL;
    const int64_t M = (int64_t)last[0] + (int64_t)last[1];

    tg_graph *g = new (std::nothrow) tg_graph();
    if (!g) return TG_ENOMEM;
    g->n = n;
    g->m_input = m;
    g->M = M;
    g->L = L;
    (void)cudaGetDevice(&g->device);
    struct Guard {
        tg_graph *g;
        cudaStream_t s;
        ~Guard() {
            if (g) {
                tg_dfree(g->rowptr, 0, s);
                tg_dfree(g->adj, 0, s);
                tg_dfree(g->toff, 0, s);
                tg_dfree(g->ntype, 0, s);
                tg_dfree(g->edges, 0, s);
                tg_dfree(g->new2old, 0, s);
                tg_dfree(g->eid, 0, s);
                tg_dfree(g->adir, 0, s);
                delete g;
            }
        }
    } guard{g, s};

    DevBuf<int32_t> lo, hi, deg;
    if (!lo.alloc(M, s) || !hi.alloc(M, s) || !deg.alloc(n, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(deg.p, 0, n * 4, s));
    if (m > 0) {
        k_compact_edges<<<grid_for(m), kThreads, 0, s>>>(sorted, flag.p, pos.p, m, n, lo.p, hi.p,
                                                         deg.p); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    k1.reset();
    k2.reset();
    flag.reset();
    pos.reset();

    // 3. relabel by degree.
    DevBuf<unsigned long long> stats;
    if (!stats.alloc(2, s)) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(stats.p, 0, 2 * sizeof(unsigned long long), s));
    k_max_deg<<<grid_for(n), kThreads, 0, s>>>(deg.p, n, stats.p, stats.p + 1); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    unsigned long long hstats[2] = {0, 0};
    TG_TRY_CUDA(cudaMemcpyAsync(hstats, stats.p, sizeof(hstats), cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    g->max_degree = (int64_t)hstats[0];
    g->n_nonisolated = (int64_t)hstats[1];

    const int nb = tg_bitlen((uint64_t)(n - 1)) > 0 ? tg_bitlen((uint64_t)(n - 1)) : 1;
    const int tb = tg_bitlen((uint64_t)(L - 1)) > 0 ? tg_bitlen((uint64_t)(L - 1)) : 1;
    DevBuf<uint64_t> r1, r2;
    if (!r1.alloc(n, s) || !r2.alloc(n, s)) return TG_ENOMEM;
    k_relabel_keys<<<grid_for(n), kThreads, 0, s>>>(deg.p, n, g->max_degree, nb, r1.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    uint64_t *rs = r1.p;
    TG_TRY(tg_radix_sort_u64(r1.p, r2.p, n, nb + tg_bitlen((uint64_t)g->max_degree), s, &rs));

    DevBuf<int32_t> old2new;
    DevBuf<int64_t> ndeg;
    if (!old2new.alloc(n, s) || !ndeg.alloc(n + 1, s)) return TG_ENOMEM;
    g->new2old = (int32_t *)tg_dalloc(n * 4, s);
    g->ntype = (uint8_t *)tg_dalloc(n, s);
    g->rowptr = (int64_t *)tg_dalloc((n + 1) * 8, s);
    if (!g->new2old || !g->ntype || !g->rowptr) return TG_ENOMEM;
    k_apply_relabel<<<grid_for(n), kThreads, 0, s>>>(rs, n, ((uint64_t)1 << nb) - 1, deg.p,
                                                     ptype, g->new2old, old2new.p, ndeg.p,
                                                     g->ntype); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    TG_TRY_CUDA(cudaMemsetAsync(ndeg.p + n, 0, 8, s));
    TG_TRY(tg_scan_i64(ndeg.p, g->rowptr, n + 1, s));
    r1.reset();
    r2.reset();
    deg.reset();
    ndeg.reset();

    // 4. adjacency sorted by (type, id).
    const int64_t total = 2 * M;
    g->adj = (uint32_t *)tg_dalloc((total > 0 ? total : 1) * 4, s);
    g->edges = (int2 *)tg_dalloc((M > 0 ? M : 1) * sizeof(int2), s);
    g->toff = (int32_t *)tg_dalloc(n * (L + 1) * 4, s);
    g->eid = (uint32_t *)tg_dalloc((total > 0 ? total : 1) * 4, s);
    if (!g->adj || !g->edges || !g->toff || !g->eid) return TG_ENOMEM;
    TG_TRY_CUDA(cudaMemsetAsync(g->toff, 0, n * (L + 1) * 4, s));
    if (M > 0) {
        DevBuf<uint64_t> d1, d2;
        DevBuf<uint32_t> v1, v2;
        if (!d1.alloc(total, s) || !d2.alloc(total, s) || !v1.alloc(total, s) ||
            !v2.alloc(total, s))
            return TG_ENOMEM;
        k_directed_keys<<<grid_for(M), kThreads, 0, s>>>(lo.p, hi.p, M, old2new.p, g->ntype, nb,
                                                         tb, d1.p, v1.p, g->edges); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
        uint64_t *ds = d1.p;
        uint32_t *vs = v1.p;
        TG_TRY(tg_radix_sort_kv(d1.p, d2.p, v1.p, v2.p, total, 2 * nb + tb, s, &ds, &vs));
        k_fill_adj<<<grid_for(total), kThreads, 0, s>>>(ds, vs, total, nb, tb, L, g->rowptr,
                                                        g->adj, g->eid, g->toff); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    if (flags & TG_DIRECTED) TG_TRY(tg_attach_arcs(g, psrc, pdst, m, old2new.p, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    TG_TRY_CUDA(cudaGetLastError());
    g->device_bytes = (n + 1) * 8 + 2 * total * 4 + n * (L + 1) * 4 + n + M * 8 + n * 4 +
                      ((flags & TG_DIRECTED) ? ((2 * M + 3) & ~(int64_t)3) : 0);
    guard.g = nullptr;
    *out = g;
    return TG_OK;
}

}  // namespace

extern "C" int tg_build_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                            const uint8_t *type, int32_t L, uint32_t flags, void *stream,
                            tg_graph **out) {
    cudaStream_t s = (cudaStream_t)stream;
    int r = build_impl(n, m, src, dst, type, L, flags, s, out);
    if (r != TG_OK) (void)cudaStreamSynchronize(s);
    return r;
}

extern "C" int tg_free_graph(tg_graph *g) {
    if (!g) return TG_OK;
    // the graph may still be read by kernels on any stream
    (void)cudaDeviceSynchronize();
    tg_sched_free(g);
    cudaStream_t s = nullptr;
    tg_dfree(g->rowptr, 0, s);
    tg_dfree(g->adj, 0, s);
    tg_dfree(g->toff, 0, s);
    tg_dfree(g->ntype, 0, s);
    tg_dfree(g->edges, 0, s);
    tg_dfree(g->new2old, 0, s);
    tg_dfree(g->eid, 0, s);
    tg_dfree(g->adir, 0, s);
    (void)cudaStreamSynchronize(s);
    delete g;
    return TG_OK;
}

int tg_free_graph_on(tg_graph *g, cudaStream_t s) {
    if (!g) return TG_OK;
    tg_sched_free_on(g, s);
    tg_dfree(g->rowptr, 0, s);
    tg_dfree(g->adj, 0, s);
    tg_dfree(g->toff, 0, s);
    tg_dfree(g->ntype, 0, s);
    tg_dfree(g->edges, 0, s);
    tg_dfree(g->new2old, 0, s);
    tg_dfree(g->eid, 0, s);
    tg_dfree(g->adir, 0, s);
    delete g;
    return TG_OK;
}

extern "C" int tg_graph_info(const tg_graph *g, tg_info *info) {
    if (!g || !info) return TG_EINVAL;
    info->n = g->n;
    info->m_input = g->m_input;
    info->M = g->M;
    info->n_nonisolated = g->n_nonisolated;
    info->max_degree = g->max_degree;
    info->device_bytes = g->device_bytes;
    info->L = g->L;
    info->reserved = 0;
    return TG_OK;
}

namespace {
__global__ void k_edge_list(const int2 *edges, const int32_t *new2old, int64_t M, int32_t *u,
                            int32_t *v) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < M;
         e += (int64_t)gridDim.x * blockDim.x) {
        int2 p = edges[e];
        int32_t a = new2old[p.x], b = new2old[p.y];
        u[e] = a < b ? a : b;
        v[e] = a < b ? b : a;
    }
}
}  // namespace

extern "C" int tg_edge_list(const tg_graph *g, int32_t *u, int32_t *v, void *stream) {
    if (!g || !u || !v) return TG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->M == 0) return TG_OK;
    DevBuf<int32_t> du, dv;
    if (!du.alloc(g->M, s) || !dv.alloc(g->M, s)) return TG_ENOMEM;
    k_edge_list<<<grid_for(g->M), kThreads, 0, s>>>(g->edges, g->new2old, g->M, du.p, dv.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    TG_TRY_CUDA(cudaMemcpyAsync(u, du.p, g->M * 4, cudaMemcpyDefault, s));
    TG_TRY_CUDA(cudaMemcpyAsync(v, dv.p, g->M * 4, cudaMemcpyDefault, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}
