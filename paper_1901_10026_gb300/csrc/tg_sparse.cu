// Sparse per-edge output (Sec. "Sparse Typed Motif Format"): only the nonzero
// typed counts of every edge, as (id, count) pairs, edge after edge in
// canonical edge order, with the edge's pairs between offsets[e] and
// offsets[e + 1].
//
// The paper keys a nonzero by its typed motif hash and remaps the hashes to
// consecutive ids through a lookup table.  Here an id numbers every typed
// graphlet (graphlet level) or typed orbit (orbit level) consecutively, block
// by block: [1: C(L+2,3)][2: C(L+2,3)] then, for k = 4, one C(L+3,4) block per
// 4-node graphlet h3..h8 (or orbit g3..g12); inside a block the entry of the
// sorted type multiset of all the subgraph's nodes is its colex rank.  The id
// therefore has one meaning for every edge (the dense slots of a row depend
// on the edge's endpoint types), and tg_sparse_id maps it back to the
// graphlet or orbit, its types and the paper's hash.
#include <algorithm>

#include "tg_device.cuh"

using namespace tgd;

namespace {

struct SparseLayout {
    int32_t L, P, k, level, n4blocks;
    int64_t n3, n4;
};

// id of slot s of an edge whose endpoints have types ti, tj
__device__ __forceinline__ uint32_t slot_id(const SparseLayout &y, int ti, int tj, int s) {
    const int L = y.L;
    if (s < 2 * L) {
        const int blk = s / L, t = s % L;
        int a = ti, b = tj, c = t;
        sort2(a, b);
        sort2(b, c);
        sort2(a, b);
        return (uint32_t)(blk * y.n3 + colex3(a, b, c));
    }
    const int r = s - 2 * L, blk = r / y.P;
    int t, u;
    unpair(L, r % y.P, t, u);
    int a = ti, b = tj, c = t, d = u;
    sort2(a, b);
    sort2(c, d);
    sort2(a, c);
    sort2(b, d);
    sort2(b, c);
    return (uint32_t)(2 * y.n3 + blk * y.n4 + colex4(a, b, c, d));
}

// Nonzero slots per row (cnt[M] = 0 for the exclusive scan's total).
__global__ void k_row_nnz(const uint64_t *rows, int64_t M, int64_t width, int64_t *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e <= M; e += nw) {
        if (e == M) {
            if (lane == 0) cnt[M] = 0;
            continue;
        }
        int64_t c = 0;
        for (int64_t s = lane; s < width; s += 32) c += rows[e * width + s] != 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
        if (lane == 0) cnt[e] = c;
    }
}

// The pairs of every row, one warp per edge, in slot order.
__global__ void k_row_pairs(const uint64_t *rows, int64_t M, int64_t width, const int64_t *offsets,
                            const int2 *edges, const uint8_t *ntype, SparseLayout y,
                            uint32_t *ids, uint64_t *counts) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned below = (1u << lane) - 1u;
    for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < M; e += nw) {
        const int2 ab = edges[e];
        const int ti = ntype[ab.x], tj = ntype[ab.y];
        int64_t at = offsets[e];
        for (int64_t s0 = 0; s0 < width; s0 += 32) {
            const int64_t s = s0 + lane;
            const uint64_t v = s < width ? rows[e * width + s] : 0ull;
            const unsigned m = __ballot_sync(kFull, v != 0ull);
            if (v) {
                const int64_t q = at + __popc(m & below);
                ids[q] = slot_id(y, ti, tj, (int)s);
                counts[q] = v;
            }
            at += __popc(m);
        }
    }
}

}  // namespace

static SparseLayout sparse_layout(int L, int k, int level) {
    SparseLayout y;
    y.L = L;
    y.P = L * (L + 1) / 2;
    y.k = k;
    y.level = level;
    y.n3 = tg_binom(L + 2, 3);
    y.n4 = tg_binom(L + 3, 4);
    y.n4blocks = k == 4 ? (level == TG_ORBIT ? 10 : 6) : 0;
    return y;
}

extern "C" int64_t tg_sparse_ids(int32_t L, int32_t k, int32_t level) {
    if (L < 1 || L > TG_MAX_TYPES || (k != 3 && k != 4) || (level != TG_GRAPHLET && level != TG_ORBIT))
        return -1;
    const SparseLayout y = sparse_layout(L, k, level);
    return 2 * y.n3 + y.n4blocks * y.n4;
}

extern "C" int tg_sparse_id(int32_t L, int32_t k, int32_t level, int64_t id, int32_t *motif,
                            int32_t *types, int32_t *k_out) {
    const int64_t total = tg_sparse_ids(L, k, level);
    if (total < 0 || id < 0 || id >= total || !motif || !types || !k_out) return TG_EINVAL;
    const SparseLayout y = sparse_layout(L, k, level);
    if (id < 2 * y.n3) {
        *motif = (int32_t)(1 + id / y.n3);
        *k_out = 3;
        return tg_config_unrank(id % y.n3, 3, types);
    }
    const int64_t r = id - 2 * y.n3;
    *motif = (int32_t)(3 + r / y.n4);
    *k_out = 4;
    return tg_config_unrank(r % y.n4, 4, types);
}

extern "C" int tg_count_per_edge_sparse(const tg_graph *g, int32_t k, int32_t level,
                                        int64_t *offsets, uint32_t *ids, uint64_t *counts,
                                        int64_t capacity, int64_t *nnz, void *stream) {
    if (!g || !offsets || !nnz || (k != 3 && k != 4) || (level != TG_GRAPHLET && level != TG_ORBIT))
        return TG_EINVAL;
    if ((ids == nullptr) != (counts == nullptr) || capacity < 0) return TG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t M = g->M, width = tg_slots(g->L, k, level);
    DevBuf<uint64_t> rows;
    DevBuf<int64_t> cnt, off;
    if (!rows.alloc((size_t)std::max<int64_t>(1, M) * width, s) || !cnt.alloc(M + 1, s) ||
        !off.alloc(M + 1, s))
        return TG_ENOMEM;
    TG_TRY(tg_rows_device(g, k, level, rows.p, s));
    const unsigned grid = (unsigned)std::min<int64_t>(((M + 1) * 32 + 255) / 256, 65535LL * 16);
    k_row_nnz<<<grid, 256, 0, s>>>(rows.p, M, width, cnt.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    TG_TRY(tg_scan_i64(cnt.p, off.p, M + 1, s));
    int64_t total = 0;
    TG_TRY_CUDA(cudaMemcpyAsync(&total, off.p + M, 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaMemcpyAsync(offsets, off.p, (M + 1) * 8, cudaMemcpyDefault, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    *nnz = total;
    if (!ids) return TG_OK;
    if (total > capacity) return TG_EOVERFLOW;
    const bool dev_out = tg_is_device_ptr(ids) && tg_is_device_ptr(counts);
    DevBuf<uint32_t> dids;
    DevBuf<uint64_t> dcounts;
    uint32_t *pi = ids;
    uint64_t *pc = counts;
    if (!dev_out) {
        if (!dids.alloc(std::max<int64_t>(1, total), s) || !dcounts.alloc(std::max<int64_t>(1, total), s))
            return TG_ENOMEM;
        pi = dids.p;
        pc = dcounts.p;
    }
    if (M > 0) {
        k_row_pairs<<<grid, 256, 0, s>>>(rows.p, M, width, off.p, g->edges, g->ntype,
                                         sparse_layout(g->L, k, level), pi, pc); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    if (!dev_out && total > 0) {
        TG_TRY_CUDA(cudaMemcpyAsync(ids, pi, total * 4, cudaMemcpyDeviceToHost, s));
        TG_TRY_CUDA(cudaMemcpyAsync(counts, pc, total * 8, cudaMemcpyDeviceToHost, s));
    }
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}
