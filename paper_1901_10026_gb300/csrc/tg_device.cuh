// Device helpers shared by the counting kernels (typed pairs, colex ranks,
// sorted-range membership, the per-edge hash of Gamma_i and the bitmap test).
#pragma once

#include "tg_internal.cuh"

namespace tgd {

constexpr unsigned kFull = 0xffffffffu;

// classes of a node relative to the edge (bit 0: in Gamma_i, bit 1: in Gamma_j)
enum { CLS_I = 0, CLS_SI = 1, CLS_SJ = 2, CLS_T = 3 };

__device__ __forceinline__ int pair_index(int L, int a, int b) {
    if (a > b) {
        int t = a;
        a = b;
        b = t;
    }
    return a * L - (a * (a - 1)) / 2 + (b - a);
}

__device__ __forceinline__ void unpair(int L, int p, int &t, int &u) {
    t = 0;
    while (p >= L - t) {
        p -= L - t;
        ++t;
    }
    u = t + p;
}

__device__ __forceinline__ uint64_t c2(uint64_t x) { return x < 2 ? 0 : x * (x - 1) / 2; }

// The closed forms of Sec. "Combinatorial Relationships" for the type pair
// (t, u) of an edge: g4 (4-path centre), g5 (4-star), g9 (tailed-triangle
// edge at the degree-3 node) and g11 (chordal-cycle chord) from the typed
// set sizes |S_i^t|, |S_i^u|, |S_j^t|, |S_j^u|, |T^t|, |T^u| and the
// enumerated g6, g7, g10, g12 of the same pair (mod 2^64).
__device__ __forceinline__ void closed_forms(bool same, uint64_t sit, uint64_t siu, uint64_t sjt,
                                             uint64_t sju, uint64_t tt, uint64_t tu, uint64_t g6,
                                             uint64_t g7, uint64_t g10, uint64_t g12, uint64_t &g4,
                                             uint64_t &g5, uint64_t &g9, uint64_t &g11) {
    if (same) {
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
}

__device__ __forceinline__ int64_t colex3(int a, int b, int c) {
    // a <= b <= c
    return (int64_t)a + (int64_t)(b + 1) * b / 2 + (int64_t)(c + 2) * (c + 1) * c / 6;
}
__device__ __forceinline__ int64_t colex4(int a, int b, int c, int d) {
    return colex3(a, b, c) + (int64_t)(d + 3) * (d + 2) * (d + 1) * d / 24;
}
__device__ __forceinline__ void sort2(int &a, int &b) {
    if (a > b) {
        int t = a;
        a = b;
        b = t;
    }
}

// Is the packed entry w in the list at adj + base?  `to` holds the list's type
// offsets, so only the typed range Gamma^{type(w)} is searched.
__device__ __forceinline__ bool contains(const uint32_t *__restrict__ adj, int64_t base,
                                         const int32_t *__restrict__ to, uint32_t w) {
    int t = (int)(w >> TG_TSHIFT);
    int lo = __ldg(to + t), hi = __ldg(to + t + 1);
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        uint32_t x = __ldg(adj + base + mid);
        if (x < w)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo < __ldg(to + t + 1) && __ldg(adj + base + lo) == w;
}

// Edge id of (j, y) when y (packed entry w) is a neighbour of j, else
// 0xffffffff.  j's list (base bj, length dj, type offsets toj) and y's list
// are both sorted by (type, id), and (j, y) is one edge: the typed range of
// the shorter list is searched (w in Gamma_j, or j's packed entry pj in
// Gamma_y), which for the low-degree nodes beyond a bitmap is a handful of
// loads instead of a search through a hub's list.
__device__ __forceinline__ uint32_t edge_to(const int64_t *__restrict__ rowptr,
                                            const uint32_t *__restrict__ adj,
                                            const uint32_t *__restrict__ eid,
                                            const int32_t *__restrict__ toff, int L, int64_t bj,
                                            int dj, const int32_t *__restrict__ toj, uint32_t pj,
                                            uint32_t w);

constexpr uint32_t kEmpty = 0xffffffffu;
constexpr size_t kMiscBytes = 3 * 16 * 4 + 16;     // Tn, Si, Sj, work item
constexpr size_t kStageBytes = 32 * 17;  // per-warp w_k slots (a multiple of 16 bytes)

// Index of packed entry w in the list at adj + base (typed range search), -1 if absent
__device__ __forceinline__ int find_pos(const uint32_t *__restrict__ adj, int64_t base,
                                        const int32_t *__restrict__ to, uint32_t w) {
    const int t = (int)(w >> TG_TSHIFT);
    int lo = __ldg(to + t), hi = __ldg(to + t + 1);
    const int end = hi;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(adj + base + mid) < w)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < end && __ldg(adj + base + lo) == w) ? lo : -1;
}

__device__ __forceinline__ uint32_t edge_to(const int64_t *__restrict__ rowptr,
                                            const uint32_t *__restrict__ adj,
                                            const uint32_t *__restrict__ eid,
                                            const int32_t *__restrict__ toff, int L, int64_t bj,
                                            int dj, const int32_t *__restrict__ toj, uint32_t pj,
                                            uint32_t w) {
    const uint32_t y = w & TG_IDMASK;
    const int64_t by = __ldg(rowptr + y);
    const int dy = (int)(__ldg(rowptr + y + 1) - by);
    if (dy < dj) {
        const int q = find_pos(adj, by, toff + (int64_t)y * (L + 1), pj);
        return q < 0 ? 0xffffffffu : __ldg(eid + by + q);
    }
    const int q = find_pos(adj, bj, toj, w);
    return q < 0 ? 0xffffffffu : __ldg(eid + bj + q);
}

// As edge_to, but the index of the adjacency entry of the edge (j, y) (in
// Gamma_j or in Gamma_y, whichever list was searched), 0xffffffff if absent.
__device__ __forceinline__ uint32_t entry_to(const int64_t *__restrict__ rowptr,
                                             const uint32_t *__restrict__ adj,
                                             const int32_t *__restrict__ toff, int L, int64_t bj,
                                             int dj, const int32_t *__restrict__ toj, uint32_t pj,
                                             uint32_t w) {
    const uint32_t y = w & TG_IDMASK;
    const int64_t by = __ldg(rowptr + y);
    const int dy = (int)(__ldg(rowptr + y + 1) - by);
    if (dy < dj) {
        const int q = find_pos(adj, by, toff + (int64_t)y * (L + 1), pj);
        return q < 0 ? 0xffffffffu : (uint32_t)(by + q);
    }
    const int q = find_pos(adj, bj, toj, w);
    return q < 0 ? 0xffffffffu : (uint32_t)(bj + q);
}

// Is y (packed entry w) a neighbour of j?  As edge_to, without the edge id.
__device__ __forceinline__ bool adjacent(const int64_t *__restrict__ rowptr,
                                         const uint32_t *__restrict__ adj,
                                         const int32_t *__restrict__ toff, int L, int64_t bj,
                                         int dj, const int32_t *__restrict__ toj, uint32_t pj,
                                         uint32_t w) {
    const uint32_t y = w & TG_IDMASK;
    const int64_t by = __ldg(rowptr + y);
    const int dy = (int)(__ldg(rowptr + y + 1) - by);
    if (dy < dj) return find_pos(adj, by, toff + (int64_t)y * (L + 1), pj) >= 0;
    return find_pos(adj, bj, toj, w) >= 0;
}

// Per-warp hash sets of node ids in shared memory (open addressing, linear
// probing, id + 1 stored, 0 empty).  Writers and readers are ordered by a
// __syncwarp or __syncthreads between them.
__device__ __forceinline__ uint32_t hset_slot(uint32_t id, int lg) {
    return (id * 0x9E3779B1u) >> (32 - lg);
}
__device__ __forceinline__ void hset_put(uint32_t *tab, int lg, uint32_t id) {
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t h = hset_slot(id, lg);
    for (int probe = 0; probe < (1 << lg); ++probe) {
        const uint32_t old = atomicCAS(tab + h, 0u, id + 1u);
        if (old == 0u || old == id + 1u) return;
        h = (h + 1u) & mask;
    }
}
__device__ __forceinline__ bool hset_has(const uint32_t *tab, int lg, uint32_t id) {
    const uint32_t mask = (1u << lg) - 1u;
    const uint32_t *t = tab;
    uint32_t h = hset_slot(id, lg);
    for (int probe = 0; probe < (1 << lg); ++probe) {
        const uint32_t k = t[h];
        if (k == id + 1u) return true;
        if (k == 0u) return false;
        h = (h + 1u) & mask;
    }
    return false;
}

// Slot of id in a hash set as above, claiming an empty slot for it; -1 when
// the table is full.  Concurrent claims of one id meet in one slot.
__device__ __forceinline__ int hset_claim(uint32_t *tab, int lg, uint32_t id) {
    const uint32_t mask = (1u << lg) - 1u;
    const volatile uint32_t *t = tab;  // slots claimed by other lanes while this one probes
    uint32_t h = hset_slot(id, lg);
    for (int probe = 0; probe < (1 << lg); ++probe) {
        const uint32_t k = t[h];
        if (k == id + 1u) return (int)h;
        if (k == 0u) {
            const uint32_t old = atomicCAS(tab + h, 0u, id + 1u);
            if (old == 0u || old == id + 1u) return (int)h;
        }
        h = (h + 1u) & mask;
    }
    return -1;
}

// Per-warp hash map of node ids to 32-bit values in shared memory (keys as
// in hset, values beside them; a value is written after its key is claimed and
// read after a __syncwarp).
__device__ __forceinline__ void hmap_put(uint32_t *keys, uint32_t *vals, int lg, uint32_t id,
                                         uint32_t val) {
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t h = hset_slot(id, lg);
    for (int probe = 0; probe < (1 << lg); ++probe) {
        const uint32_t old = atomicCAS(keys + h, 0u, id + 1u);
        if (old == 0u || old == id + 1u) {
            vals[h] = val;
            return;
        }
        h = (h + 1u) & mask;
    }
}
// the value of id, or 0xffffffff when absent
__device__ __forceinline__ uint32_t hmap_get(const uint32_t *keys, const uint32_t *vals, int lg,
                                             uint32_t id) {
    const uint32_t mask = (1u << lg) - 1u;
    const volatile uint32_t *k = keys;
    const volatile uint32_t *v = vals;
    uint32_t h = hset_slot(id, lg);
    for (int probe = 0; probe < (1 << lg); ++probe) {
        const uint32_t x = k[h];
        if (x == id + 1u) return v[h];
        if (x == 0u) return 0xffffffffu;
        h = (h + 1u) & mask;
    }
    return 0xffffffffu;
}

__device__ __forceinline__ uint32_t hslot(uint32_t id, int lg) {
    return (id * 2654435761u) >> (32 - lg);
}

__device__ __forceinline__ void hinsert(uint32_t *hk, int lg, uint32_t id, int cls) {
    const uint32_t mask = (1u << lg) - 1u, v = (id << 2) | (uint32_t)cls;
    uint32_t h = hslot(id, lg);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        if (atomicCAS(hk + h, kEmpty, v) == kEmpty) return;
        h = (h + 1) & mask;
    }
}

// class of a Gamma_i member (CLS_SI or CLS_T), 0 if absent.  The table is
// read through volatile loads: it is filled with atomicCAS, and with plain
// loads here the paper-literal CTA kernel with its smallest caps (128
// threads, 32 hash slots, 96 bitmap bits) gave wrong classes on the GPU while
// every other kernel and launch shape stayed exact; the cause is not known.
__device__ __forceinline__ int hlookup(const uint32_t *hk, int lg, uint32_t id) {
    const volatile uint32_t *vk = hk;
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t h = hslot(id, lg);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint32_t v = vk[h];
        if (v == kEmpty) return 0;
        if ((v >> 2) == id) return (int)(v & 3u);
        h = (h + 1) & mask;
    }
    return 0;  // unreachable: the table is never more than half full
}

// mark bit of node id in the shared-memory bitmap (written before a barrier)
__device__ __forceinline__ bool bm_test(const uint32_t *bm, uint32_t id) {
    return (bm[id >> 5] >> (id & 31u)) & 1u;
}


}  // namespace tgd
