// Host-side helpers of the C ABI: status strings, layout arithmetic,
// configuration ranks, the paper's typed motif hash and the host finalize.
#include <string.h>

#include "tg_internal.cuh"

extern "C" const char *tg_strerror(int status) {
    switch (status) {
        case TG_OK: return "ok";
        case TG_EINVAL: return "invalid argument";
        case TG_ENOMEM: return "out of memory";
        case TG_ECUDA: return "CUDA runtime error";
        case TG_EOVERFLOW: return "count overflow";
        case TG_EINTERNAL: return "internal consistency check failed";
        case TG_EBUSY: return "server queue full";
        case TG_ENOMEM_ADMIT: return "request exceeds the server memory budget";
        case TG_ETIMEDOUT: return "timed out";
        case TG_ENOTFOUND: return "unknown ticket";
        default: return "unknown status";
    }
}

extern "C" int tg_version(void) { return 100; }

extern "C" int64_t tg_slots(int32_t L, int32_t k, int32_t level) {
    if (L < 1 || L > TG_MAX_TYPES || (k != 3 && k != 4)) return 0;
    if (level != TG_GRAPHLET && level != TG_ORBIT) return 0;
    const int64_t P = (int64_t)L * (L + 1) / 2;
    if (k == 3) return 2 * (int64_t)L;
    return 2 * (int64_t)L + (level == TG_ORBIT ? 10 : 6) * P;
}

extern "C" int64_t tg_global_len(int32_t L, int32_t k) {
    if (L < 1 || L > TG_MAX_TYPES || (k != 3 && k != 4)) return 0;
    int64_t len = tg_binom(L + 1, 2) + 2 * tg_binom(L + 2, 3);
    if (k == 4) len += 6 * tg_binom(L + 3, 4);
    return len;
}

extern "C" int64_t tg_config_count(int32_t L, int32_t k) {
    if (L < 1 || k < 1) return 0;
    return tg_binom(L + k - 1, k);
}

static void sort_small(int32_t *c, int k) {
    for (int a = 1; a < k; ++a) {
        int32_t x = c[a];
        int b = a - 1;
        while (b >= 0 && c[b] > x) {
            c[b + 1] = c[b];
            --b;
        }
        c[b + 1] = x;
    }
}

extern "C" int64_t tg_config_rank(const int32_t *types, int32_t k) {
    if (!types || k < 1 || k > 4) return -1;
    int32_t c[4];
    for (int m = 0; m < k; ++m) {
        if (types[m] < 0) return -1;
        c[m] = types[m];
    }
    sort_small(c, k);
    int64_t r = 0;
    for (int m = 1; m <= k; ++m) r += tg_binom(c[m - 1] + m - 1, m);
    return r;
}

extern "C" int tg_config_unrank(int64_t rank, int32_t k, int32_t *types) {
    if (!types || k < 1 || k > 4 || rank < 0) return TG_EINVAL;
    // greedy colex decoding of the k-subset {c_m + m - 1}
    for (int m = k; m >= 1; --m) {
        int64_t x = m - 1;
        while (tg_binom(x + 1, m) <= rank) ++x;
        rank -= tg_binom(x, m);
        types[m - 1] = (int32_t)(x - (m - 1));
    }
    return TG_OK;
}

extern "C" uint64_t tg_paper_hash(int32_t g, const int32_t *types, int32_t k, int32_t L) {
    if (!types || k < 1 || k > 4 || L < 1 || g < 0) return 0;
    int32_t c[4] = {0, 0, 0, 0};
    for (int m = 0; m < k; ++m) {
        if (types[m] < 0 || types[m] >= L) return 0;
        c[m] = types[m] + 1;  // types 1..L, 0 is padding
    }
    sort_small(c, k);
    const uint64_t base = L < 10 ? 10 : 100;
    uint64_t h = (uint64_t)g;
    for (int m = 0; m < 4; ++m) h = h * base + (uint64_t)c[m];
    return h;
}

extern "C" int tg_slot_config(int32_t L, int32_t k, int32_t level, int32_t phi_i, int32_t phi_j,
                              int64_t slot, int32_t *motif, int32_t *types, int32_t *k_out) {
    const int64_t width = tg_slots(L, k, level);
    if (width == 0 || slot < 0 || slot >= width || !motif || !types || !k_out) return TG_EINVAL;
    if (phi_i < 0 || phi_i >= L || phi_j < 0 || phi_j >= L) return TG_EINVAL;
    if (slot < 2 * L) {
        *motif = slot < L ? 1 : 2;
        int32_t c[3] = {phi_i, phi_j, (int32_t)(slot % L)};
        sort_small(c, 3);
        memcpy(types, c, sizeof(c));
        *k_out = 3;
        return TG_OK;
    }
    const int64_t P = (int64_t)L * (L + 1) / 2;
    int64_t q = (slot - 2 * L) / P, p = (slot - 2 * L) % P;
    int32_t t = 0;
    while (p >= L - t) {
        p -= L - t;
        ++t;
    }
    int32_t c[4] = {phi_i, phi_j, t, (int32_t)(t + p)};
    sort_small(c, 4);
    memcpy(types, c, sizeof(c));
    *motif = (int32_t)q + 3;
    *k_out = 4;
    return TG_OK;
}

extern "C" int tg_global_finalize(int32_t L, int32_t k, const uint64_t *sums, uint64_t *out) {
    const int64_t len = tg_global_len(L, k);
    if (!len || !sums || !out) return TG_EINVAL;
    const int64_t off1 = tg_binom(L + 1, 2), n3 = tg_binom(L + 2, 3), n4 = tg_binom(L + 3, 4);
    const uint64_t eh[6] = {3, 3, 4, 4, 5, 6};
    int status = TG_OK;
    for (int64_t x = 0; x < len; ++x) {
        uint64_t d = 1;
        if (x >= off1 + 2 * n3)
            d = eh[(x - off1 - 2 * n3) / n4];
        else if (x >= off1 + n3)
            d = 3;
        else if (x >= off1)
            d = 2;
        if (sums[x] % d) status = TG_EINTERNAL;
        out[x] = sums[x] / d;
    }
    return status;
}
