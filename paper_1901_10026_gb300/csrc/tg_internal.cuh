// Internal declarations of the typed-graphlet library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "tg.h"

// Packed adjacency entry: (type << TG_TSHIFT) | node id (new, degree-ordered
// ids).  Sorting entries as unsigned integers sorts a list by (type, id), so
// every typed neighbourhood is a contiguous range and the type of a
// neighbour is read from the entry itself.
#define TG_TSHIFT 28
#define TG_IDMASK ((1u << TG_TSHIFT) - 1u)

// Device-side error bits (OR-ed into a flag word the host reads back).
#define TG_DERR_INPUT 1u      // node id or type out of range in the input
#define TG_DERR_DIVISIBLE 2u  // a global sum not divisible by |E(H)|
#define TG_DERR_BOUNDS 4u     // an internal bounds check failed

struct tg_sched;  // per-graph counting schedule (tg_count.cu)

struct tg_graph {
    int64_t n = 0;
    int64_t m_input = 0;
    int64_t M = 0;
    int64_t n_nonisolated = 0;
    int64_t max_degree = 0;
    int32_t L = 0;
    int device = 0;
    int64_t device_bytes = 0;

    int64_t *rowptr = nullptr;   // n+1, new ids
    uint32_t *adj = nullptr;     // 2M packed entries
    int32_t *toff = nullptr;     // n*(L+1) relative type offsets per node
    uint8_t *ntype = nullptr;    // n, type of new id
    int2 *edges = nullptr;       // M, (new a, new b) in canonical order
    uint32_t *eid = nullptr;     // 2M, canonical edge id of each adjacency entry
    int32_t *new2old = nullptr;  // n
    uint8_t *adir = nullptr;     // 2M (TG_DIRECTED only): arcs of each adjacency entry,
                                 // bit 0 owner -> neighbour, bit 1 neighbour -> owner

    mutable std::mutex mu;           // guards the lazily built schedule
    mutable tg_sched *sched = nullptr;
};

// ----------------------------------------------------------------- memory --
void *tg_dalloc(size_t bytes, cudaStream_t s);  // NULL on failure
void tg_dfree(void *p, size_t bytes, cudaStream_t s);

// Scoped device buffer: freed (stream-ordered) when the scope ends.
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { reset(); }
    bool alloc(size_t count, cudaStream_t st) {
        reset();
        s = st;
        bytes = count * sizeof(T);
        if (bytes == 0) bytes = sizeof(T);
        p = static_cast<T *>(tg_dalloc(bytes, st));
        return p != nullptr;
    }
    void reset() {
        if (p) tg_dfree(p, bytes, s);
        p = nullptr;
    }
    T *release() {
        T *q = p;
        p = nullptr;
        return q;
    }
};

// Records the cudaError_t behind a TG_ECUDA for tg_last_cuda_error (per
// host thread).
void tg_note_cuda_error(cudaError_t e);

#define TG_TRY_CUDA(call)                         \
    do {                                          \
        cudaError_t _e = (call);                  \
        if (_e != cudaSuccess) {                  \
            tg_note_cuda_error(_e);               \
            return TG_ECUDA;                      \
        }                                         \
    } while (0)

#define TG_TRY(call)                              \
    do {                                          \
        int _r = (call);                          \
        if (_r != TG_OK) return _r;               \
    } while (0)

// ------------------------------------------------------------- primitives --
// Direction bits of a graph built with TG_DIRECTED (tg_directed.cu): for
// every non-loop input arc src -> dst (original ids, device arrays), marks the
// entry of dst in the list of src as outgoing and the entry of src in the list
// of dst as incoming.  old2new maps original ids to the graph's ids.
int tg_attach_arcs(tg_graph *g, const int32_t *src, const int32_t *dst, int64_t m,
                   const int32_t *old2new, cudaStream_t s);

// Exclusive prefix sums (out may alias in).  n >= 0.
int tg_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s);
int tg_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
// LSD radix sort of uint64 keys on their low `bits` bits (stable).  `keys` and
// `tmp` hold n entries each; *result points at whichever holds the output.
int tg_radix_sort_u64(uint64_t *keys, uint64_t *tmp, int64_t n, int bits, cudaStream_t s,
                      uint64_t **result);
// Same, carrying a uint32 value per key (vals/vtmp); *vresult gets the output.
int tg_radix_sort_kv(uint64_t *keys, uint64_t *tmp, uint32_t *vals, uint32_t *vtmp, int64_t n,
                     int bits, cudaStream_t s, uint64_t **result, uint32_t **vresult);

int tg_bitlen(uint64_t x);  // number of bits needed to represent x (0 -> 0)

// Counts every kernel this library launches (reported by tg_launch_count).
void tg_note_launch();

// Lets `func` take the device's opt-in maximum of dynamic shared memory (less
// its static shared memory).  Every caller writes the same value, so a call on
// another host thread can never lower the limit between this thread's sizing
// and its launch; launches are then checked against their own size only.
// Multiprocessors of the current device, and the shared memory a block may
// opt in to (48 KB when the attribute cannot be read).
int tg_num_sms();
int tg_smem_optin();
int tg_allow_max_smem(const void *func);

// Is p a device pointer (or managed)?  Host pointers, registered or not, -> false.
bool tg_is_device_ptr(const void *p);

// ------------------------------------------------------------- layout -----
static inline int64_t tg_binom(int64_t a, int64_t b) {
    if (b < 0 || a < b) return 0;
    int64_t r = 1;
    for (int64_t i = 1; i <= b; ++i) r = r * (a - b + i) / i;
    return r;
}

// Free the lazily built schedule of a graph (tg_count.cu).
void tg_sched_free(tg_graph *g);
// Stream-ordered frees for a graph used only on stream s (no device sync).
void tg_sched_free_on(tg_graph *g, cudaStream_t s);
int tg_free_graph_on(tg_graph *g, cudaStream_t s);

// Work units of a grouped order (runs of edges sharing their high-degree end
// j, tg_reuse.cu): unit u is order[ustart[u] .. ustart[u+1]).  Units whose j
// has at most TG_LIGHT_DEGREE neighbours are listed in `light` (one warp each,
// Gamma_j in a per-warp hash), the others in `heavy` (one CTA each, Gamma_j
// in a shared-memory bitmap).
#define TG_LIGHT_DEGREE 256
#define TG_LIGHT_LG 9  // log2 of the per-warp hash slots (2 x TG_LIGHT_DEGREE)
struct tg_units {
    DevBuf<uint32_t> ustart, heavy, light;
    uint32_t nunits = 0, nheavy = 0, nlight = 0;
};

// Whole-graph enumerations and the per-edge pass of the cycles kernel
// (tg_cycles.cu).  Per-edge mode: c4e holds M x L x L and k4e M x L(L+1)/2
// zeroed counters (g4 = NULL).  Global mode (c4e / k4e = NULL): g4 gets, by
// type multiset (C(L+3,4) zeroed entries), the non-induced 4-cycles (cycles)
// or the 4-cliques (cliques); tg_cyc_correct then adds their share
// to undivided sums counted with Q = C4 = 0.
// Share of the whole-graph enumerations a call takes when the global count is
// split across ranks: the 4-cycle anchors and the 4-clique lowest nodes v
// with v mod count == index (ids are degree-ordered, so hubs spread evenly).
struct tg_part {
    int32_t index = 0, count = 1;
};

int tg_cyc_cycles(const tg_graph *g, unsigned long long *c4e, unsigned long long *g4,
                  unsigned long long *work, const tg_tune &t, const tg_part &part, cudaStream_t s);
int tg_cyc_cliques(const tg_graph *g, unsigned long long *k4e, unsigned long long *g4,
                   unsigned long long *work, const tg_tune &t, const tg_part &part, cudaStream_t s);
int tg_cyc_correct(unsigned long long *hist, int L, const unsigned long long *c4w,
                   const unsigned long long *k4, cudaStream_t s);
int tg_cyc_edges(const tg_graph *g, int k, int level, const uint32_t *order, int64_t count,
                 const tg_units &un, uint64_t *rows, int64_t width,
                 unsigned long long *hist, const uint32_t *tau, const uint32_t *tau_adj,
                 const uint32_t *theta,
                 const uint32_t *dsum, const unsigned long long *c4e,
                 const unsigned long long *k4e, unsigned long long *work, const tg_tune &t,
                 cudaStream_t s);

// Counts through Alg. 1's typed triangle counts (tg_reuse.cu).  full_order is
// the grouped order of all M edges; order[0..count) the edges to count.  With
// TG_KERNEL_CYCLES (or AUTO) the per-edge pass is tg_cyc_*, else k_count_reuse.
// With part.count > 1 (global sums only, k = 4), the call is one share of a
// split count: order[0..count) is its slice of the edges, and the 4-cycle and
// 4-clique totals (with their correction of the sums) are the part's own.
int tg_reuse_count(const tg_graph *g, int k, int level, const uint32_t *full_order,
                   const uint32_t *order, int64_t count, uint64_t *rows, int64_t width,
                   unsigned long long *hist, const tg_tune &t, cudaStream_t s,
                   const tg_part &part = tg_part());

// Per-edge rows of the whole graph into device memory `rows` (M x
// tg_slots(L, k, level)), queued on s (tg_count.cu).
int tg_rows_device(const tg_graph *g, int k, int level, uint64_t *rows, cudaStream_t s);
