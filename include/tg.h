/*
 * tg.h — exact typed 3- and 4-node graphlet counting on one NVIDIA GB300
 * (sm_103a).  C ABI: plain pointers and sizes, no C++ or framework types.
 *
 * Method: Rossi et al., "Heterogeneous Network Motifs" (arXiv 1901.10026).
 * Problem statement: an undirected graph G = (V, E) with a node-type map
 * phi : V -> {0..L-1} (Def. "Heterogeneous network"); for every edge (i, j)
 * count the connected induced 3- and 4-node subgraphs containing it, keyed by
 * graphlet (or edge orbit, Table 2) and by the multiset of node types
 * (Def. "Typed Graphlet Instance"); global counts are the per-edge sums
 * divided by the graphlet's edge count (Eq. C = x^T e / |E(H)|).
 *
 * Conventions shared by every call:
 *   - Return value: TG_OK (0) or a negative TG_E* code.  On error no partial
 *     state is left behind (outputs may have been written partially).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is ordered on it; calls that return results in
 *     host memory synchronise the stream before returning.
 *   - Pointers marked "host or device" may point to either; the library tells
 *     them apart through unified addressing.
 *   - The library allocates its own device memory (stream-ordered) for graphs
 *     and scratch; see tg_set_allocator to route that through a caller's
 *     allocator.
 *   - A tg_graph is read-only after tg_build_csr; concurrent counting calls on
 *     one graph from several host threads are safe.
 *
 * Per-edge row layout (slot s of row e).  P = L(L+1)/2 unordered type pairs
 * (t, t'), t <= t', in lexicographic order.  Orbit level (k = 4):
 *     [g1: L][g2: L][g3: P][g4: P][g5: P] ... [g12: P]     2L + 10P slots
 * graphlet level (k = 4):
 *     [h1: L][h2: L][h3: P][h4: P] ... [h8: P]              2L + 6P slots
 * k = 3 keeps the first 2L slots.  A 3-node slot t holds the subgraphs whose
 * third node has type t; a 4-node slot (t, t') those whose two other nodes
 * have types {t, t'}.  Orbits (Table 2): g1 3-path, g2 triangle, g3 4-path
 * end edge, g4 4-path centre edge, g5 4-star, g6 4-cycle, g7 tailed-triangle
 * tail edge, g8 tailed-triangle centre (triangle edge opposite the degree-3
 * node), g9 tailed-triangle tri-edge (triangle edge at the degree-3 node),
 * g10 chordal-cycle outer edge, g11 chordal-cycle chord, g12 4-clique.
 * Graphlets (Sec. "From Typed Orbits to Graphlets"): h1 3-path, h2 triangle,
 * h3 4-path (g3+g4), h4 4-star (g5), h5 4-cycle (g6), h6 tailed triangle
 * (g7+g8+g9), h7 chordal cycle (g10+g11), h8 4-clique (g12).
 *
 * Global layout: [edges: C(L+1,2)][h1: C(L+2,3)][h2: C(L+2,3)] followed, for
 * k = 4, by [h3..h8: C(L+3,4) each].  Inside a block the entry for the sorted
 * type multiset c_1 <= ... <= c_m is tg_config_rank(c, m) (colex order).
 *
 * Canonical edge order: the simplified graph's edges (u, v), u < v, in
 * ascending (u, v) order of the ORIGINAL node ids; row e of every per-edge
 * output belongs to the e-th edge of tg_edge_list.
 */
#ifndef TG_H
#define TG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status ---- */
#define TG_OK 0
#define TG_EINVAL (-1)       /* an argument is out of range or inconsistent   */
#define TG_ENOMEM (-2)       /* a device or host allocation failed            */
#define TG_ECUDA (-3)        /* a CUDA runtime call failed                    */
#define TG_EOVERFLOW (-4)    /* a count could exceed its integer width        */
#define TG_EINTERNAL (-5)    /* a device-side consistency check failed        */
#define TG_EBUSY (-6)        /* server queue full                              */
#define TG_ENOMEM_ADMIT (-7) /* request can never fit the server's memory cap */
#define TG_ETIMEDOUT (-8)    /* a bounded wait ran out                         */
#define TG_ENOTFOUND (-9)    /* unknown server ticket                          */

/* Human-readable name of a status code (static storage, never NULL). */
const char *tg_strerror(int status);

/* Library version as 10000*major + 100*minor + patch. */
int tg_version(void);

/* ----------------------------------------------------------- graphs ----- */
typedef struct tg_graph tg_graph;

/* tg_build_csr flags */
#define TG_INPUT_DEVICE 1u /* src, dst, type are device pointers (else host) */
#define TG_DIRECTED 2u     /* also keep the direction of every pair: (src, dst)
                              is the arc src -> dst (Sec. "Directed Typed
                              Graphlets"); needed by tg_count_directed_*     */

/* Limits checked by tg_build_csr. */
#define TG_MAX_TYPES 16
#define TG_MAX_NODES (1 << 28)

/*
 * Build the resident, read-only graph used by every counting call
 * (Def. "Heterogeneous network", Def. "Typed Neighborhood"): self-loops are
 * dropped, duplicate and reversed pairs merged, nodes relabelled by degree
 * (descending, ties by original id), and every adjacency list sorted by
 * (neighbour type, neighbour id) so that each typed neighbourhood Gamma_v^t
 * is one contiguous range.
 *
 *   n     number of nodes, 1 <= n <= TG_MAX_NODES; ids are 0..n-1
 *   m     number of input pairs (src[e], dst[e]), m >= 0
 *   src, dst  int32 node ids, host or device per TG_INPUT_DEVICE
 *   type  uint8 node types, length n, each < L
 *   L     number of node types, 1 <= L <= TG_MAX_TYPES
 *   out   receives the graph; the library owns it until tg_free_graph
 *
 * The caller keeps ownership of src, dst and type; they are read during the
 * call only (the call synchronises `stream` before returning).
 * Errors: TG_EINVAL (n, m, L out of range; an id outside [0, n); a type >= L;
 * out == NULL), TG_ENOMEM, TG_ECUDA.
 */
int tg_build_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                 const uint8_t *type, int32_t L, uint32_t flags, void *stream,
                 tg_graph **out);

/* Release a graph and its device memory (NULL is a no-op). */
int tg_free_graph(tg_graph *g);

typedef struct {
    int64_t n;             /* nodes                                      */
    int64_t m_input;       /* input pairs given to tg_build_csr          */
    int64_t M;             /* undirected edges after simplification      */
    int64_t n_nonisolated; /* nodes with degree >= 1                     */
    int64_t max_degree;    /* Delta                                      */
    int64_t device_bytes;  /* device memory held by the graph            */
    int32_t L;             /* node types                                 */
    int32_t reserved;
} tg_info;

int tg_graph_info(const tg_graph *g, tg_info *info);

/*
 * Canonical edge list: u[e] < v[e], original ids, ascending (u, v).  u and v
 * hold M entries each, host or device.  Synchronises `stream`.
 */
int tg_edge_list(const tg_graph *g, int32_t *u, int32_t *v, void *stream);

/* ----------------------------------------------------------- layout ----- */
#define TG_GRAPHLET 0
#define TG_ORBIT 1

/* Slots per per-edge row: 2L (k = 3) or 2L + {6|10}*L(L+1)/2 (k = 4). */
int64_t tg_slots(int32_t L, int32_t k, int32_t level);

/* Entries of the global histogram for (L, k); see the global layout above. */
int64_t tg_global_len(int32_t L, int32_t k);

/* Number of typed configurations of one k-node graphlet: C(L+k-1, k)
 * (Eq. "number of typed motifs", Table 1). */
int64_t tg_config_count(int32_t L, int32_t k);

/* Colex rank of a sorted type multiset: sum_m C(c_m + m - 1, m), m = 1..k.
 * `types` need not be sorted (it is sorted internally); returns -1 when k is
 * not in 1..4 or a type is negative. */
int64_t tg_config_rank(const int32_t *types, int32_t k);

/* Inverse of tg_config_rank for k in 1..4: writes the sorted multiset. */
int tg_config_unrank(int64_t rank, int32_t k, int32_t *types);

/*
 * Typed motif hash of Sec. "Typed Motif Hash Functions":
 *   F = g*10^4 + t1*10^3 + t2*10^2 + t3*10 + t4      (L < 10)
 *   F = g*10^8 + t1*10^6 + t2*10^4 + t3*10^2 + t4    (L >= 10)
 * with the k node types shifted to 1..L, sorted ascending (every ordering of
 * the types maps to the same value), and padded with 0 for k < 4.  g is the
 * caller's motif or orbit number.  Returns 0 on invalid input.
 */
uint64_t tg_paper_hash(int32_t g, const int32_t *types, int32_t k, int32_t L);

/* Per-edge slot -> (orbit or graphlet id, sorted config of all k nodes).
 * phi_i, phi_j are the edge's endpoint types; writes `k_out` (3 or 4) types. */
int tg_slot_config(int32_t L, int32_t k, int32_t level, int32_t phi_i, int32_t phi_j,
                   int64_t slot, int32_t *motif, int32_t *types, int32_t *k_out);

/* ----------------------------------------------------------- counting --- */
/*
 * Global typed graphlet counts (Sec. "Global Typed Graphlet Counts").
 *   k    3 or 4 (k = 4 also fills the 2- and 3-node blocks)
 *   out  tg_global_len(L, k) uint64 entries, host or device
 * The default kernel (TG_KERNEL_CYCLES) runs Alg. 1 for every edge, then
 * obtains the orbits that Alg. 2-3 enumerate per edge from identities over
 * Alg. 1's typed triangle counts plus two whole-graph enumerations (4-cycles
 * and 4-cliques, each met once in degree order), adds the closed forms,
 * reduces into a per-configuration histogram and divides by |E(H)|; the
 * other TG_KERNEL_* choices run Alg. 2-3 per edge as the paper does.  The
 * counts are the same.  Errors: TG_EINVAL,
 * TG_EOVERFLOW (the graph is too large for the 32-bit per-edge counters:
 * 2M >= 2^31), TG_EINTERNAL (a sum not divisible by |E(H)|), TG_ENOMEM,
 * TG_ECUDA.
 */
int tg_count_global(const tg_graph *g, int32_t k, uint64_t *out, void *stream);

/*
 * Per-edge typed counts (Def. "Local Typed Graphlet Counting").
 *   level  TG_GRAPHLET or TG_ORBIT
 *   rows   M x tg_slots(L, k, level) uint64, row-major, canonical edge order,
 *          host or device
 */
int tg_count_per_edge(const tg_graph *g, int32_t k, int32_t level, uint64_t *rows,
                      void *stream);

/*
 * Sparse per-edge counts (Sec. "Sparse Typed Motif Format"): only the nonzero
 * typed counts of each edge, as (id, count) pairs, edge after edge in
 * canonical edge order, each edge's pairs in slot order.  An id numbers every
 * typed graphlet (level TG_GRAPHLET: h1, h2, then h3..h8 for k = 4) or typed
 * orbit (TG_ORBIT: g1, g2, then g3..g12) consecutively, block by block, one
 * block per graphlet or orbit with its sorted type multisets of all the
 * subgraph's nodes in colex order (C(L+2,3) entries for 3-node blocks,
 * C(L+3,4) for 4-node ones); unlike a dense slot, an id means the same for
 * every edge.  tg_sparse_id is the lookup table back to the graphlet or orbit
 * and its types (tg_paper_hash of those gives the paper's key).
 *   offsets  M + 1 int64, host or device: edge e's pairs are the entries
 *            [offsets[e], offsets[e + 1]) of ids and counts
 *   ids      capacity uint32, counts capacity uint64: host or device, both
 *            or neither; with ids == counts == NULL only offsets and *nnz
 *            are written (a sizing call)
 *   nnz      receives the number of pairs (host)
 * The dense rows are formed in device scratch first (M x tg_slots(L, k,
 * level) uint64).  Errors: TG_EINVAL, TG_EOVERFLOW (nnz > capacity; offsets
 * and *nnz are still written), TG_ENOMEM, TG_ECUDA.  Synchronises `stream`.
 */
int tg_count_per_edge_sparse(const tg_graph *g, int32_t k, int32_t level, int64_t *offsets,
                             uint32_t *ids, uint64_t *counts, int64_t capacity, int64_t *nnz,
                             void *stream);

/* Number of sparse ids for (L, k, level); -1 for invalid arguments. */
int64_t tg_sparse_ids(int32_t L, int32_t k, int32_t level);

/* The graphlet (level TG_GRAPHLET: 1..8) or orbit (TG_ORBIT: 1..12) of a
 * sparse id and the sorted types of its k_out (3 or 4) nodes. */
int tg_sparse_id(int32_t L, int32_t k, int32_t level, int64_t id, int32_t *motif,
                 int32_t *types, int32_t *k_out);

/*
 * Undivided per-configuration sums over the canonical edge range [e0, e1):
 * sum over those edges of the per-edge graphlet counts, in the global layout.
 * Summing the outputs of disjoint ranges that cover [0, M) and passing the
 * total to tg_global_finalize gives tg_count_global's result; this is the
 * unit of work one rank does when the edges are sharded across GPUs.
 *   sums  tg_global_len(L, k) uint64, host or device
 */
int tg_count_range(const tg_graph *g, int32_t k, int64_t e0, int64_t e1, uint64_t *sums,
                   void *stream);

/*
 * One share of a global count split across `nshards` ranks (the unit of work
 * of one GPU when the count is sharded): undivided sums in the global layout
 * whose total over shard = 0 .. nshards - 1, passed to tg_global_finalize,
 * is tg_count_global's result (Sec. "Global Typed Graphlet Counts": the
 * global count is a sum over edges).  Every shard runs Alg. 1 over the whole
 * graph (the identities read the triangle counts of edges outside its
 * slice); the per-edge pass takes a slice of the edges balanced by their
 * Gamma_i lengths; the whole-graph 4-cycle and 4-clique enumerations take the
 * anchors and lowest nodes v with v mod nshards == shard, and each shard adds
 * the correction of its own cycle and clique totals (the correction is
 * linear in them).  No per-edge counters of the whole graph are kept.
 *   sums  tg_global_len(L, k) uint64, host or device; synchronises `stream`
 * Errors as tg_count_range; TG_EINVAL for shard outside [0, nshards).
 */
int tg_count_shard(const tg_graph *g, int32_t k, int32_t shard, int32_t nshards, uint64_t *sums,
                   void *stream);

/*
 * Divide undivided sums by |E(H)| (1 for edges, 2 for h1, 3 for h2, then
 * 3, 3, 4, 4, 5, 6 for h3..h8) on the host.  Returns TG_EINTERNAL if a sum is
 * not divisible.  `sums` and `out` are host arrays of tg_global_len(L, k)
 * entries (they may alias).
 */
int tg_global_finalize(int32_t L, int32_t k, const uint64_t *sums, uint64_t *out);

/*
 * Paper work model of the count (Thm. "time complexity for all 3 and 4-node
 * typed graphlet orbits"): for every edge (i, j), 2 d_i + d_j adjacency
 * entries for Alg. 1 (d_i <= d_j) plus sum over w in S_i u S_j u T_ij of d_w
 * for Alg. 2-3.  Writes the total entry count; computed on the GPU.
 */
int tg_work_model(const tg_graph *g, uint64_t *entries, void *stream);

/* ------------------------------------------ directed typed graphlets ---- */
/*
 * Directed typed 3-node graphlets (Sec. "Directed Typed Graphlets": the typed
 * neighbourhoods split into out- and in-neighbours, Gamma_i^{t,+} and
 * Gamma_i^{t,-}, and every combination of the split sets enumerated, each
 * directed typed motif with an id of its own).  The graph must have been
 * built with TG_DIRECTED; the underlying undirected graph is the one every
 * other call counts (a pair with arcs both ways is one edge whose two ends
 * are each other's out- and in-neighbour).
 *
 * A directed 3-node graphlet is a connected induced subgraph on three nodes
 * with its arcs; it is keyed by its isomorphism class and the sorted multiset
 * of its node types (as Def. "Typed Graphlet Instance").  The 13 classes, in
 * this order, are defined by these representatives on nodes A, B, C
 * (labels after the M-A-N triad census; the representative defines the class):
 *    0 021D  B->A, B->C            7 201   A<->B, B<->C
 *    1 021U  A->B, C->B            8 120D  B->A, B->C, A<->C
 *    2 021C  A->B, B->C            9 120U  A->B, C->B, A<->C
 *    3 111D  A<->B, C->B          10 120C  A->B, B->C, A<->C
 *    4 111U  A<->B, B->C          11 210   A->B, B<->C, A<->C
 *    5 030T  A->B, C->B, A->C     12 300   A<->B, B<->C, A<->C
 *    6 030C  A->B, B->C, C->A
 * Classes 0-4 and 7 have two underlying edges (paths), the others three.
 *
 * Per-edge rows (tg_count_directed_per_edge): M rows of tg_dir_slots(L) =
 * 13 L uint64 in canonical edge order (tg_edge_list); slot c L + t counts the
 * graphlets of class c on {i, j, w} with phi(w) = t containing the edge.
 * Global counts (tg_count_directed_global): tg_dir_global_len(L) =
 * 13 C(L+2, 3) uint64, class c's block at c C(L+2, 3), inside it the colex
 * rank of the sorted type multiset (as tg_config_rank with k = 3); each is
 * the per-edge sum divided by the class's number of underlying edges.
 * Errors: TG_EINVAL (NULL arguments, a graph built without TG_DIRECTED),
 * TG_ENOMEM, TG_ECUDA, TG_EINTERNAL (a sum not divisible).  `out`/`rows` are
 * host or device memory; synchronises `stream`.
 */
#define TG_TRIAD_CLASSES 13
int64_t tg_dir_slots(int32_t L);
int64_t tg_dir_global_len(int32_t L);
int tg_count_directed_per_edge(const tg_graph *g, uint64_t *rows, void *stream);
int tg_count_directed_global(const tg_graph *g, uint64_t *out, void *stream);

/*
 * Directed typed 4-node graphlets (same section; the paper lists no directed
 * 4-node motifs).  A directed 4-node graphlet is a connected induced subgraph
 * on four nodes with its arcs, keyed by its isomorphism class and the sorted
 * multiset of its node types.  There are 199 classes, numbered by canonical
 * code: the code of a digraph on positions 0..3 is the sum of 2^(4a + b) over
 * its arcs a -> b, its canonical code the smallest over the 24 relabellings,
 * and class c has the c-th smallest canonical code among the connected ones.
 * Per-edge rows: M rows of tg_dir4_slots(L) = 199 P uint64 (P = L(L+1)/2),
 * slot c P + pair(t, u) for the types t <= u of the two other nodes
 * (pair(a, b) = a L - a(a-1)/2 + (b - a)).  Global counts:
 * tg_dir4_global_len(L) = 199 C(L+3, 4), class c's block at c C(L+3, 4),
 * inside it the colex rank of the sorted type multiset; each the per-edge sum
 * divided by the class's number of underlying edges (3 to 6).  One warp per
 * edge enumerates the candidate sets {i, j, w, r} (w a neighbour of i or j, r
 * a later such neighbour or a neighbour of w): work grows with the square of
 * the endpoint degrees, so this form suits graphs of moderate degree.
 * Arguments, ownership and errors as tg_count_directed_*.
 */
#define TG_TETRAD_CLASSES 199
int64_t tg_dir4_slots(int32_t L);
int64_t tg_dir4_global_len(int32_t L);
int tg_count_directed4_per_edge(const tg_graph *g, uint64_t *rows, void *stream);
int tg_count_directed4_global(const tg_graph *g, uint64_t *out, void *stream);

/* ----------------------------------------------------- no allocation ---- */
/*
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory when they need a count: code running inside
 * an arena or pool that owns all device memory, plugins of a host program
 * that forbids allocation after start-up, or latency-critical loops that
 * cannot absorb cudaMalloc's implicit synchronisation.
 *
 * tg_count_global_noalloc computes the same result as tg_count_global (same
 * layout, same errors) but the library allocates nothing during the call: no
 * cudaMalloc, cudaFree, stream-ordered allocation or allocator callback.  Its
 * scratch (the undivided sums, a work counter, an error word) is one fixed
 * device array of (TG_NOALLOC_MAX_GLOBAL + 32) * 8 bytes (33 KB) that every
 * GPU which loads the library keeps until the process exits.
 *   - tg_global_len(L, k) must not exceed TG_NOALLOC_MAX_GLOBAL (k = 4 with
 *     L <= 9, or k = 3 with any L); larger requests return TG_EINVAL.
 *   - The first call on a device looks up the array's device address with
 *     that device current and loads the library's device code there; make
 *     that first call before any stream capture.  With the CUDA runtime's
 *     lazy module loading (the default), that first use is when the CUDA
 *     driver itself places the array and the kernels' code on the device, so
 *     a caller whose arena will own all device memory makes its first call
 *     (a one-edge graph will do) before the arena takes the device; later
 *     calls take no device memory at all.  Resetting the device between
 *     calls (cudaDeviceReset) is not supported: the address is cached.
 *   - All calls share the array.  Calls whose work overlaps on the GPU (other
 *     streams, other host threads) race on it and give wrong counts; order
 *     them on one stream or synchronise between them.
 *   - `out` is caller-owned host or device memory; the graph is an input
 *     built earlier (tg_build_csr).  Synchronises `stream`.
 * The counting kernel is the warp-per-edge form of Alg. 1-3 with binary-search
 * membership, so it suits graphs of moderate size and degree.
 */
#define TG_NOALLOC_MAX_GLOBAL 4096
int tg_count_global_noalloc(const tg_graph *g, int32_t k, uint64_t *out, void *stream);

/* ------------------------------------------------------------ tuning ---- */
#define TG_KERNEL_AUTO 0
#define TG_KERNEL_WARP_SEARCH 1 /* warp per edge, binary-search membership      */
#define TG_KERNEL_CTA_BITMAP 2  /* CTA per edge, shared-memory bitmap marks     */
#define TG_KERNEL_REUSE 3       /* Alg. 1 triangle counts reused for Alg. 2-3   */
#define TG_KERNEL_CYCLES 4      /* REUSE's identities, with 4-cycles and 4-cliques
                                   enumerated once over the whole graph (default) */

/*
 * Launch configuration of the counting kernels (process-wide).  Zero fields
 * mean "default".  Counts never depend on these values, only speed does.
 */
typedef struct {
    int32_t kernel;      /* TG_KERNEL_*                                     */
    int32_t cta_threads; /* threads per CTA of the bitmap kernel (32..1024) */
    int32_t unroll;      /* 1, 2 or 4 adjacency windows in flight per warp;
                            CYCLES kernel: 4-cycle anchors split over the
                            grid: 1 none, 4 all, 2 (default) the costly ones */
    int32_t hash_slots;  /* slots of the per-edge Gamma_i hash (power of 2);
                            CYCLES kernel: cap on the 4-clique candidates
                            staged per warp and on the per-warp far-end
                            table of the lightest 4-cycle anchors (global
                            counts); below 64 the costly 4-cycle anchors are
                            walked in member tiles instead of warp units    */
    int64_t bitmap_bits; /* cap on the node ids covered by the bitmap       */
    int32_t grid_limit;  /* cap on the CTAs of one counting launch          */
    int32_t edge_pass;   /* CYCLES kernel, k = 4: TG_EDGE_PASS_AUTO keeps the
                            per-edge T sums in memory between two kernels
                            when they fit in a quarter of free memory, else
                            runs the fused kernel; TG_EDGE_PASS_FUSED always
                            runs the fused kernel                           */
    int32_t edge_batch;  /* CYCLES kernel, k = 4: most edges whose T sums are
                            held in memory at once (the per-edge pass runs in
                            batches of work units); 0: as many as fit in a
                            quarter of free memory                          */
    int32_t c4_bin_fill; /* CYCLES kernel, global counts: a costly 4-cycle
                            anchor goes to the binned waves when its walk
                            averages at least this many wedges per far-end
                            window it spans (0: 32)                          */
} tg_tune;

#define TG_EDGE_PASS_AUTO 0
#define TG_EDGE_PASS_FUSED 1

int tg_set_tune(const tg_tune *t); /* NULL restores the defaults */
int tg_get_tune(tg_tune *t);

/*
 * Launch-configuration search for one graph class.  Times tg_count_global of
 * `g` (CUDA events on `stream`, one warm-up count first) under a coordinate
 * search that starts from the current tuning: unroll {2, 4}, then (k = 4)
 * c4_bin_fill {8, 32, 128} and edge_pass {AUTO, FUSED}, then hash_slots
 * {4096, 32}; a value is kept when it beats the best so far by 2 %.  The
 * winner becomes the process-wide tuning (as tg_set_tune) and is written to
 * `best` when non-NULL.  Results are cached per (device, L, k, bit length of
 * M, bit length of the maximum degree): a graph of a cached class takes the
 * cached tuning at once, with no count.  Uncached it costs about seven counts
 * of `g`.  Counts never depend on the result.  On error the tuning in force
 * before the call is restored.  Synchronises `stream`.
 */
int tg_autotune(const tg_graph *g, int32_t k, tg_tune *best, void *stream);
int tg_autotune_reset(void); /* forgets every cached class */

/* ---------------------------------------------------------- batches ----- */
/*
 * Many graphs counted together, by one of two paths:
 *  - persistent: every (graph, edge) pair is a work item; items are ordered
 *    by an estimate of their Alg. 2-3 work (heaviest first) in one shared
 *    queue that the warps of a single persistent launch drain (the paper's
 *    per-edge enumeration, binary-search membership); runs are replayed from
 *    a captured CUDA graph;
 *  - union: the graphs of each type count L form one disjoint union (built
 *    once per plan), counted per edge by the whole-graph path of
 *    tg_count_per_edge; each graph's rows are one block of the union's rows
 *    (copied to its output, or summed into its global counts).
 * The union is built unless tune->kernel is TG_KERNEL_WARP_SEARCH (persistent
 * only; with TG_KERNEL_CYCLES a union that cannot be built fails the call,
 * otherwise the plan falls back to the persistent path) and is used from the
 * start; tg_batch_tune times both paths and keeps the faster.  A plan holds the descriptors, the queue, the unions and their
 * row scratch (M_L x row width uint64 for the largest group).
 *
 * mode: TG_BATCH_GLOBAL        outs[g]: tg_global_len(L_g, k) uint64
 *       TG_BATCH_PER_EDGE_GRAPHLET / _ORBIT
 *                              outs[g]: M_g x tg_slots(L_g, k, level) uint64
 * outs[g] must be device memory (TG_EINVAL otherwise).  The graphs must stay
 * alive, and the outputs valid, for the life of the plan.
 */
#define TG_BATCH_GLOBAL 0
#define TG_BATCH_PER_EDGE_GRAPHLET 1
#define TG_BATCH_PER_EDGE_ORBIT 2

typedef struct tg_batch tg_batch;

/* Build a plan.  tune may be NULL; tune->cta_threads (if set) fixes the CTA
 * size of the persistent kernel.  Synchronises `stream`. */
int tg_batch_create(int32_t G, tg_graph *const *graphs, int32_t k, int32_t mode,
                    uint64_t *const *outs, const tg_tune *tune, void *stream, tg_batch **out);

/* One run of the plan (captured into a CUDA graph on first use and replayed
 * afterwards).  Synchronises `stream`; TG_EINTERNAL if a global sum is not
 * divisible by |E(H)|. */
int tg_batch_run(tg_batch *b, void *stream);

/* Autotuner: times the persistent kernel with 4, 8 and 16 warps per CTA, with
 * and without the cost-ordered queue, and the union path when the plan has
 * one; keeps the fastest (re-capturing the CUDA graph for the persistent
 * path).  *best_threads (may be NULL) receives the CTA size, negative when
 * the natural item order won, 0 when the union path won. */
int tg_batch_tune(tg_batch *b, void *stream, int32_t *best_threads);

int tg_batch_destroy(tg_batch *b);

/* One-shot form: create, autotune when tune == NULL, run, destroy. */
int tg_count_batch(int32_t G, tg_graph *const *graphs, int32_t k, int32_t mode,
                   uint64_t *const *outs, const tg_tune *tune, void *stream);

/* ---------------------------------------------------------- serving ----- */
/*
 * A serving loop for global-count requests on graphs of different sizes.
 * A dispatcher thread admits queued requests, in arrival order, whenever the
 * request's device-memory estimate fits the remaining budget and a slot is
 * free (a small request may pass a large one that waits for memory); admitted
 * requests run on `slots` worker threads, each with its own CUDA stream, so
 * their work overlaps on the GPU; a small admitted request (input pairs <=
 * batch_edges) takes further small queued requests along, up to batch_max,
 * and they run as one batched launch (continuous batching).
 */
typedef struct tg_server tg_server;

typedef struct {
    int32_t slots;            /* requests in flight at once (default 4)         */
    int32_t queue_cap;        /* queued requests before TG_EBUSY (default 4096) */
    int64_t mem_budget_bytes; /* device bytes admitted requests may use (8 GiB)  */
    int32_t device;           /* CUDA device of the server                       */
    int32_t batch_max;        /* most requests in one batched launch (32)        */
    int64_t batch_edges;      /* input pairs of a request that may be grouped
                                 (default 20000; 0 disables grouping)            */
} tg_serve_cfg;

typedef struct {
    int64_t n, m;             /* nodes, input pairs                              */
    const int32_t *src, *dst; /* host arrays of m ids (copied by submit)         */
    const uint8_t *type;      /* host array of n types (copied by submit)        */
    int32_t L, k;             /* types, graphlet size (3 or 4)                   */
} tg_request;

typedef struct {
    int32_t status;           /* TG_OK or the request's error                    */
    int32_t cuda_error;       /* cudaError_t behind a TG_ECUDA status, else 0    */
    int64_t len;              /* entries of the global histogram                 */
    double latency_ms;        /* submit to completion                            */
} tg_result;

typedef struct {
    uint64_t completed, failed, queued;
    double p50_ms, p99_ms, max_ms; /* latency of completed requests              */
    double graphs_per_s;           /* completed / (last completion - first submit) */
    int64_t peak_in_flight, peak_bytes;
    uint64_t batched_launches, grouped_requests;
} tg_serve_stats_t;

/* NULL cfg uses the defaults.  Returns NULL if the threads cannot start. */
tg_server *tg_serve_create(const tg_serve_cfg *cfg);

/* Copy the request and queue it.  TG_EINVAL (bad ids/types/sizes),
 * TG_ENOMEM_ADMIT (its estimate exceeds the whole budget: it can never run),
 * TG_EBUSY (queue full). */
int tg_serve_submit(tg_server *sv, const tg_request *req, uint64_t *ticket);

/* Wait up to timeout_ms for the ticket's result (TG_ETIMEDOUT otherwise; the
 * request stays pending).  On success the histogram (tg_global_len(L, k)
 * entries) is copied to the host array `out` of out_len entries and the ticket
 * is released.  TG_ENOTFOUND for unknown or already released tickets. */
int tg_serve_wait(tg_server *sv, uint64_t ticket, int32_t timeout_ms, uint64_t *out,
                  int64_t out_len, tg_result *info);

int tg_serve_stats(tg_server *sv, tg_serve_stats_t *stats);

/* Stop accepting work, run what is admitted, refuse what is queued (those
 * tickets complete with TG_EBUSY), join the threads and free the server. */
void tg_serve_destroy(tg_server *sv);

/* ------------------------------------------------------- allocation ----- */
/*
 * Route the library's device allocations through caller functions (for
 * example a framework's caching allocator).  alloc returns NULL on failure.
 * Pass NULLs to restore the default (cudaMallocAsync / cudaFreeAsync).
 * Not thread-safe with respect to calls in flight; set it once at start-up.
 */
typedef void *(*tg_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*tg_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
int tg_set_allocator(tg_alloc_fn alloc, tg_free_fn free_fn, void *ctx);

/*
 * Scratch kept between calls (default allocation path only).  With bytes = 0
 * (the default) scratch comes from the device's default stream-ordered pool,
 * which hands freed memory back to the device at each synchronisation, so
 * every call maps its scratch anew (milliseconds for the gigabytes a large
 * count needs).  With bytes > 0 the library allocates from a pool of its own
 * per device that keeps up to `bytes` of freed scratch mapped for later calls;
 * other allocators in the process cannot use that memory meanwhile.
 * tg_set_memory_retention(0) also releases what the pools hold;
 * tg_trim_memory releases it and keeps the setting.  TG_ECUDA on a failed
 * CUDA call (tg_last_cuda_error has its code).
 */
int tg_set_memory_retention(uint64_t bytes);
int tg_trim_memory(void);

/* ------------------------------------------------------- measurement ---- */
/* Kernels launched by this library since it was loaded. */
uint64_t tg_launch_count(void);

/* The cudaError_t value of the last CUDA call of this library that failed on
 * the calling host thread (the cause of its last TG_ECUDA), or 0. */
int32_t tg_last_cuda_error(void);

/*
 * Timing and work of the calling host thread's last counting call that used
 * the REUSE or CYCLES kernel (CUDA events recorded on that call's stream
 * around each phase).  Waits for those events.  Returns TG_ENOTFOUND before
 * any such call on this thread.  Each host thread keeps its own record, so
 * calls made concurrently from several threads do not mix.  Phases a kernel
 * does not have read 0.
 */
typedef struct {
    double tau_ms;            /* Alg. 1 typed triangle counts, every edge   */
    double aggregate_ms;      /* per-node sums of tau and typed degrees     */
    double count_ms;          /* per-edge pass: identities, closed forms,
                                 output                                      */
    uint64_t edges;           /* edges counted                               */
    uint64_t gamma_entries;   /* entries of Gamma_i read by the per-edge pass */
    uint64_t walked_entries;  /* REUSE: entries of S_i / T lists walked      */
    uint64_t probe_pairs;     /* REUSE: (T member, T member) adjacency probes */
    uint64_t t_members;       /* T members whose tau rows were read          */
    double cycles_ms;         /* CYCLES: 4-cycle enumeration                 */
    double cliques_ms;        /* CYCLES: 4-clique enumeration                */
    uint64_t wedges;          /* CYCLES: degree-ordered wedges (per pass)    */
    uint64_t clique_tests;    /* CYCLES: candidate tests of the clique search
                                 (pairs (v, w) for the bitmap kernels)       */
    uint64_t cliques;         /* CYCLES: 4-cliques found                     */
} tg_timing;

int tg_last_timing(tg_timing *out);

/* Failure injection for tests: make the n-th device allocation from now on
 * fail (n >= 1), or disable with n = 0.  Host-side only: the allocation is
 * refused before any CUDA call is made. */
int tg_debug_fail_alloc(int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* TG_H */
