// Device primitives of the library: stream-ordered allocation with failure
// injection, exclusive scans and a stable LSD radix sort on uint64 keys.
// All kernels here are this library's own; no vendor sort or scan is used.
#include <atomic>
#include <mutex>
#include <utility>
#include <vector>

#include "tg_internal.cuh"

// ------------------------------------------------------------ allocation --
static tg_alloc_fn g_alloc = nullptr;
static tg_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;
static std::atomic<int64_t> g_fail_countdown{0};
static std::atomic<uint64_t> g_launches{0};

void tg_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static thread_local int32_t g_cuda_error = 0;

void tg_note_cuda_error(cudaError_t e) { g_cuda_error = (int32_t)e; }

extern "C" int32_t tg_last_cuda_error(void) { return g_cuda_error; }

extern "C" uint64_t tg_launch_count(void) { return g_launches.load(); }

int tg_num_sms() {
    int dev = 0, sms = 0;
    (void)cudaGetDevice(&dev);
    (void)cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

int tg_smem_optin() {
    int dev = 0, v = 0;
    (void)cudaGetDevice(&dev);
    (void)cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v > 0 ? v : 48 * 1024;
}

// (device, kernel) pairs whose limit is already raised: the attribute is set
// once per kernel and device, not before every launch.
static std::mutex g_smem_mu;
static std::vector<std::pair<int, const void *>> g_smem_done;

int tg_allow_max_smem(const void *func) {
    int dev = 0, optin = 0;
    TG_TRY_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(g_smem_mu);
        for (const auto &d : g_smem_done)
            if (d.first == dev && d.second == func) return TG_OK;
    }
    TG_TRY_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    TG_TRY_CUDA(cudaFuncGetAttributes(&fa, func));
    const int v = optin - (int)fa.sharedSizeBytes;
    if (v <= 0) return TG_EINVAL;
    TG_TRY_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
    std::lock_guard<std::mutex> lk(g_smem_mu);
    g_smem_done.emplace_back(dev, func);
    return TG_OK;
}

extern "C" int tg_set_allocator(tg_alloc_fn alloc, tg_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) return TG_EINVAL;
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = ctx;
    return TG_OK;
}

extern "C" int tg_debug_fail_alloc(int64_t n) {
    if (n < 0) return TG_EINVAL;
    g_fail_countdown.store(n);
    return TG_OK;
}

// Retained scratch: with a positive retention the library allocates from a
// pool of its own per device whose release threshold is that many bytes, so
// freed scratch stays mapped for the next call instead of going back to the
// device at each synchronisation.
constexpr int kMaxDevices = 64;
static std::mutex g_pool_mu;
static std::atomic<uint64_t> g_retain{0};
static cudaMemPool_t g_pools[kMaxDevices] = {};

static cudaMemPool_t lib_pool(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        uint64_t thr = g_retain.load();
        (void)cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}

extern "C" int tg_set_memory_retention(uint64_t bytes) {
    g_retain.store(bytes);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int d = 0; d < kMaxDevices; ++d) {
        if (!g_pools[d]) continue;
        uint64_t thr = bytes;
        if (cudaMemPoolSetAttribute(g_pools[d], cudaMemPoolAttrReleaseThreshold, &thr) != cudaSuccess ||
            (bytes == 0 && cudaMemPoolTrimTo(g_pools[d], 0) != cudaSuccess)) {
            tg_note_cuda_error(cudaGetLastError());
            return TG_ECUDA;
        }
    }
    return TG_OK;
}

extern "C" int tg_trim_memory(void) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int d = 0; d < kMaxDevices; ++d) {
        if (g_pools[d] && cudaMemPoolTrimTo(g_pools[d], 0) != cudaSuccess) {
            tg_note_cuda_error(cudaGetLastError());
            return TG_ECUDA;
        }
    }
    return TG_OK;
}

void *tg_dalloc(size_t bytes, cudaStream_t s) {
    int64_t c = g_fail_countdown.load();
    while (c > 0) {
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) {
            if (c == 1) return nullptr;  // the injected failure
            break;
        }
    }
    if (g_alloc) return g_alloc(bytes, s, g_alloc_ctx);
    void *p = nullptr;
    cudaMemPool_t pool = nullptr;
    if (g_retain.load() > 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) pool = lib_pool(dev);
    }
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return p;
}

void tg_dfree(void *p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (g_free) {
        g_free(p, bytes, s, g_alloc_ctx);
        return;
    }
    (void)cudaFreeAsync(p, s);
}

bool tg_is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int tg_bitlen(uint64_t x) {
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

// ------------------------------------------------------------------ scans --
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T *warp_tot, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (kScanThreads / 32) ? warp_tot[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < (kScanThreads / 32)) warp_tot[lane] = wi - w;
        if (lane == (kScanThreads / 32) - 1) *total = wi;
    }
    __syncthreads();
    T r = x - v + warp_tot[warp];
    __syncthreads();
    return r;
}

template <typename T>
__global__ void k_tile_reduce(const T *in, int64_t n, T *partial) {
    __shared__ T wt[kScanThreads / 32];
    __shared__ T tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (base + q < n) s += in[base + q];
    (void)block_exclusive_scan<T>(s, wt, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_tile_scan(const T *in, T *out, int64_t n, const T *offsets) {
    __shared__ T wt[kScanThreads / 32];
    __shared__ T tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        v[q] = (base + q < n) ? in[base + q] : T(0);
        s += v[q];
    }
    T run = block_exclusive_scan<T>(s, wt, &tot) + (offsets ? offsets[blockIdx.x] : T(0));
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (base + q < n) out[base + q] = run;
        run += v[q];
    }
}

template <typename T>
int scan_impl(const T *in, T *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return TG_OK;
    int64_t blocks = (n + kScanTile - 1) / kScanTile;
    if (blocks == 1) {
        k_tile_scan<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
        return TG_OK;
    }
    DevBuf<T> part;
    if (!part.alloc(blocks, s)) return TG_ENOMEM;
    k_tile_reduce<T><<<(unsigned)blocks, kScanThreads, 0, s>>>(in, n, part.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    TG_TRY(scan_impl<T>(part.p, part.p, blocks, s));
    k_tile_scan<T><<<(unsigned)blocks, kScanThreads, 0, s>>>(in, out, n, part.p); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    return TG_OK;
}

}  // namespace

int tg_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<uint32_t>(in, out, n, s);
}
int tg_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, s);
}

// ------------------------------------------------------------- radix sort --
// One pass sorts on an 8-bit digit.  A tile of kSortTile keys belongs to one
// block; each of its 8 warps owns kSortItems consecutive chunks of 32 keys.
// Ranks inside a chunk come from __match_any_sync, so the pass is stable.
namespace {

constexpr int kSortWarps = 8;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortWarps * 32 * kSortItems;  // 4096 keys

__global__ void k_sort_hist(const uint64_t *in, int64_t n, int shift, uint32_t *hist,
                            int64_t nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int q = threadIdx.x; q < kSortTile; q += blockDim.x) {
        int64_t i = base + q;
        if (i < n) atomicAdd(&h[(in[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_sort_scatter(const uint64_t *in, uint64_t *out, const uint32_t *vin,
                               uint32_t *vout, int64_t n, int shift, const uint32_t *offs,
                               int64_t nblocks) {
    __shared__ uint32_t wcnt[kSortWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < kSortWarps * 256; q += blockDim.x) (&wcnt[0][0])[q] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    int64_t wbase = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * 32 * kSortItems;
    uint64_t key[kSortItems];
    uint32_t val[kSortItems];
    uint32_t rank[kSortItems];
#pragma unroll
    for (int c = 0; c < kSortItems; ++c) {
        int64_t i = wbase + c * 32 + lane;
        bool valid = i < n;
        key[c] = valid ? in[i] : 0;
        val[c] = (valid && vin) ? vin[i] : 0u;
        uint32_t d = valid ? (uint32_t)((key[c] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = valid ? wcnt[warp][d] : 0;
        __syncwarp();
        rank[c] = before + __popc(peers & lt);
        int leader = 31 - __clz(peers);
        if (valid && lane == leader) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        uint32_t run = 0;
        int d = threadIdx.x;  // blockDim.x == 256
        for (int w = 0; w < kSortWarps; ++w) {
            uint32_t t = wcnt[w][d];
            wcnt[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kSortItems; ++c) {
        int64_t i = wbase + c * 32 + lane;
        if (i < n) {
            uint32_t d = (uint32_t)((key[c] >> shift) & 255u);
            uint32_t pos = offs[(int64_t)d * nblocks + blockIdx.x] + wcnt[warp][d] + rank[c];
            out[pos] = key[c];
            if (vout) vout[pos] = val[c];
        }
    }
}

}  // namespace

int tg_radix_sort_kv(uint64_t *keys, uint64_t *tmp, uint32_t *vals, uint32_t *vtmp, int64_t n,
                     int bits, cudaStream_t s, uint64_t **result, uint32_t **vresult) {
    *result = keys;
    if (vresult) *vresult = vals;
    if (n <= 1 || bits <= 0) return TG_OK;
    if (n >= (int64_t)UINT32_MAX) return TG_EOVERFLOW;
    int64_t nblocks = (n + kSortTile - 1) / kSortTile;
    DevBuf<uint32_t> hist;
    if (!hist.alloc((size_t)nblocks * 256, s)) return TG_ENOMEM;
    uint64_t *a = keys, *b = tmp;
    uint32_t *va = vals, *vb = vtmp;
    for (int shift = 0; shift < bits; shift += 8) {
        k_sort_hist<<<(unsigned)nblocks, 256, 0, s>>>(a, n, shift, hist.p, nblocks); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
        TG_TRY(tg_scan_u32(hist.p, hist.p, nblocks * 256, s));
        k_sort_scatter<<<(unsigned)nblocks, kSortWarps * 32, 0, s>>>(a, b, va, vb, n, shift,
                                                                     hist.p, nblocks); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
        uint64_t *t = a;
        a = b;
        b = t;
        uint32_t *vt = va;
        va = vb;
        vb = vt;
    }
    *result = a;
    if (vresult) *vresult = va;
    return TG_OK;
}

int tg_radix_sort_u64(uint64_t *keys, uint64_t *tmp, int64_t n, int bits, cudaStream_t s,
                      uint64_t **result) {
    return tg_radix_sort_kv(keys, tmp, nullptr, nullptr, n, bits, s, result, nullptr);
}
