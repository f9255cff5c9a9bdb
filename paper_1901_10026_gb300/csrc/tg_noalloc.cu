// Global typed counts without any allocation by the library.
//
// Some callers cannot allocate device memory at the point where they need a
// count: code running inside a custom memory pool or arena that owns every
// byte of the device, plugins of a host application that forbids allocation
// calls after start-up, or real-time loops where cudaMalloc's implicit
// synchronisation is not acceptable.  tg_count_global_noalloc serves them: the
// only scratch it needs (the undivided per-configuration sums, a work counter
// and an error word) lives in a fixed, file-scope device array that every GPU
// loading this library holds until the process exits.
//
// The kernel is a variant of the warp-per-edge counter (Alg. 1-3, membership
// by binary search in the (type, id)-sorted lists, closed forms of Sec.
// "Combinatorial Relationships"), accumulating straight into that array.
#include <mutex>

#include "tg_device.cuh"

using namespace tgd;

namespace {

constexpr int kNaWarps = 8;
constexpr int kNaBlock = kNaWarps * 32;
constexpr int kNaMaxDevices = 64;
enum { C3 = 0, C6 = 1, C7 = 2, C8 = 3, C10 = 4, C12 = 5, CN = 6 };

}  // namespace

// The fixed scratch: TG_NOALLOC_MAX_GLOBAL sums, then the work counter and
// the error word.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[TG_NOALLOC_MAX_GLOBAL + 32];

namespace {

struct NaParams {
    const int64_t *rowptr;
    const uint32_t *adj;
    const int32_t *toff;
    const uint8_t *ntype;
    const int2 *edges;
    int64_t M;
    int32_t L, P, k;
    unsigned long long *sums;
    unsigned long long *queue;
    int64_t off1, off2, off4, n4;
};

__global__ void __launch_bounds__(kNaBlock) k_noalloc_count(NaParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = p.L, P = p.P;
    const size_t wbytes = ((size_t)CN * P * 4 + 3 * 16 * 4 + 15) & ~(size_t)15;
    int *cnt = reinterpret_cast<int *>(smem + warp * wbytes);
    unsigned *Tn = reinterpret_cast<unsigned *>(smem + warp * wbytes + (size_t)CN * P * 4);
    unsigned *Si = Tn + 16;
    unsigned *Sj = Si + 16;
    const int64_t *__restrict__ rowptr = p.rowptr;
    const uint32_t *__restrict__ adj = p.adj;
    const int32_t *__restrict__ toff = p.toff;

    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(p.queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= (unsigned long long)p.M) break;
        const int2 ab = p.edges[item];
        const int j = min(ab.x, ab.y), i = max(ab.x, ab.y);
        const int ti = p.ntype[i], tj = p.ntype[j];
        const int64_t bi = rowptr[i], bj = rowptr[j];
        const int di = (int)(rowptr[i + 1] - bi), dj = (int)(rowptr[j + 1] - bj);
        const int32_t *toi = toff + (int64_t)i * (L + 1);
        const int32_t *toj = toff + (int64_t)j * (L + 1);
        for (int x = lane; x < CN * P; x += 32) cnt[x] = 0;
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
        // Alg. 2 and 3: every w_k of S_i u S_j u T, one lane per neighbour w_r
        if (p.k == 4) {
            for (int side = 0; side < 2; ++side) {
                const int64_t sb = side == 0 ? bi : bj;
                const int sd = side == 0 ? di : dj;
                for (int y = 0; y < sd; ++y) {
                    const uint32_t wk = __ldg(adj + sb + y);
                    const int kid = (int)(wk & TG_IDMASK), kt = (int)(wk >> TG_TSHIFT);
                    int cls;
                    if (side == 0) {
                        if (kid == j) continue;
                        cls = contains(adj, bj, toj, wk) ? CLS_T : CLS_SI;
                    } else {
                        if (kid == i || contains(adj, bi, toi, wk)) continue;
                        cls = CLS_SJ;
                    }
                    const int64_t kb = rowptr[kid];
                    const int dk = (int)(rowptr[kid + 1] - kb);
                    for (int x = lane; x < dk; x += 32) {
                        const uint32_t wr = __ldg(adj + kb + x);
                        const int rid = (int)(wr & TG_IDMASK);
                        if (rid == i || rid == j) continue;
                        const int rc = (contains(adj, bi, toi, wr) ? 1 : 0) |
                                       (contains(adj, bj, toj, wr) ? 2 : 0);
                        const int pr = pair_index(L, kt, (int)(wr >> TG_TSHIFT));
                        if (rc == CLS_I) {
                            atomicAdd(&cnt[(cls == CLS_T ? C8 : C3) * P + pr], 1);
                        } else if (cls == CLS_SI) {
                            if (rc == CLS_SI && rid < kid) atomicAdd(&cnt[C7 * P + pr], 1);
                        } else if (cls == CLS_SJ) {
                            if (rc == CLS_SJ && rid < kid)
                                atomicAdd(&cnt[C7 * P + pr], 1);
                            else if (rc == CLS_SI)
                                atomicAdd(&cnt[C6 * P + pr], 1);
                        } else {
                            if (rc == CLS_T) {
                                if (rid < kid) atomicAdd(&cnt[C12 * P + pr], 1);
                            } else {
                                atomicAdd(&cnt[C10 * P + pr], 1);
                            }
                        }
                    }
                }
            }
            __syncwarp();
        }
        // closed forms and the undivided sums
        if (lane == 0) {
            int a = ti, b = tj;
            sort2(a, b);
            atomicAdd(p.sums + a + (b + 1) * b / 2, 1ull);
        }
        for (int t = lane; t < L; t += 32) {
            int a = ti, b = tj, c = t;
            sort2(a, b);
            sort2(b, c);
            sort2(a, b);
            const int64_t r = colex3(a, b, c);
            if (Si[t] + Sj[t]) atomicAdd(p.sums + p.off1 + r, (unsigned long long)Si[t] + Sj[t]);
            if (Tn[t]) atomicAdd(p.sums + p.off2 + r, (unsigned long long)Tn[t]);
        }
        if (p.k == 4) {
            for (int pr = lane; pr < P; pr += 32) {
                int t, u;
                unpair(L, pr, t, u);
                const uint64_t sit = Si[t], siu = Si[u], sjt = Sj[t], sju = Sj[u];
                const uint64_t tt = Tn[t], tu = Tn[u];
                const uint64_t g3 = (uint64_t)cnt[C3 * P + pr], g6 = (uint64_t)cnt[C6 * P + pr];
                const uint64_t g7 = (uint64_t)cnt[C7 * P + pr], g8 = (uint64_t)cnt[C8 * P + pr];
                const uint64_t g10 = (uint64_t)cnt[C10 * P + pr], g12 = (uint64_t)cnt[C12 * P + pr];
                uint64_t g4, g5, g9, g11;
                closed_forms(t == u, sit, siu, sjt, sju, tt, tu, g6, g7, g10, g12, g4, g5, g9, g11);
                const uint64_t h[6] = {g3 + g4, g5, g6, g7 + g8 + g9, g10 + g11, g12};
                int a = ti, b = tj, c = t, d = u;
                sort2(a, b);
                sort2(c, d);
                sort2(a, c);
                sort2(b, d);
                sort2(b, c);
                const int64_t r = colex4(a, b, c, d);
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    if (h[q]) atomicAdd(p.sums + p.off4 + q * p.n4 + r, (unsigned long long)h[q]);
            }
        }
        __syncwarp();
    }
}

// Divide the sums by |E(H)| into out (device), or in place when out is NULL.
__global__ void k_noalloc_finalize(unsigned long long *sums, uint64_t *out, int64_t len,
                                   int64_t off1, int64_t off2, int64_t off4, int64_t n4,
                                   unsigned long long *err) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < len;
         x += (int64_t)gridDim.x * blockDim.x) {
        uint64_t d = 1;
        if (x >= off4)
            d = (uint64_t)(((x - off4) / n4) < 2 ? 3 : ((x - off4) / n4) < 4 ? 4 : ((x - off4) / n4) == 4 ? 5 : 6);
        else if (x >= off2)
            d = 3;
        else if (x >= off1)
            d = 2;
        const uint64_t v = sums[x];
        if (v % d) atomicOr(err, 1ull);
        if (out)
            out[x] = v / d;
        else
            sums[x] = v / d;
    }
}

std::mutex g_na_mu;
void *g_na_ptr[kNaMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, set up once per
// device with that device current.  The set-up also loads the two kernels:
// under the CUDA runtime's lazy module loading, the driver places a module's
// code and its __device__ arrays on a device when they are first used there,
// so this first call is where the driver itself may take device memory; later
// calls take none.  The cached address belongs to the device's primary
// context: resetting the device between calls is not supported.
int scratch_address(unsigned long long **out) {
    int dev = 0;
    TG_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) return TG_EINVAL;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            tg_note_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
            (void)cudaGetLastError();
            return TG_ECUDA;
        }
        cudaFuncAttributes fa{};
        TG_TRY_CUDA(cudaFuncGetAttributes(&fa, (const void *)k_noalloc_count));
        TG_TRY_CUDA(cudaFuncGetAttributes(&fa, (const void *)k_noalloc_finalize));
        TG_TRY(tg_allow_max_smem((const void *)k_noalloc_count));
        g_na_ptr[dev] = ptr;
    }
    *out = static_cast<unsigned long long *>(g_na_ptr[dev]);
    return TG_OK;
}

}  // namespace

extern "C" int tg_count_global_noalloc(const tg_graph *g, int32_t k, uint64_t *out,
                                       void *stream) {
    if (!g || !out || (k != 3 && k != 4)) return TG_EINVAL;
    const int L = g->L;
    const int64_t len = tg_global_len(L, k);
    if (len <= 0 || len > TG_NOALLOC_MAX_GLOBAL) return TG_EINVAL;
    if (2 * g->M >= ((int64_t)1 << 31)) return TG_EOVERFLOW;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *scratch = nullptr;
    TG_TRY(scratch_address(&scratch));
    unsigned long long *sums = scratch;
    unsigned long long *queue = scratch + TG_NOALLOC_MAX_GLOBAL;
    unsigned long long *err = scratch + TG_NOALLOC_MAX_GLOBAL + 1;
    // the array keeps the previous call's contents: clear what starts at zero
    TG_TRY_CUDA(cudaMemsetAsync(sums, 0, (size_t)len * 8, s));
    TG_TRY_CUDA(cudaMemsetAsync(queue, 0, 2 * 8, s));
    NaParams p{};
    p.rowptr = g->rowptr;
    p.adj = g->adj;
    p.toff = g->toff;
    p.ntype = g->ntype;
    p.edges = g->edges;
    p.M = g->M;
    p.L = L;
    p.P = L * (L + 1) / 2;
    p.k = k;
    p.sums = sums;
    p.queue = queue;
    p.off1 = tg_binom(L + 1, 2);
    p.off2 = p.off1 + tg_binom(L + 2, 3);
    p.off4 = p.off1 + 2 * tg_binom(L + 2, 3);
    p.n4 = tg_binom(L + 3, 4);
    if (g->M > 0) {
        const size_t wbytes = ((size_t)CN * p.P * 4 + 3 * 16 * 4 + 15) & ~(size_t)15;
        const size_t smem = kNaWarps * wbytes;
        TG_TRY(tg_allow_max_smem((const void *)k_noalloc_count));
        int dev = 0, sms = 1, per_sm = 1;
        TG_TRY_CUDA(cudaGetDevice(&dev));
        TG_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        TG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_noalloc_count,
                                                                  kNaBlock, smem));
        int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
        const int64_t need = (g->M + kNaWarps - 1) / kNaWarps;
        if (grid > need) grid = need;
        k_noalloc_count<<<(unsigned)grid, kNaBlock, smem, s>>>(p); tg_note_launch();
        TG_TRY_CUDA(cudaGetLastError());
    }
    const bool dev_out = tg_is_device_ptr(out);
    const int64_t blocks = (len + 255) / 256;
    k_noalloc_finalize<<<(unsigned)blocks, 256, 0, s>>>(sums, dev_out ? out : nullptr, len, p.off1,
                                                       p.off2, p.off4, p.n4, err); tg_note_launch();
    TG_TRY_CUDA(cudaGetLastError());
    unsigned long long herr = 0;
    TG_TRY_CUDA(cudaMemcpyAsync(&herr, err, 8, cudaMemcpyDeviceToHost, s));
    if (!dev_out) TG_TRY_CUDA(cudaMemcpyAsync(out, sums, (size_t)len * 8, cudaMemcpyDeviceToHost, s));
    TG_TRY_CUDA(cudaStreamSynchronize(s));
    return herr ? TG_EINTERNAL : TG_OK;
}
