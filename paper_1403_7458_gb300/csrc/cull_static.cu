// cull_static.cu -- a variant of the culling pass that allocates nothing.
//
// Some callers cannot allocate device memory: codes that hand all of HBM to
// their own memory pool up front (so any cudaMalloc would fail or fragment
// the pool), and latency-critical host loops where the implicit device
// synchronisation of cudaMalloc/cudaFree is not acceptable.  For them,
// spamm_cull_noalloc() takes the two leaf-norm grids and the output buffers
// from the caller and keeps its only scratch -- the per-output-leaf counts --
// in a fixed, file-scope device array.
//
// Limits and sharing rules:
//   - the scratch holds SPAMM_NOALLOC_MAX_NB^2 int32 counts (4 MiB), so the
//     leaf grid is limited to nb <= SPAMM_NOALLOC_MAX_NB; every GPU that loads
//     this library holds that array until the process exits;
//   - all calls share the one array; two calls whose work overlaps on the GPU
//     (e.g. on two streams without ordering between them) race on it;
//   - the array keeps the previous call's counts; every count a call reads is
//     written earlier in the same call, so nothing has to start at zero.
//   - every call looks up the array's device address in the current context
//     with cudaGetSymbolAddress; the first call on a device may load the
//     module, so make it before any stream capture.

#include "internal.cuh"

#define SPAMM_NOALLOC_MAX_NB 1024

static __device__ __align__(256) int32_t g_noalloc_counts[SPAMM_NOALLOC_MAX_NB * SPAMM_NOALLOC_MAX_NB];

namespace {

constexpr int kWarps = 8;
constexpr int kScanThreads = 1024;

// Device address of the scratch array in the current context, looked up on
// every call: an address cached per device ordinal would go stale when the
// context is destroyed and recreated (cudaDeviceReset), and the lookup is
// cheap once the module is loaded.  The first call on a device may load the
// module, so it belongs before any stream capture.
int scratch_address(int32_t **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_counts);
    if (e != cudaSuccess || !p)
        return spamm_cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress(g_noalloc_counts)",
                               __FILE__, __LINE__);
    *out = static_cast<int32_t *>(p);
    return SPAMM_OK;
}

// B's leaf norms are read in place (row-major, stride ldb), one column per
// warp: no transposed copy is made.
__global__ void __launch_bounds__(kWarps * 32)
k_noalloc_count(const double *__restrict__ n2A, int64_t lda, const double *__restrict__ n2B,
                int64_t ldb, int64_t nb, double tau2, int32_t *__restrict__ counts)
{
    int64_t g = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (g >= nb * nb) return;
    int64_t i = g / nb, j = g % nb;
    int cnt = 0;
    for (int64_t k0 = 0; k0 < nb; k0 += 32) {
        int64_t k = k0 + lane;
        bool p = k < nb && keep_product(n2A[i * lda + k], n2B[k * ldb + j], tau2);
        cnt += __popc(__ballot_sync(0xffffffffu, p));
    }
    if (lane == 0) counts[g] = cnt;
}

__global__ void __launch_bounds__(kScanThreads)
k_noalloc_scan(const int32_t *__restrict__ counts, int64_t G, int64_t *__restrict__ off)
{
    __shared__ int64_t part[kScanThreads];
    int t = threadIdx.x;
    int64_t chunk = (G + kScanThreads - 1) / kScanThreads;
    int64_t lo = t * chunk, hi = lo + chunk < G ? lo + chunk : G;
    int64_t s = 0;
    for (int64_t q = lo; q < hi; q++) s += counts[q];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        int64_t v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - s;
    for (int64_t q = lo; q < hi; q++) {
        off[q] = run;
        run += counts[q];
    }
    if (t == kScanThreads - 1) off[G] = part[t];
}

__global__ void __launch_bounds__(kWarps * 32)
k_noalloc_emit(const double *__restrict__ n2A, int64_t lda, const double *__restrict__ n2B,
               int64_t ldb, int64_t nb, double tau2, const int64_t *__restrict__ off,
               uint32_t *__restrict__ klist, int64_t cap)
{
    int64_t g = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (g >= nb * nb) return;
    if (off[g + 1] > cap) return;  // the caller sees off[nb*nb] > cap
    int64_t i = g / nb, j = g % nb;
    int64_t base = off[g];
    unsigned lt = (1u << lane) - 1u;
    for (int64_t k0 = 0; k0 < nb; k0 += 32) {
        int64_t k = k0 + lane;
        bool p = k < nb && keep_product(n2A[i * lda + k], n2B[k * ldb + j], tau2);
        unsigned m = __ballot_sync(0xffffffffu, p);
        if (p) klist[base + __popc(m & lt)] = (uint32_t)k;
        base += __popc(m);
    }
}

}  // namespace

extern "C" int spamm_cull_noalloc(const double *n2A, int64_t lda, const double *n2B, int64_t ldb,
                                  int64_t nb, double tau, int64_t *off, uint32_t *klist, int64_t cap,
                                  void *stream)
{
    if (!n2A || !n2B || !off || nb < 1 || lda < nb || ldb < nb || cap < 0 || (cap > 0 && !klist) ||
        !(tau >= 0.0) || tau > 1e300) {
        spamm_set_error("spamm_cull_noalloc: bad arguments");
        return SPAMM_E_INVAL;
    }
    if (nb > SPAMM_NOALLOC_MAX_NB) {
        spamm_set_error("spamm_cull_noalloc: nb = %lld exceeds the fixed scratch limit %d",
                        (long long)nb, SPAMM_NOALLOC_MAX_NB);
        return SPAMM_E_CAPACITY;
    }
    int32_t *counts = nullptr;
    int rc = scratch_address(&counts);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t G = nb * nb;
    const double tau2 = tau * tau;
    const unsigned blocks = (unsigned)((G + kWarps - 1) / kWarps);
    k_noalloc_count<<<blocks, kWarps * 32, 0, s>>>(n2A, lda, n2B, ldb, nb, tau2, counts);
    SPAMM_CK_LAUNCH();
    k_noalloc_scan<<<1, kScanThreads, 0, s>>>(counts, G, off);
    SPAMM_CK_LAUNCH();
    if (cap > 0) {
        k_noalloc_emit<<<blocks, kWarps * 32, 0, s>>>(n2A, lda, n2B, ldb, nb, tau2, off, klist, cap);
        SPAMM_CK_LAUNCH();
    }
    return SPAMM_OK;
}
