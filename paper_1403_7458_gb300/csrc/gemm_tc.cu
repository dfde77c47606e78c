// gemm_tc.cu -- grouped leaf products on the tcgen05 tensor cores with exact
// BF16 slices (the mixed-precision form of Algorithm 1's leaf branch).
//
// Tiles.  A tile is four consecutive output leaf rows i = 4I..4I+3 and one
// output leaf column j (M = 128 rows, N = 32 columns).  Its work list holds
// every k for which at least one of the four triples (i, k, j) survives the
// culling test of Eq. 4, with a 4-bit mask of the survivors; leaves of culled
// triples are replaced by zeros, so each output leaf receives exactly the
// products of its own task list (no extra products, no missing ones).
//
// Slices.  With s slices per operand (see slice.cu), the MMA for A slice p
// multiplies the 128 x 32 A slab by B slices 0..s-1-p (N = 32 (s - p)) and
// accumulates into TMEM columns [32p, 32s): column block d then holds the
// exact integer S_d = sum_{p+q=d} sum_k sum_l dA_p dB_q.  Pairs with
// p + q >= s are never formed.  The epilogue forms
//     C = 2^(sigmaA + sigmaB - 7s - 7) * sum_d S_d 128^(s-1-d)
// with integer arithmetic and one rounding to FP64.
//
// Kernel roles (192 threads, one CTA per SM, persistent):
//   warp 0     : producer; bulk-copies (cp.async.bulk) 4 A leaves + 1 B leaf
//                per work item into a 3-stage ring (zero leaves come from a
//                zero page), completion on the stage's mbarrier;
//   warp 1     : allocates 512 TMEM columns; lane 0 issues 2s tcgen05.mma per
//                work item and commits to the stage's "empty" barrier and, at
//                the end of a tile, to the accumulator's "full" barrier;
//   warps 2-5  : epilogue; tcgen05.ld of the s diagonal blocks of the row the
//                thread owns, integer combine, FP64 store, diagonal traces.
// Two accumulators (TMEM columns 0 and 256) let the epilogue of one tile run
// under the MMAs of the next.  Every wait is bounded (%globaltimer); on
// timeout the kernel records the error, drains and frees TMEM, and returns.
//
// Roofline: tensor pipe.  Useful work 2 b^3 per surviving triple; issued
// tensor work 2 * 128 * 32 * 32 * s(s+1)/2 per work item.
#include "internal.cuh"

namespace {

constexpr int kStages = 3;
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 256;
constexpr unsigned long long kTimeoutNs = 4000000000ull;  // 4 s per wait

// ---------------------------------------------------------------------------
// tile cull: work lists of (k | mask << 24), grouped by tile t = I * nb + j
// ---------------------------------------------------------------------------
constexpr int kWarps = 8;

__device__ __forceinline__ uint32_t tile_mask(const double *n2A, const double *n2BT, int64_t nb,
                                              int64_t P, int64_t I, int64_t j, int64_t k, double tau2)
{
    uint32_t m = 0;
    if (k < nb) {
        const double b = __ldg(n2BT + j * P + k);
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int64_t i = 4 * I + r;
            if (i < nb && keep_product(__ldg(n2A + i * P + k), b, tau2)) m |= 1u << r;
        }
    }
    return m;
}

__global__ void __launch_bounds__(kWarps * 32)
k_tile_count(const double *__restrict__ n2A, const double *__restrict__ n2BT, int64_t nb, int64_t P,
             int64_t nI, double tau2, int32_t *__restrict__ counts, int32_t *__restrict__ tasks)
{
    const int64_t t = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= nI * nb) return;
    const int64_t I = t / nb, j = t % nb;
    int cnt = 0, ntask = 0;
    for (int64_t k0 = 0; k0 < nb; k0 += 32) {
        const uint32_t m = tile_mask(n2A, n2BT, nb, P, I, j, k0 + lane, tau2);
        cnt += __popc(__ballot_sync(0xffffffffu, m != 0));
        ntask += __popc(m);
    }
    for (int o = 16; o > 0; o >>= 1) ntask += __shfl_xor_sync(0xffffffffu, ntask, o);
    if (lane == 0) {
        counts[t] = cnt;
        tasks[t] = ntask;
    }
}

__global__ void __launch_bounds__(kWarps * 32)
k_tile_emit(const double *__restrict__ n2A, const double *__restrict__ n2BT, int64_t nb, int64_t P,
            int64_t nI, double tau2, const int64_t *__restrict__ off, uint32_t *__restrict__ list,
            int64_t cap, int32_t *__restrict__ err)
{
    const int64_t t = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= nI * nb) return;
    if (off[t + 1] > cap) {
        if (lane == 0) atomicExch(err, 1);
        return;
    }
    const int64_t I = t / nb, j = t % nb;
    int64_t base = off[t];
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t k0 = 0; k0 < nb; k0 += 32) {
        const int64_t k = k0 + lane;
        const uint32_t m = tile_mask(n2A, n2BT, nb, P, I, j, k, tau2);
        const unsigned bal = __ballot_sync(0xffffffffu, m != 0);
        if (m) list[base + __popc(bal & lt)] = (uint32_t)k | (m << 24);
        base += __popc(bal);
    }
}

constexpr int kScanThreads = 1024;

// exclusive scan of counts -> off (one block), plus the total of `tasks`
__global__ void __launch_bounds__(kScanThreads)
k_tile_scan(const int32_t *__restrict__ counts, const int32_t *__restrict__ tasks, int64_t G,
            int64_t *__restrict__ off, int64_t *__restrict__ task_total)
{
    __shared__ int64_t part[kScanThreads];
    __shared__ int64_t tpart[kScanThreads];
    const int t = threadIdx.x;
    const int64_t chunk = (G + kScanThreads - 1) / kScanThreads;
    const int64_t lo = t * chunk, hi = lo + chunk < G ? lo + chunk : G;
    int64_t s = 0, ts = 0;
    for (int64_t q = lo; q < hi; q++) {
        s += counts[q];
        ts += tasks[q];
    }
    part[t] = s;
    tpart[t] = ts;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        const int64_t v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    for (int o = kScanThreads / 2; o > 0; o >>= 1) {
        if (t < o) tpart[t] += tpart[t + o];
        __syncthreads();
    }
    int64_t run = part[t] - s;
    for (int64_t q = lo; q < hi; q++) {
        off[q] = run;
        run += counts[q];
    }
    if (t == kScanThreads - 1) off[G] = part[t];
    if (t == 0) *task_total = tpart[0];
}

// Heaviest-first tile order (counting sort on the work-list length):
// hist -> descending exclusive scan -> scatter.
__global__ void k_tile_hist(const int32_t *__restrict__ counts, int64_t G, int32_t *__restrict__ bins)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < G) atomicAdd(bins + counts[t], 1);
}

__global__ void k_tile_bins_scan(int32_t *__restrict__ bins, int64_t nbins)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int32_t run = 0;
        for (int64_t c = nbins - 1; c >= 0; c--) {
            const int32_t v = bins[c];
            bins[c] = run;
            run += v;
        }
    }
}

__global__ void k_tile_scatter(const int32_t *__restrict__ counts, int64_t G, int32_t *__restrict__ bins,
                               int32_t *__restrict__ order)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < G) order[atomicAdd(bins + counts[t], 1)] = (int32_t)t;
}

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after kTimeoutNs (or when another role already failed).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (uint32_t it = 1;; it++) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 1023) == 0) {
            if (*abort_flag) return false;
            if (globaltimer() - t0 > kTimeoutNs) return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// tcgen05 shared-memory descriptor: no swizzle, K-major core matrices.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both K-major.
__device__ __forceinline__ uint32_t mma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred pa;\n setp.ne.b32 pa, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}\n" ::"r"(
            dtmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// RN(v * 2^k) for a signed 64-bit integer v, by integer operations only.
__device__ __forceinline__ double i64_scaled(long long v, int k)
{
    if (v == 0) return 0.0;
    const uint64_t sign = v < 0 ? (1ull << 63) : 0ull;
    uint64_t u = v < 0 ? (uint64_t)(-v) : (uint64_t)v;
    const int msb = 63 - __clzll((long long)u);
    uint64_t mant;
    if (msb <= 52) {
        mant = u << (52 - msb);
    } else {
        const int sh = msb - 52;
        mant = u >> sh;
        const uint64_t rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (mant & 1))) mant++;
        if (mant == (1ull << 53)) {
            mant >>= 1;
            k++;
        }
    }
    const int be = msb + k + 1023;
    if (be >= 1 && be <= 2046)
        return __longlong_as_double((long long)(sign | ((uint64_t)be << 52) | (mant & 0xFFFFFFFFFFFFFull)));
    const double r = ldexp((double)(mant >> 0), msb - 52 + k);  // rare: subnormal / overflow
    return sign ? -r : r;
}

struct TcArgs {
    const uint16_t *slA;   // A-role slices, per slot s*1024 BF16
    const uint16_t *slB;   // B-role slices
    const int32_t *slotA;  // nb*nb
    const int32_t *slotB;
    const uint16_t *zero;  // s*1024 BF16 zeros
    double *leafC;
    const int32_t *slotC;
    const int64_t *off;    // tile work-list offsets (nI*nb + 1)
    const uint32_t *list;  // k | mask << 24
    const int32_t *order;  // heaviest-first tile order
    const int32_t *sigA;   // sigma of A
    const int32_t *sigB;
    double *tr_part;       // diagonal-leaf traces (may be null)
    int32_t *err;          // error word (timeout)
    int64_t nb;
    int64_t nI;
};

template <int S>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(TcArgs g)
{
    constexpr uint32_t kLeafBytes = S * 2048;          // one leaf, all slices
    constexpr uint32_t kStageA = 4 * kLeafBytes;
    constexpr uint32_t kStageBytes = 5 * kLeafBytes;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages];
    __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2], done_bar;
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t T = g.nI * g.nb;

    if (threadIdx.x == 0) {
        for (int q = 0; q < kStages; q++) {
            mbar_init(smem_u32(&full_bar[q]), 1);
            mbar_init(smem_u32(&empty_bar[q]), 1);
        }
        for (int q = 0; q < 2; q++) {
            mbar_init(smem_u32(&accf_bar[q]), 1);
            mbar_init(smem_u32(&acce_bar[q]), 4);
        }
        mbar_init(smem_u32(&done_bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder;
    const uint32_t sbase = smem_u32(smem);
    volatile int *abort_v = &abort_flag;

    if (warp == 0) {
        // ------------------------------ producer ------------------------------
        if (lane == 0) {
            uint32_t st = 0, ph = 0;
            bool ok = true;
            for (int64_t it = blockIdx.x; it < T && ok; it += gridDim.x) {
                const int64_t t = g.order[it];
                const int64_t I = t / g.nb, j = t % g.nb;
                for (int64_t e = g.off[t]; e < g.off[t + 1]; e++) {
                    if (!mbar_wait(smem_u32(&empty_bar[st]), ph ^ 1, abort_v)) {
                        ok = false;
                        break;
                    }
                    const uint32_t w = g.list[e];
                    const int64_t k = w & 0xFFFFFF;
                    const uint32_t mask = w >> 24;
                    const uint32_t fb = smem_u32(&full_bar[st]);
                    const uint32_t dst = sbase + st * kStageBytes;
                    mbar_expect_tx(fb, kStageBytes);
#pragma unroll
                    for (int L = 0; L < 4; L++) {
                        const uint16_t *src = g.zero;
                        if (mask & (1u << L))
                            src = g.slA + (int64_t)g.slotA[(4 * I + L) * g.nb + k] * (S * 1024);
                        bulk_g2s(dst + L * kLeafBytes, src, kLeafBytes, fb);
                    }
                    bulk_g2s(dst + kStageA, g.slB + (int64_t)g.slotB[k * g.nb + j] * (S * 1024), kLeafBytes,
                             fb);
                    if (++st == kStages) {
                        st = 0;
                        ph ^= 1;
                    }
                }
            }
            if (!ok) {
                atomicExch(g.err, 1);
                abort_flag = 1;
            }
            // drain: every issued stage is consumed (and so landed) before exit
            for (uint32_t q = 0; q < kStages; q++) {
                mbar_wait(smem_u32(&empty_bar[st]), ph ^ 1, abort_v);
                if (++st == kStages) {
                    st = 0;
                    ph ^= 1;
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------ MMA issuer ------------------------------
        if (lane == 0) {
            uint32_t st = 0, ph = 0, acc = 0, aph = 0;
            bool ok = true;
            for (int64_t it = blockIdx.x; it < T && ok; it += gridDim.x) {
                const int64_t t = g.order[it];
                if (!mbar_wait(smem_u32(&acce_bar[acc]), aph ^ 1, abort_v)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dacc = tmem + acc * kAccStride;
                bool first = true;
                for (int64_t e = g.off[t]; e < g.off[t + 1]; e++) {
                    if (!mbar_wait(smem_u32(&full_bar[st]), ph, abort_v)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = sbase + st * kStageBytes;
                    const uint32_t sb = sa + kStageA;
#pragma unroll
                    for (int p = 0; p < S; p++) {
                        const uint32_t idesc = mma_idesc(128, 32 * (S - p));
#pragma unroll
                        for (int h = 0; h < 2; h++) {
                            const uint64_t da = smem_desc(sa + p * 512 + h * 256, 128, S * 512);
                            const uint64_t db = smem_desc(sb + h * 256, 128, 512);
                            const uint32_t accum = (first && p == 0 && h == 0) ? 0u : 1u;
                            mma_bf16(dacc + 32 * p, da, db, idesc, accum);
                        }
                    }
                    first = false;
                    mma_commit(smem_u32(&empty_bar[st]));
                    if (++st == kStages) {
                        st = 0;
                        ph ^= 1;
                    }
                }
                mma_commit(smem_u32(&accf_bar[acc]));
                if (++acc == 2) {
                    acc = 0;
                    aph ^= 1;
                }
            }
            if (!ok) {
                atomicExch(g.err, 1);
                abort_flag = 1;
            }
            // all MMAs issued by this thread complete before TMEM is freed
            mma_commit(smem_u32(&done_bar));
            mbar_wait(smem_u32(&done_bar), 0, abort_v);
        }
        __syncwarp();
    } else {
        // ------------------------------ epilogue ------------------------------
        const int quad = warp & 3;             // TMEM lane quadrant of this warp
        const int row = quad * 32 + lane;      // tile row 0..127
        const int L = row >> 5, r = row & 31;  // leaf within tile, row within leaf
        uint32_t acc = 0, aph = 0;
        for (int64_t it = blockIdx.x; it < T; it += gridDim.x) {
            const int64_t t = g.order[it];
            const int64_t I = t / g.nb, j = t % g.nb;
            const bool has_work = g.off[t + 1] > g.off[t];
            if (!mbar_wait(smem_u32(&accf_bar[acc]), aph, abort_v)) {
                if (lane == 0) atomicExch(g.err, 1);
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            long long cint[32];
#pragma unroll
            for (int c = 0; c < 32; c++) cint[c] = 0;
            if (has_work) {
                const uint32_t tbase = tmem + acc * kAccStride + ((uint32_t)(quad * 32) << 16);
#pragma unroll
                for (int d = 0; d < S; d++) {
                    uint32_t v[32];
                    tmem_ld32(tbase + 32 * d, v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int c = 0; c < 32; c++) {
                        const long long sd = (long long)__float2ll_rn(__uint_as_float(v[c]));
                        cint[c] += sd * (1ll << (7 * (S - 1 - d)));
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acce_bar[acc]));
            if (++acc == 2) {
                acc = 0;
                aph ^= 1;
            }
            const int64_t i = 4 * I + L;
            if (i < g.nb) {
                const int k = *g.sigA + *g.sigB - 7 * S - 7;
                double *dst = g.leafC + (int64_t)g.slotC[i * g.nb + j] * 1024 + r * 32;
                double diag = 0.0;
#pragma unroll
                for (int c = 0; c < 32; c += 2) {
                    double2 v;
                    v.x = i64_scaled(cint[c], k);
                    v.y = i64_scaled(cint[c + 1], k);
                    if (c == (r & ~1)) diag = (r & 1) ? v.y : v.x;
                    reinterpret_cast<double2 *>(dst)[c >> 1] = v;
                }
                if (g.tr_part && i == j) {
                    // fixed butterfly over the 32 rows of the diagonal leaf
                    for (int o = 16; o > 0; o >>= 1) diag += __shfl_xor_sync(0xffffffffu, diag, o);
                    if (lane == 0) g.tr_part[i] = diag;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
}

template <int S>
int launch_tc_s(const TcArgs &a, cudaStream_t s)
{
    const size_t smem = (size_t)kStages * 5 * S * 2048;
    static int configured = 0;
    if (!configured) {
        SPAMM_CK(cudaFuncSetAttribute(k_gemm_tc<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = 1;
    }
    const int64_t T = a.nI * a.nb;
    int64_t grid = spamm_num_sms();
    if (grid > T) grid = T;
    if (grid < 1) grid = 1;
    k_gemm_tc<S><<<(unsigned)grid, kThreads, smem, s>>>(a);
    SPAMM_CK_LAUNCH();
    return SPAMM_OK;
}

}  // namespace

int tc_slices_ok(int s) { return s >= 3 && s <= 7 && (size_t)kStages * 5 * s * 2048 <= 227 * 1024; }

// Tile cull for the tensor-core path into ws (tile lists + heaviest-first
// order); *tasks_dev receives the number of surviving triples.
static int tile_cull(spamm_mat_t A, spamm_mat_t B, double tau, SpammWorkspace *ws, cudaStream_t s)
{
    const int64_t nb = A->nb, P = A->P, nI = (nb + 3) / 4, T = nI * nb;
    int rc;
    if (ws->tile_cap < T) {
        spamm_release(ws->tcounts, s);
        spamm_release(ws->ttasks, s);
        spamm_release(ws->toff, s);
        spamm_release(ws->torder, s);
        spamm_release(ws->tbins, s);
        ws->tcounts = ws->ttasks = ws->torder = ws->tbins = nullptr;
        ws->toff = nullptr;
        ws->tile_cap = 0;
        if ((rc = spamm_alloc((void **)&ws->tcounts, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->ttasks, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->toff, sizeof(int64_t) * (T + 2), s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->torder, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->tbins, sizeof(int32_t) * (nb + 1), s))) return rc;
        ws->tile_cap = T;
    }
    const double tau2 = tau * tau;
    const unsigned blocks = (unsigned)((T + kWarps - 1) / kWarps);
    k_tile_count<<<blocks, kWarps * 32, 0, s>>>(A->n2 + tier_offset(A->depth), B->n2T, nb, P, nI, tau2,
                                                 ws->tcounts, ws->ttasks);
    SPAMM_CK_LAUNCH();
    k_tile_scan<<<1, kScanThreads, 0, s>>>(ws->tcounts, ws->ttasks, T, ws->toff, ws->toff + T + 1);
    SPAMM_CK_LAUNCH();
    const int64_t worst = T * nb;
    if (ws->tlist_cap < worst) {
        spamm_release(ws->tlist, s);
        ws->tlist = nullptr;
        ws->tlist_cap = 0;
        if ((rc = spamm_alloc((void **)&ws->tlist, sizeof(uint32_t) * worst, s))) return rc;
        ws->tlist_cap = worst;
    }
    k_tile_emit<<<blocks, kWarps * 32, 0, s>>>(A->n2 + tier_offset(A->depth), B->n2T, nb, P, nI, tau2,
                                                ws->toff, ws->tlist, ws->tlist_cap, ws->counter + 8);
    SPAMM_CK_LAUNCH();
    SPAMM_CK(cudaMemsetAsync(ws->tbins, 0, sizeof(int32_t) * (nb + 1), s));
    k_tile_hist<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(ws->tcounts, T, ws->tbins);
    SPAMM_CK_LAUNCH();
    k_tile_bins_scan<<<1, 32, 0, s>>>(ws->tbins, nb + 1);
    SPAMM_CK_LAUNCH();
    k_tile_scatter<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(ws->tcounts, T, ws->tbins, ws->torder);
    SPAMM_CK_LAUNCH();
    return SPAMM_OK;
}

int launch_gemm_tc(spamm_mat_t A, spamm_mat_t B, spamm_mat_t C, SpammWorkspace *ws, double tau,
                   double *tr_part, int slices, cudaStream_t s)
{
    if (A->b != 32 || !tc_slices_ok(slices)) {
        spamm_set_error("tensor-core path: leaf must be 32 and slices in 3..7 (leaf %d, slices %d)", A->b,
                        slices);
        return SPAMM_E_NOTSUP;
    }
    int rc = tile_cull(A, B, tau, ws, s);
    if (rc) return rc;
    if (!ws->zero || ws->zero_bytes < (size_t)slices * 2048) {
        spamm_release(ws->zero, s);
        ws->zero = nullptr;
        if ((rc = spamm_alloc((void **)&ws->zero, (size_t)slices * 2048, s))) return rc;
        ws->zero_bytes = (size_t)slices * 2048;
        SPAMM_CK(cudaMemsetAsync(ws->zero, 0, ws->zero_bytes, s));
    }
    TcArgs a;
    a.slA = A->slA;
    a.slB = B->slB;
    a.slotA = A->slot;
    a.slotB = B->slot;
    a.zero = ws->zero;
    a.leafC = C->leaf;
    a.slotC = C->slot;
    a.off = ws->toff;
    a.list = ws->tlist;
    a.order = ws->torder;
    a.sigA = reinterpret_cast<const int32_t *>(A->scale + 1);
    a.sigB = reinterpret_cast<const int32_t *>(B->scale + 1);
    a.tr_part = tr_part;
    a.err = ws->counter + 9;
    a.nb = A->nb;
    a.nI = (A->nb + 3) / 4;
    switch (slices) {
    case 3: return launch_tc_s<3>(a, s);
    case 4: return launch_tc_s<4>(a, s);
    case 5: return launch_tc_s<5>(a, s);
    case 6: return launch_tc_s<6>(a, s);
    case 7: return launch_tc_s<7>(a, s);
    default: return SPAMM_E_NOTSUP;
    }
}
