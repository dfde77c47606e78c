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
// multiplies the 128 x 32 A slab by B slices q = zB..s-1-p (N = 32 (s-p-zB))
// and accumulates into TMEM columns [32 (p + zB), 32 s): column block d then
// holds the exact integer S_d = sum_{p+q=d} sum_k sum_l dA_p dB_q.  Pairs
// with p + q >= s are never formed, nor pairs with p < zA or q < zB, where zA
// (the least over the item's kept A leaves) and zB count leading slices that
// are zero in every element: those products are exactly zero.  An item whose
// kept leaves all have zA + zB >= s contributes exactly nothing and is not
// listed.  The epilogue forms
//     C = 2^(sigmaA + sigmaB - 7s - 7) * sum_d S_d 128^(s-1-d)
// with integer arithmetic and one rounding to FP64, then zeroes the
// accumulator for the next tile.
//
// Kernel roles (192 threads, one CTA per SM, persistent):
//   warp 0     : producer; two bulk copies (cp.async.bulk) per work item:
//                the needed slices of the four A leaves (one contiguous block
//                of the tile-major array, stage layout [p][leaf][2 KB]) and of
//                the B leaf, into a 3-stage ring, completion on the stage's
//                mbarrier;
//   warp 1     : allocates 512 TMEM columns; once a stage lands, the warp
//                zeroes the leaves of culled triples in it, then lane 0 issues
//                the tcgen05.mma of the item and commits to the stage's
//                "empty" barrier and, at the end of a tile, to the
//                accumulator's "full" barrier;
//   warps 2-5  : epilogue; tcgen05.ld of the s diagonal blocks of the row the
//                thread owns, integer combine, FP64 store, diagonal traces.
// Two accumulators (TMEM columns 0 and 256) let the epilogue of one tile run
// under the MMAs of the next.  Every wait is bounded (SM cycle counter); on
// timeout the kernel records the error, drains and frees TMEM, and returns.
//
// Roofline: tensor pipe.  Useful work 2 b^3 per surviving triple; issued
// tensor work 2 * 128 * 32 * 32 * s(s+1)/2 per work item.
#include "internal.cuh"

namespace {

// Shared-memory byte ring for work items: an item needing m slices per
// operand takes exactly m * 10 KB (A: m x 8 KB, B: m x 2 KB), so small items
// (many leading zero slices) leave room for more items in flight.
constexpr uint32_t kRingBytes = 216 * 1024;
constexpr int kSlots = 16;  // work items in flight at most
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 256;
constexpr long long kTimeoutCycles = 8000000000ll;  // about 4 s at 2 GHz per wait
// Tile order: true = heaviest first (tiles are handed out dynamically, so
// this is longest-processing-time-first scheduling); false = row-major.
constexpr bool kHeaviestFirst = true;
constexpr int kTileRing = 4;  // tiles handed from the producer to the other roles

// ---------------------------------------------------------------------------
// tile cull: work lists of (k | mask << 24), grouped by tile t = I * nb + j
// ---------------------------------------------------------------------------
constexpr int kWarps = 8;

struct CullArgs {
    const double *n2A, *n2BT;
    const uint8_t *zA, *zB;        // leading zero slices per slot
    const int32_t *slotA, *slotB;  // slot maps (B: of the matrix whose slices serve as B)
    int64_t nb, P, nI;
    double tau2;
    int sym, S;
    const int32_t *stop;  // set once an SP2 loop has stopped: nothing to do
};

// Work item of tile (I, j) at k: k | mask << 15 | zA << 19 | zB << 22, or 0
// when no kept leaf has a nonzero product.  *ntask += surviving triples;
// *npair += slice pairs those triples need (p >= zA_i, q >= zB, p + q < S).
__device__ __forceinline__ uint32_t tile_item(const CullArgs &c, int64_t I, int64_t j, int64_t k, int &ntask,
                                              int &npair)
{
    if (k >= c.nb) return 0;
    const double b = __ldg(c.n2BT + j * c.P + k);
    // B operand leaf (k, j); in symmetric mode its image is leaf (j, k)'s A role
    const int zb = c.sym ? c.zA[c.slotA[j * c.nb + k]] : c.zB[c.slotB[k * c.nb + j]];
    uint32_t mask = 0;
    int za = c.S;
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int64_t i = 4 * I + r;
        if (i < c.nb && keep_product(__ldg(c.n2A + i * c.P + k), b, c.tau2)) {
            ntask++;
            const int zr = c.zA[c.slotA[i * c.nb + k]];
            if (zr + zb < c.S) {
                const int mr = c.S - zr - zb;
                npair += mr * (mr + 1) / 2;
                mask |= 1u << r;
                za = zr < za ? zr : za;
            }
        }
    }
    if (!mask) return 0;
    return (uint32_t)k | (mask << 15) | ((uint32_t)za << 19) | ((uint32_t)zb << 22);
}

__device__ __forceinline__ int item_pairs(uint32_t w, int S)
{
    const int m = S - (int)((w >> 19) & 7) - (int)((w >> 22) & 7);
    return m * (m + 1) / 2;
}

__global__ void __launch_bounds__(kWarps * 32)
k_tile_count(CullArgs c, int32_t *__restrict__ counts, int32_t *__restrict__ tasks,
             int32_t *__restrict__ pairs, int32_t *__restrict__ useful)
{
    if (c.stop && *c.stop) return;
    const int64_t t = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= c.nI * c.nb) return;
    const int64_t I = t / c.nb, j = t % c.nb;
    const bool active = !c.sym || j >= 4 * I;
    int cnt = 0, ntask = 0, npair = 0, nuse = 0;
    for (int64_t k0 = 0; k0 < c.nb; k0 += 32) {
        const uint32_t w = tile_item(c, I, j, k0 + lane, ntask, nuse);
        cnt += __popc(__ballot_sync(0xffffffffu, w != 0));
        if (w) npair += item_pairs(w, c.S);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ntask += __shfl_xor_sync(0xffffffffu, ntask, o);
        npair += __shfl_xor_sync(0xffffffffu, npair, o);
        nuse += __shfl_xor_sync(0xffffffffu, nuse, o);
    }
    if (lane == 0) {
        counts[t] = active ? cnt : 0;
        tasks[t] = ntask;
        pairs[t] = active ? npair : 0;
        useful[t] = active ? nuse : 0;
    }
}

__global__ void __launch_bounds__(kWarps * 32)
k_tile_emit(CullArgs c, const int64_t *__restrict__ off, uint32_t *__restrict__ list, int64_t cap,
            int32_t *__restrict__ err)
{
    if (c.stop && *c.stop) return;
    const int64_t t = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= c.nI * c.nb) return;
    const int64_t I = t / c.nb, j = t % c.nb;
    if (c.sym && j < 4 * I) return;
    if (off[t + 1] > cap) {
        if (lane == 0) atomicExch(err, 1);
        return;
    }
    int64_t base = off[t];
    const unsigned lt = (1u << lane) - 1u;
    int dummy = 0, dummy2 = 0;
    for (int64_t k0 = 0; k0 < c.nb; k0 += 32) {
        const uint32_t w = tile_item(c, I, j, k0 + lane, dummy, dummy2);
        const unsigned bal = __ballot_sync(0xffffffffu, w != 0);
        if (w) list[base + __popc(bal & lt)] = w;
        base += __popc(bal);
    }
}

constexpr int kScanThreads = 1024;

// exclusive scan of counts -> off (one block), plus the total of `tasks`
__global__ void __launch_bounds__(kScanThreads)
k_tile_scan(const int32_t *__restrict__ stop, const int32_t *__restrict__ counts, const int32_t *__restrict__ tasks,
            const int32_t *__restrict__ pairs, const int32_t *__restrict__ useful, int64_t G,
            int64_t *__restrict__ off, int64_t *__restrict__ task_total, int64_t *__restrict__ pair_total,
            int64_t *__restrict__ useful_total)
{
    __shared__ int64_t part[kScanThreads];
    __shared__ int64_t tpart[kScanThreads];
    __shared__ int64_t ppart[kScanThreads];
    __shared__ int64_t upart[kScanThreads];
    if (stop && *stop) return;  // the SP2 loop has already stopped
    const int t = threadIdx.x;
    const int64_t chunk = (G + kScanThreads - 1) / kScanThreads;
    const int64_t lo = t * chunk, hi = lo + chunk < G ? lo + chunk : G;
    int64_t s = 0, ts = 0, ps = 0, us = 0;
    for (int64_t q = lo; q < hi; q++) {
        s += counts[q];
        ts += tasks[q];
        ps += pairs[q];
        us += useful[q];
    }
    part[t] = s;
    tpart[t] = ts;
    ppart[t] = ps;
    upart[t] = us;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        const int64_t v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    for (int o = kScanThreads / 2; o > 0; o >>= 1) {
        if (t < o) {
            tpart[t] += tpart[t + o];
            ppart[t] += ppart[t + o];
            upart[t] += upart[t + o];
        }
        __syncthreads();
    }
    int64_t run = part[t] - s;
    for (int64_t q = lo; q < hi; q++) {
        off[q] = run;
        run += counts[q];
    }
    if (t == kScanThreads - 1) off[G] = part[t];
    if (t == 0) {
        *task_total = tpart[0];
        *pair_total = ppart[0];
        *useful_total = upart[0];
    }
}

// Heaviest-first tile order (counting sort on the work-list length):
// hist -> descending exclusive scan -> scatter.
__global__ void k_tile_hist(const int32_t *__restrict__ stop, const int32_t *__restrict__ counts, int64_t nb,
                            int64_t G, int sym, int32_t *__restrict__ bins)
{
    if (stop && *stop) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < G && !(sym && t % nb < 4 * (t / nb))) atomicAdd(bins + counts[t], 1);
}

__global__ void k_tile_bins_scan(const int32_t *__restrict__ stop, int32_t *__restrict__ bins, int64_t nbins)
{
    if (stop && *stop) return;
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int32_t run = 0;
        for (int64_t c = nbins - 1; c >= 0; c--) {
            const int32_t v = bins[c];
            bins[c] = run;
            run += v;
        }
    }
}

// Row-major order of the active tiles: all tiles, or in symmetric mode the
// tiles with j >= 4I (row I holds nb - 4I of them).
__global__ void k_tile_natural(int64_t nb, int64_t nI, int sym, int32_t *__restrict__ order)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nI * nb) return;
    const int64_t I = t / nb, j = t % nb;
    if (!sym) {
        order[t] = (int32_t)t;
    } else if (j >= 4 * I) {
        order[I * nb - 2 * I * (I - 1) + (j - 4 * I)] = (int32_t)t;
    }
}

__global__ void k_tile_scatter(const int32_t *__restrict__ stop, const int32_t *__restrict__ counts, int64_t nb,
                               int64_t G, int sym, int32_t *__restrict__ bins, int32_t *__restrict__ order)
{
    if (stop && *stop) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < G && !(sym && t % nb < 4 * (t / nb))) order[atomicAdd(bins + counts[t], 1)] = (int32_t)t;
}

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

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

// Bounded wait: false after about kTimeoutCycles SM cycles (or as soon as
// another role has failed).  The SM cycle counter is read, not the global
// timer, which is far slower to read and would sit on every handoff.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t it = 1;; it++) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255) == 0) {
            if (*abort_flag) return false;
            if (clock64() - t0 > kTimeoutCycles) return false;
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
    const uint16_t *slA;   // A operand: tile-major [I][k][p][L][1024] BF16
    const uint16_t *slB;   // B operand: per slot [q][1024] (symmetric: A-role of the transpose)
    const int32_t *slotA;  // nb*nb
    const int32_t *slotB;
    double *leafC;
    const int32_t *slotC;
    const int64_t *off;    // tile work-list offsets
    const uint32_t *list;  // k | mask << 15 | zA << 19 | zB << 22
    const int32_t *order;  // tile order
    const int32_t *sigA;   // sigma of A
    const int32_t *sigB;
    double *tr_part;       // diagonal-leaf traces (may be null)
    int32_t *err;          // error word (timeout)
    int32_t *next_tile;    // dynamic scheduler: next position in `order` (zeroed per launch)
    int64_t nb;
    int64_t nI;
    int64_t T;             // tiles in the order list
    int sym;               // symmetric product: upper block triangle + mirror
    const int32_t *stop;   // set once an SP2 loop has stopped: nothing to do
    int float_split;       // slices are a float split: C = sum_d S_d in FP64, no scaling
};

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_zero16(uint32_t taddr)
{
    const uint32_t z = 0;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(z)
        : "memory");
}

template <int S>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(TcArgs g)
{
    constexpr uint32_t kSlice = 2048;  // one slice of one leaf
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full_bar[kSlots], empty_bar[kSlots];
    __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2], done_bar;
    __shared__ uint32_t slot_off[kSlots];  // ring byte offset of each in-flight item
    __shared__ uint32_t slot_w[kSlots];    // its work-list entry
    __shared__ int32_t tile_q[kTileRing];  // tiles handed out, -1 = no more
    __shared__ __align__(8) uint64_t tfull_bar[kTileRing], tempty_bar[kTileRing];
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;

    if (g.stop && *g.stop) return;  // before any barrier or TMEM is touched
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t T = g.T;

    if (threadIdx.x == 0) {
        for (int q = 0; q < kSlots; q++) {
            mbar_init(smem_u32(&full_bar[q]), 1);
            mbar_init(smem_u32(&empty_bar[q]), 1);
        }
        for (int q = 0; q < 2; q++) {
            mbar_init(smem_u32(&accf_bar[q]), 1);
            mbar_init(smem_u32(&acce_bar[q]), 4);
        }
        mbar_init(smem_u32(&done_bar), 1);
        for (int q = 0; q < kTileRing; q++) {
            mbar_init(smem_u32(&tfull_bar[q]), 1);
            mbar_init(smem_u32(&tempty_bar[q]), 5);  // MMA warp + four epilogue warps
        }
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
        // The warp loads 32 work entries (and their B slots) at a time; lane 0
        // then allocates ring space and issues the copies item by item.
        // cumulative byte pointers (allocation incl. wrap padding, release)
        unsigned long long alloc_ptr = 0, free_ptr = 0;
        unsigned long long end_ptr[kSlots];
        uint32_t issued = 0, released = 0;
        bool ok = true;
        uint32_t tq = 0, tph = 0;
        for (;;) {
            // take the next tile and hand it to the MMA and epilogue warps
            int32_t tt = -1;
            int tgood = 1;
            if (lane == 0) {
                if (!mbar_wait(smem_u32(&tempty_bar[tq]), tph ^ 1, abort_v)) {
                    tgood = 0;
                } else {
                    const int32_t pos = atomicAdd(g.next_tile, 1);
                    tt = pos < T ? g.order[pos] : -1;
                    tile_q[tq] = tt;
                    mbar_arrive(smem_u32(&tfull_bar[tq]));
                }
            }
            tt = __shfl_sync(0xffffffffu, tt, 0);
            if (!__shfl_sync(0xffffffffu, tgood, 0)) {
                ok = false;
                break;
            }
            if (++tq == kTileRing) {
                tq = 0;
                tph ^= 1;
            }
            if (tt < 0) break;
            const int64_t t = tt;
            const int64_t I = t / g.nb, j = t % g.nb;
            const int64_t e0 = g.off[t], e1 = g.off[t + 1];
            for (int64_t base = e0; base < e1 && ok; base += 32) {
                const int cnt = (int)(e1 - base < 32 ? e1 - base : 32);
                uint32_t wl = 0;
                int64_t bl = 0;
                if (lane < cnt) {
                    wl = g.list[base + lane];
                    const int64_t kk = wl & 0x7FFF;
                    bl = g.sym ? g.slotA[j * g.nb + kk] : g.slotB[kk * g.nb + j];
                }
                for (int q = 0; q < cnt; q++) {
                    const uint32_t w = __shfl_sync(0xffffffffu, wl, q);
                    const int64_t bslot = __shfl_sync(0xffffffffu, bl, q);
                    int good = 1;
                    if (lane == 0) {
                        const int64_t k = w & 0x7FFF;
                        const int za = (w >> 19) & 7, zb = (w >> 22) & 7;
                        const int m = S - za - zb;  // slices needed from each operand
                        const uint32_t need = (uint32_t)m * 5 * kSlice;
                        uint32_t pos = (uint32_t)(alloc_ptr % kRingBytes);
                        if (pos + need > kRingBytes) {
                            alloc_ptr += kRingBytes - pos;
                            pos = 0;
                        }
                        const unsigned long long new_end = alloc_ptr + need;
                        // wait (in order) for released items until the region and a slot are free
                        while (new_end - free_ptr > kRingBytes || issued - released >= (uint32_t)kSlots) {
                            const uint32_t rs = released % kSlots;
                            if (!mbar_wait(smem_u32(&empty_bar[rs]), (released / kSlots) & 1, abort_v)) {
                                good = 0;
                                break;
                            }
                            free_ptr = end_ptr[rs];
                            released++;
                        }
                        if (good) {
                            const uint32_t sl = issued % kSlots;
                            slot_off[sl] = pos;
                            slot_w[sl] = w;
                            end_ptr[sl] = new_end;
                            alloc_ptr = new_end;
                            const uint32_t fb = smem_u32(&full_bar[sl]);
                            const uint32_t dst = sbase + pos;
                            mbar_expect_tx(fb, need);
                            // A: slices za..za+m-1 of the four rows' leaves, one contiguous block
                            bulk_g2s(dst, g.slA + ((I * g.nb + k) * S + za) * 4096, (uint32_t)m * 4 * kSlice, fb);
                            // B: slices zb..zb+m-1 of leaf (k, j) (symmetric: leaf (j, k))
                            bulk_g2s(dst + (uint32_t)m * 4 * kSlice, g.slB + bslot * (S * 1024) + zb * 1024,
                                     (uint32_t)m * kSlice, fb);
                            issued++;
                        }
                    }
                    if (!__shfl_sync(0xffffffffu, good, 0)) {
                        ok = false;
                        break;
                    }
                }
            }
        }
        if (lane == 0) {
            if (!ok) {
                atomicExch(g.err, 1);
                abort_flag = 1;
            }
            // drain: every issued item is consumed (and so landed) before exit
            while (released < issued) {
                if (!mbar_wait(smem_u32(&empty_bar[released % kSlots]), (released / kSlots) & 1, abort_v)) break;
                released++;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------ MMA issuer ------------------------------
        // Lane 0 issues; the whole warp zeroes the leaves of culled triples in
        // a landed stage before the MMAs read it.
        uint32_t consumed = 0, acc = 0, aph = 0;
        bool ok = true;
        uint32_t tq = 0, tph = 0;
        for (;;) {
            int32_t tt = -1;
            int tgood = 1;
            if (lane == 0) {
                tgood = mbar_wait(smem_u32(&tfull_bar[tq]), tph, abort_v);
                if (tgood) {
                    tt = tile_q[tq];
                    mbar_arrive(smem_u32(&tempty_bar[tq]));
                }
            }
            tt = __shfl_sync(0xffffffffu, tt, 0);
            if (!__shfl_sync(0xffffffffu, tgood, 0)) {
                ok = false;
                break;
            }
            if (++tq == kTileRing) {
                tq = 0;
                tph ^= 1;
            }
            if (tt < 0) break;
            const int64_t t = tt;
            // the accumulator was zeroed by the epilogue (phase u of its barrier)
            int good = 1;
            if (lane == 0) good = mbar_wait(smem_u32(&acce_bar[acc]), aph, abort_v);
            if (!__shfl_sync(0xffffffffu, good, 0)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dacc = tmem + acc * kAccStride;
            for (int64_t e = g.off[t]; e < g.off[t + 1]; e++) {
                const uint32_t sl = consumed % kSlots;
                good = 1;
                if (lane == 0) good = mbar_wait(smem_u32(&full_bar[sl]), (consumed / kSlots) & 1, abort_v);
                if (!__shfl_sync(0xffffffffu, good, 0)) {
                    ok = false;
                    break;
                }
                // lane 0 observed the landed data (and the slot's metadata);
                // hand both to the other lanes
                __syncwarp();
                const uint32_t w = __shfl_sync(0xffffffffu, lane == 0 ? slot_w[sl] : 0u, 0);
                const uint32_t pos = __shfl_sync(0xffffffffu, lane == 0 ? slot_off[sl] : 0u, 0);
                const uint32_t mask = (w >> 15) & 15;
                const int za = (w >> 19) & 7, zb = (w >> 22) & 7;
                const int m = S - za - zb;
                if (mask != 15) {
                    const uint4 zero4 = make_uint4(0, 0, 0, 0);
                    for (int L = 0; L < 4; L++) {
                        if (mask & (1u << L)) continue;
                        for (int pp = 0; pp < m; pp++) {
                            uint4 *z = reinterpret_cast<uint4 *>(smem + pos + pp * (4 * kSlice) + L * kSlice);
#pragma unroll
                            for (int q = 0; q < 4; q++) z[q * 32 + lane] = zero4;
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                }
                __syncwarp();
                if (lane == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = sbase + pos;                        // A slice za
                    const uint32_t sb = sa + (uint32_t)m * 4 * kSlice;      // B slice zb
                    // descriptors advance by adding (bytes >> 4) to the address field
                    // (shared addresses stay below 256 KB, so the field never carries)
                    const uint64_t da0 = smem_desc(sa, 128, 512);
                    const uint64_t db0 = smem_desc(sb, 128, 512);
                    uint32_t idesc = mma_idesc(128, 32 * m);
                    uint32_t dcol = dacc + 32 * (za + zb);
                    for (int pp = 0; pp < m; pp++) {
                        const uint64_t da = da0 + (uint64_t)(pp * (4 * kSlice / 16));
                        mma_bf16(dcol, da, db0, idesc, 1u);
                        mma_bf16(dcol, da + 16, db0 + 16, idesc, 1u);  // second K half: +256 B
                        idesc -= 4u << 17;                              // N shrinks by 32
                        dcol += 32;
                    }
                    mma_commit(smem_u32(&empty_bar[sl]));
                }
                __syncwarp();
                consumed++;
            }
            if (lane == 0) mma_commit(smem_u32(&accf_bar[acc]));
            if (++acc == 2) {
                acc = 0;
                aph ^= 1;
            }
        }
        if (lane == 0) {
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
        const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
        // both accumulators start at zero (first phase of their "empty" barriers)
        for (int b = 0; b < 2; b++) {
            for (int d = 0; d < S; d++)
                for (int h = 0; h < 2; h++) tmem_zero16(tmem + b * kAccStride + lane_off + 32 * d + 16 * h);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(smem_u32(&acce_bar[0]));
            mbar_arrive(smem_u32(&acce_bar[1]));
        }
        uint32_t acc = 0, aph = 0;
        uint32_t tq = 0, tph = 0;
        for (;;) {
            int32_t tt = -1;
            int tgood = 1;
            if (lane == 0) {
                tgood = mbar_wait(smem_u32(&tfull_bar[tq]), tph, abort_v);
                if (tgood) {
                    tt = tile_q[tq];
                    mbar_arrive(smem_u32(&tempty_bar[tq]));
                }
            }
            tt = __shfl_sync(0xffffffffu, tt, 0);
            if (!__shfl_sync(0xffffffffu, tgood, 0)) {
                if (lane == 0) atomicExch(g.err, 1);
                abort_flag = 1;
                break;
            }
            if (++tq == kTileRing) {
                tq = 0;
                tph ^= 1;
            }
            if (tt < 0) break;
            const int64_t t = tt;
            const int64_t I = t / g.nb, j = t % g.nb;
            const bool has_work = g.off[t + 1] > g.off[t];
            if (!mbar_wait(smem_u32(&accf_bar[acc]), aph, abort_v)) {
                if (lane == 0) atomicExch(g.err, 1);
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int64_t i = 4 * I + L;
            // symmetric mode: leaf (i, j) is written only for i <= j, and for
            // i < j its transpose goes to leaf (j, i)
            const bool store = i < g.nb && (!g.sym || i <= j);
            const int kexp = *g.sigA + *g.sigB - 7 * S - 7;
            double *dst = store ? g.leafC + (int64_t)g.slotC[i * g.nb + j] * 1024 + r * 32 : nullptr;
            double *mir = (store && g.sym && i < j) ? g.leafC + (int64_t)g.slotC[j * g.nb + i] * 1024 + r : nullptr;
            double diag = 0.0;
            const uint32_t tbase = tmem + acc * kAccStride + lane_off;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                long long cint[16];   // exact slices: integer combination
                double cflt[16];      // float split: FP64 sum of the FP32 diagonals
#pragma unroll
                for (int c = 0; c < 16; c++) {
                    cint[c] = 0;
                    cflt[c] = 0.0;
                }
                if (has_work) {
#pragma unroll
                    for (int d = 0; d < S; d++) {
                        uint32_t v[16];
                        tmem_ld16(tbase + 32 * d + 16 * h, v);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        if (g.float_split) {
#pragma unroll
                            for (int c = 0; c < 16; c++) cflt[c] += (double)__uint_as_float(v[c]);
                        } else {
#pragma unroll
                            for (int c = 0; c < 16; c++)
                                cint[c] += (long long)__float2ll_rn(__uint_as_float(v[c])) * (1ll << (7 * (S - 1 - d)));
                        }
                        tmem_zero16(tbase + 32 * d + 16 * h);
                    }
                }
                if (store) {
#pragma unroll
                    for (int c = 0; c < 16; c += 2) {
                        const int col = 16 * h + c;
                        double2 v;
                        v.x = g.float_split ? cflt[c] : i64_scaled(cint[c], kexp);
                        v.y = g.float_split ? cflt[c + 1] : i64_scaled(cint[c + 1], kexp);
                        if (col == (r & ~1)) diag = (r & 1) ? v.y : v.x;
                        reinterpret_cast<double2 *>(dst)[col >> 1] = v;
                        if (mir) {
                            mir[col * 32] = v.x;
                            mir[(col + 1) * 32] = v.y;
                        }
                    }
                }
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acce_bar[acc]));
            if (++acc == 2) {
                acc = 0;
                aph ^= 1;
            }
            if (store && g.tr_part && i == j) {
                // fixed butterfly over the 32 rows of the diagonal leaf
                for (int o = 16; o > 0; o >>= 1) diag += __shfl_xor_sync(0xffffffffu, diag, o);
                if (lane == 0) g.tr_part[i] = diag;
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
    const size_t smem = kRingBytes;
    static int configured = 0;
    if (!configured) {
        SPAMM_CK(cudaFuncSetAttribute(k_gemm_tc<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = 1;
    }
    const int64_t T = a.T;
    int64_t grid = spamm_num_sms();
    if (grid > T) grid = T;
    if (grid < 1) grid = 1;
    k_gemm_tc<S><<<(unsigned)grid, kThreads, smem, s>>>(a);
    SPAMM_CK_LAUNCH();
    return SPAMM_OK;
}

}  // namespace

int tc_slices_ok(int s) { return s >= 3 && s <= 7 && (uint32_t)s * 5 * 2048 <= kRingBytes; }

// Tile cull for the tensor-core path into ws (tile lists + heaviest-first
// order); toff[T + 1] receives the number of surviving triples.
int tc_tile_cull(spamm_mat_t A, spamm_mat_t B, double tau, SpammWorkspace *ws, int sym, int slices,
                 cudaStream_t s)
{
    const int64_t nb = A->nb, P = A->P, nI = (nb + 3) / 4, T = nI * nb;
    int rc;
    if (ws->tile_cap < T) {
        spamm_release(ws->tcounts, s);
        spamm_release(ws->ttasks, s);
        spamm_release(ws->tpairs, s);
        spamm_release(ws->toff, s);
        spamm_release(ws->torder, s);
        spamm_release(ws->tbins, s);
        spamm_release(ws->tuseful, s);
        ws->tcounts = ws->ttasks = ws->tpairs = ws->tuseful = ws->torder = ws->tbins = nullptr;
        ws->toff = nullptr;
        ws->tile_cap = 0;
        if ((rc = spamm_alloc((void **)&ws->tcounts, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->ttasks, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->tpairs, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->tuseful, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->toff, sizeof(int64_t) * (T + 4), s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->torder, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->tbins, sizeof(int32_t) * (nb + 1), s))) return rc;
        ws->tile_cap = T;
    }
    CullArgs c;
    c.n2A = A->n2 + tier_offset(A->depth);
    c.n2BT = B->n2T;
    c.zA = A->zlead;
    c.zB = B->zlead;
    c.slotA = A->slot;
    c.slotB = B->slot;
    c.nb = nb;
    c.P = P;
    c.nI = nI;
    c.tau2 = tau * tau;
    c.sym = sym;
    c.S = slices;
    c.stop = ws->stop;
    const unsigned blocks = (unsigned)((T + kWarps - 1) / kWarps);
    k_tile_count<<<blocks, kWarps * 32, 0, s>>>(c, ws->tcounts, ws->ttasks, ws->tpairs, ws->tuseful);
    SPAMM_CK_LAUNCH();
    // toff[0..T] offsets, toff[T+1] surviving triples, toff[T+2] issued slice-pair
    // work, toff[T+3] slice pairs the surviving triples need
    k_tile_scan<<<1, kScanThreads, 0, s>>>(ws->stop, ws->tcounts, ws->ttasks, ws->tpairs, ws->tuseful, T,
                                           ws->toff, ws->toff + T + 1, ws->toff + T + 2, ws->toff + T + 3);
    SPAMM_CK_LAUNCH();
    const int64_t worst = T * nb;
    if (ws->tlist_cap < worst) {
        spamm_release(ws->tlist, s);
        ws->tlist = nullptr;
        ws->tlist_cap = 0;
        if ((rc = spamm_alloc((void **)&ws->tlist, sizeof(uint32_t) * worst, s))) return rc;
        ws->tlist_cap = worst;
    }
    k_tile_emit<<<blocks, kWarps * 32, 0, s>>>(c, ws->toff, ws->tlist, ws->tlist_cap, ws->counter + 8);
    SPAMM_CK_LAUNCH();
    ws->tsym = sym;
    ws->tactive = sym ? nI * nb - 2 * nI * (nI - 1) : T;
    if (kHeaviestFirst) {
        SPAMM_CK(cudaMemsetAsync(ws->tbins, 0, sizeof(int32_t) * (nb + 1), s));
        k_tile_hist<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(ws->stop, ws->tcounts, nb, T, sym, ws->tbins);
        SPAMM_CK_LAUNCH();
        k_tile_bins_scan<<<1, 32, 0, s>>>(ws->stop, ws->tbins, nb + 1);
        SPAMM_CK_LAUNCH();
        k_tile_scatter<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(ws->stop, ws->tcounts, nb, T, sym, ws->tbins,
                                                                     ws->torder);
        SPAMM_CK_LAUNCH();
    } else {
        k_tile_natural<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(nb, nI, sym, ws->torder);
        SPAMM_CK_LAUNCH();
    }
    return SPAMM_OK;
}

int launch_gemm_tc(spamm_mat_t A, spamm_mat_t B, spamm_mat_t C, SpammWorkspace *ws,
                   double *tr_part, int slices, cudaStream_t s, bool float_split)
{
    if (A->b != 32 || !(float_split ? (slices == 1 || slices == 2) : tc_slices_ok(slices) != 0)) {
        spamm_set_error("tensor-core path: leaf must be 32 and slices in 3..7 (leaf %d, slices %d)", A->b,
                        slices);
        return SPAMM_E_NOTSUP;
    }
    int rc;
    TcArgs a;
    a.slA = A->slA;
    a.slB = B->slB;  // per-leaf slices: B-role layout, or (symmetric) A-role of the transpose
    a.slotA = A->slot;
    a.slotB = B->slot;
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
    a.T = ws->tactive;
    a.sym = ws->tsym;
    a.stop = ws->stop;
    a.next_tile = ws->counter + 10;
    a.float_split = float_split ? 1 : 0;
    SPAMM_CK(cudaMemsetAsync(a.next_tile, 0, sizeof(int32_t), s));
    switch (slices) {
    case 1: return launch_tc_s<1>(a, s);
    case 2: return launch_tc_s<2>(a, s);
    case 3: return launch_tc_s<3>(a, s);
    case 4: return launch_tc_s<4>(a, s);
    case 5: return launch_tc_s<5>(a, s);
    case 6: return launch_tc_s<6>(a, s);
    case 7: return launch_tc_s<7>(a, s);
    default: return SPAMM_E_NOTSUP;
    }
}
