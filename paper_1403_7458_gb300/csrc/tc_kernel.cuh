// tc_kernel.cuh -- grouped leaf products on the tcgen05 tensor cores (the
// mixed-precision form of Algorithm 1's leaf branch), shared by the
// translation units that instantiate it per leaf size.
//
// Tiles.  A tile is R = 128 / b consecutive output leaf rows i = R I ..
// R I + R - 1 and W consecutive output leaf columns j = W J .. W J + W - 1
// (W = 2 at leaf 32, else 1; M = 128 rows).  Its work list holds every k
// for which at least one of its R W triples (i, k, j) survives the culling
// test of Eq. 4, with an R-bit mask of the survivors per column: the item's
// A slab (the R leaves (i, k)) is copied once for all W columns.  The MMAs
// of a column run over all R A leaves, with the TMEM lanes (output rows) of
// that column's culled triples disabled (the instruction's
// disable-output-lane mask), so each output leaf receives exactly the
// products of its own task list (no extra products, no missing ones).
//
// Slices.  With s slices per operand (see slice.cu), the MMAs for A slice p
// multiply the 128 x b A slab by B slices q = zB..s-1-p (N = b (s - p - zB))
// of a column's B leaf and accumulate into that column's TMEM columns
// [b (p + zB), b s) (column c's block starts at c s b): column block d then
// holds S_d = sum_{p+q=d} sum_k sum_l dA_p dB_q.  Pairs with p + q >= s are
// never formed, nor pairs with p < zA or q < zB, where zA (the least over
// the item's kept A leaves) and zB count leading slices that are zero in
// every element: those products are exactly zero.  An item whose kept leaves
// all have zA + zB >= s contributes exactly nothing and is not listed.  For
// exact (Ozaki) slices the S_d are integer-valued FP32 sums (exact while the
// absolute values of a diagonal's terms add up to less than 2^24, rounded by
// FP32 beyond that) and the epilogue forms
//     C = 2^(sigmaA + sigmaB - 7s - 7) * sum_d S_d 128^(s-1-d)
// exactly (int64, or 128-bit when the total could overflow) with one
// rounding to FP64; for float splits (BF16 or TF32 terms) it forms
// C = sum_d S_d in FP64.  It then zeroes the accumulator for the next tile.
//
// Element types.  BF16 slices use tcgen05.mma kind::f16 (K = 16 per
// instruction), TF32 slices kind::tf32 (K = 8); either way one instruction
// covers 32 bytes of K, so a b-wide leaf takes b e / 32 instructions per
// slice pair for e-byte elements.
//
// Batches.  The kernel parameters carry a table of up to kMaxBatch products
// (pointers, leaf grid, tile order); tiles of all of them are handed out
// from one device counter over the concatenated orders, so one persistent
// launch serves many independent SpAMMs.
//
// Kernel roles (320 threads, one CTA per SM, persistent):
//   warp 0     : producer; two bulk copies (cp.async.bulk) per work item:
//                the needed slices of the R A leaves (one contiguous block of
//                the tile-major array, stage layout [p][leaf][slice]) and of
//                the B leaf, into a shared-memory byte ring, completion on
//                the item's mbarrier;
//   warp 1     : allocates 512 TMEM columns; lane 0 issues the tcgen05.mma
//                of each landed item and commits to the item's "empty"
//                barrier and, at the end of a tile, to the accumulator's
//                "full" barrier;
//   warps 2-9  : epilogue, two warps per TMEM lane quadrant (each takes half
//                of a tile column's 16-column groups); tcgen05.ld of the s
//                diagonal blocks of the row the thread owns, combine, FP64
//                store, partial diagonal traces (two per leaf row).
// Two accumulators (TMEM columns 0 and 256) let the epilogue of one tile run
// under the MMAs of the next when a tile's W s b columns fit in 256 (else
// one accumulator: at leaf 32 with 7 slices a tile takes 448 columns).
// Every wait is bounded (SM cycle counter); on timeout the kernel records
// the error, drains and frees TMEM, and returns.
//
// Roofline: tensor pipe.  Useful work 2 b^3 per surviving triple; issued
// tensor work 2 * 128 * b * b per slice pair of a work item.
#pragma once

#include <type_traits>

#include "internal.cuh"

namespace tc {

// Shared-memory byte ring for work items: an item needing m slices per
// operand takes exactly m (R + 1) b^2 e bytes, so small items (many leading
// zero slices) leave room for more items in flight.
constexpr uint32_t kRingBytes = 216 * 1024;
constexpr int kSlots = 16;  // work items in flight at most
constexpr int kEpiWarps = 8;  // two epilogue warps per TMEM lane quadrant
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 256;
constexpr long long kTimeoutCycles = 8000000000ll;  // about 4 s at 2 GHz per wait
constexpr int kTileRing = 8;  // tiles handed from the producer to the other roles

// Work item of tile (I, j) at k: k | mask << 15 | zA << 23 | zB << 26.
__host__ __device__ constexpr uint32_t item_k(uint32_t w) { return w & 0x7FFF; }
__host__ __device__ constexpr uint32_t item_mask(uint32_t w) { return (w >> 15) & 0xFF; }
__host__ __device__ constexpr int item_za(uint32_t w) { return (int)((w >> 23) & 7); }
__host__ __device__ constexpr int item_zb(uint32_t w) { return (int)((w >> 26) & 7); }
__host__ __device__ constexpr uint32_t item_make(uint32_t k, uint32_t mask, int za, int zb)
{
    return k | (mask << 15) | ((uint32_t)za << 23) | ((uint32_t)zb << 26);
}
// Tiles of two output leaf columns (leaf 32, R = 4): mask bits 0-3 are
// column 0's kept rows, bits 4-7 column 1's; zB of column c at bits 26 + 3 c
// (7 for a column without kept rows).
__host__ __device__ constexpr uint32_t item_make2(uint32_t k, uint32_t mask0, uint32_t mask1, int za, int zb0,
                                                  int zb1)
{
    return k | (mask0 << 15) | (mask1 << 19) | ((uint32_t)za << 23) | ((uint32_t)zb0 << 26) | ((uint32_t)zb1 << 29);
}
template <int R, int W>
__host__ __device__ constexpr uint32_t item_mask_col(uint32_t w, int c)
{
    return (item_mask(w) >> (c * R)) & ((1u << R) - 1u);
}
__host__ __device__ constexpr int item_zb_col(uint32_t w, int c) { return (int)((w >> (26 + 3 * c)) & 7); }

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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          long long limit = kTimeoutCycles)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t it = 1;; it++) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255) == 0) {
            if (*abort_flag) return false;
            if (clock64() - t0 > limit) return false;
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

// Tensor copy of a 5-D box (tile mode) from the tensor described by the map
// at `map` (global memory) into shared memory, completion on the mbarrier.
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const void *map, int c0, int c1, int c2, int c3, int c4,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

// The tensor maps were written to global memory by an earlier kernel:
// order those writes before the tensor copies that read the map.
__device__ __forceinline__ void tmap_acquire(const void *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

// tcgen05 shared-memory descriptor of a K-major swizzled operand: start
// address, leading offset (unused by swizzled K-major layouts: 16 B), stride
// offset (8-row groups), version 1, swizzle mode for an atom of AW bytes
// (128 B: 2, 64 B: 4, 32 B: 6).  The atom's base is aligned to its repeat
// (8 AW bytes), so the base-offset field stays 0.
template <int AW>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo)
{
    constexpr uint64_t mode = AW == 128 ? 2 : AW == 64 ? 4 : 6;
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) |
           ((uint64_t)1 << 46) | (mode << 61);
}

// instruction descriptor: FP32 accumulator (bit 4), A and B types (bits 7
// and 10: BF16 = 1 under kind::f16, TF32 = 2 under kind::tf32), both
// K-major, N / 8 at bit 17, M / 16 at bit 24.
template <int E>
__device__ __forceinline__ uint32_t mma_idesc(int M, int N)
{
    constexpr uint32_t ab = E == 4 ? 2u : 1u;
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (TMEM) += A (smem) x B (smem); BF16 (E = 2, K = 16) or TF32 (E = 4,
// K = 8): 32 bytes of K per instruction either way.  Bit r of the 128-bit
// mask dis (dis[0] bit 0 = lane 0) set: TMEM lane r of D keeps its value.
template <int E>
__device__ __forceinline__ void mma_issue(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc,
                                          const uint32_t (&dis)[4])
{
    if (E == 4)
        asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, {%4, %5, %6, %7}, 1;" ::"r"(dtmem),
                     "l"(da), "l"(db), "r"(idesc), "r"(dis[0]), "r"(dis[1]), "r"(dis[2]), "r"(dis[3])
                     : "memory");
    else
        asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, {%4, %5, %6, %7}, 1;" ::"r"(dtmem),
                     "l"(da), "l"(db), "r"(idesc), "r"(dis[0]), "r"(dis[1]), "r"(dis[2]), "r"(dis[3])
                     : "memory");
}

// Word q of the disable-output-lane mask of an item with kept-leaf mask
// `mask`: the 32 TMEM lanes 32 q .. 32 q + 31 are rows of leaves
// 32 q / B .. (32 q + 31) / B; a lane is disabled when its leaf is culled.
template <int B>
__device__ __forceinline__ uint32_t culled_lanes(uint32_t mask, int q)
{
    if (B >= 32) return ((mask >> (32 * q / B)) & 1u) ? 0u : 0xFFFFFFFFu;
    uint32_t v = 0;
#pragma unroll
    for (int u = 0; u < 32 / B; u++)
        if (!((mask >> (q * (32 / B) + u)) & 1u)) v |= ((1u << B) - 1u) << (u * B);
    return v;
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
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

// The same value, RN(v * 2^k), from the hardware conversion: RN(v) (ties to
// even) scaled by 2^k through the exponent field, exact while the result is
// normal; the integer routine handles subnormal and overflowing results.
__device__ __forceinline__ double i64_scaled_fast(long long v, int k)
{
    if (v == 0) return 0.0;
    const double f = __ll2double_rn(v);
    const uint64_t u = (uint64_t)__double_as_longlong(f);
    const int e = (int)((u >> 52) & 0x7FF) + k;
    if (e >= 1 && e <= 2046) return __longlong_as_double((long long)(u + ((uint64_t)(int64_t)k << 52)));
    return i64_scaled(v, k);
}

// Exact combination of the diagonal sums of one output element (exact
// slices): RN(2^k sum_{d >= d0} S_d 128^(S-1-d)), every S_d an integer held
// in FP32 (integer-valued whatever its size).
// Fast path, when every |S_d| is below 2^22 and the int64 total cannot
// overflow (|S_d| 128^(S-1-d) < 2^59): each S_d becomes an int32 by the
// magic-number addition (f + 1.5 2^23 puts the integer in the low mantissa
// bits: one FP32 add, one integer subtract, both full-rate, where a
// float-to-int64 conversion runs on a slow unit), the int64 total is formed
// with shifts and adds and rounded once.  Otherwise a 128-bit total
// (float-to-int64 conversions, exact for integer-valued floats).
template <int S>
__device__ __noinline__ double combine_exact_slow(const uint32_t *f, int d0, int k)
{
    // every |S_d| < 2^31 (the usual case off the fast path): int32
    // conversions, the terms with shifts >= 28 in hi (scaled down by 2^28,
    // |hi| < 2^46) and the rest in lo (|lo| < 2^53); both convert exactly and
    // one fused multiply-add rounds hi 2^28 + lo once
    bool medium = true;
    for (int d = d0; d < S; d++) medium = medium && fabsf(__uint_as_float(f[d])) < 2147483648.0f;
    if (medium) {
        long long hi = 0, lo = 0;
        for (int d = d0; d < S; d++) {
            const int sh = 7 * (S - 1 - d);
            const long long iv = __float2int_rn(__uint_as_float(f[d]));
            if (sh >= 28) hi += iv << (sh - 28);
            else lo += iv << sh;
        }
        const double x = fma((double)hi, 268435456.0, (double)lo);  // RN(hi 2^28 + lo)
        if (x == 0.0) return 0.0;
        const uint64_t u = (uint64_t)__double_as_longlong(x);
        const int e = (int)((u >> 52) & 0x7FF) + k;
        if (e >= 1 && e <= 2046) return __longlong_as_double((long long)(u + ((uint64_t)(int64_t)k << 52)));
    }
    __int128 a = 0;
    for (int d = d0; d < S; d++)
        a += (__int128)__float2ll_rn(__uint_as_float(f[d])) << (7 * (S - 1 - d));
    if (a == 0) return 0.0;
    const bool neg = a < 0;
    const double r = u128_round_scaled((u128)(neg ? -a : a), k);
    return neg ? -r : r;
}

// The 16 values of one TMEM load group at once (straight-line code, so that
// the 16 chains interleave): fast path for all of them when every one
// qualifies, else the 128-bit path for each.  The fast path pairs the
// diagonals from the bottom, P_j = S_(S-1-2j) + 128 S_(S-2-2j): with every
// |S_d| < 2^22 a pair fits an int32 and is formed on the raw FP32 bits
// (each S_d + 1.5 2^23 carries the integer in its low bits; the offsets are
// removed once per pair, modulo 2^32, which is exact since the true value
// fits), and the total is sum_j P_j 2^(14 j) in int64.
// Returns the number of the 16 values with a diagonal sum at or beyond 2^24
// (certainly rounded by its FP32 accumulation); only the slow path can see
// one.
template <int S>
__device__ __forceinline__ int combine_exact16(const uint32_t (&v)[S][16], int d0, int k, double (&res)[16])
{
    constexpr uint32_t kMagicBits = 0x4B400000u;  // bits of 1.5 2^23
    bool fast = true;
    long long a[16];
#pragma unroll
    for (int q = 0; q < 16; q++) a[q] = 0;
#pragma unroll
    for (int j = 0; j < (S + 1) / 2; j++) {
        const int da = S - 1 - 2 * j, db = da - 1;  // db < 0: the top diagonal alone (S odd)
        if (da < d0) continue;  // warp-uniform: both diagonals below d0 are zero
        // |S_d| < 2^min(22, 59 - 7 (S - 1 - d)): exact conversion, no int64 overflow
        const float lima = 7 * (S - 1 - da) + 22 <= 59 ? 4194304.0f : __int_as_float((127 + 59 - 7 * (S - 1 - da)) << 23);
        const float limb = db < 0 || 7 * (S - 1 - db) + 22 <= 59 ? 4194304.0f
                                                               : __int_as_float((127 + 59 - 7 * (S - 1 - db)) << 23);
#pragma unroll
        for (int q = 0; q < 16; q++) {
            const float fa = __uint_as_float(v[da][q]);
            fast = fast && fabsf(fa) < lima;
            const uint32_t ua = __float_as_uint(fa + 12582912.0f);
            int32_t p;
            if (db >= 0) {
                const float fb = __uint_as_float(v[db][q]);
                fast = fast && fabsf(fb) < limb;
                const uint32_t ub = __float_as_uint(fb + 12582912.0f);
                p = (int32_t)(ua + (ub << 7) - 129u * kMagicBits);
            } else {
                p = (int32_t)(ua - kMagicBits);
            }
            a[q] += (long long)p << (14 * j);
        }
    }
    int rounded = 0;
    if (fast) {
#pragma unroll
        for (int q = 0; q < 16; q++) res[q] = i64_scaled_fast(a[q], k);
    } else {
        for (int q = 0; q < 16; q++) {
            uint32_t f[S];
            bool big = false;
#pragma unroll
            for (int d = 0; d < S; d++) {
                f[d] = v[d][q];
                big = big || (d >= d0 && fabsf(__uint_as_float(f[d])) >= 16777216.0f);
            }
            rounded += big;
            res[q] = combine_exact_slow<S>(f, d0, k);
        }
    }
    return rounded;
}

// One product of a launch.
struct TcProb {
    const uint8_t *slA;    // A operand: tile-major [I][k][p][L][slice]
    const uint8_t *slB;    // B operand: per slot [q][slice] (symmetric: A-role of the transpose)
    const int32_t *slotA;  // nb*nb
    const int32_t *slotB;
    const int32_t *slotC;
    double *leafC;
    const int32_t *cnt;    // work items per tile
    const int32_t *d0;     // per tile and column c: least zA + zB of its items (4 bits at 4 c; S: none),
                           // leaf rows with work (R bits at 8 + 8 c)
    const uint32_t *list;  // work items: tile t's at [t nb, t nb + cnt[t])
    const int32_t *order;  // tile order (tile ids of this product; -1 after the tiles with work)
    const void *tmB;       // symmetric product: tensor maps of slA for the B leaves (map h - 1:
                           // h slices of one leaf), used instead of slB; else null
    const int32_t *sigA;   // sigma of A
    const int32_t *sigB;
    double *tr_part;       // diagonal-leaf partial traces, two per leaf row (may be null; b <= 32)
    int64_t nb;
    int64_t nbt;           // tiles per tile row: ceil(nb / W), W output leaf columns per tile
    int64_t pos0;          // first hand-out position of this product
    int32_t sym;           // symmetric product: upper block triangle + mirror
    int32_t tw;            // output leaf columns per tile of its work lists
    int32_t mirror;        // symmetric product: also store C_ji = C_ij^T (else leaves i <= j only)
    int32_t skip_idle;     // output leaves without work in a tile with work are not written (else zeroed)
    int32_t *rounded;      // exact slices: += output elements with a diagonal sum >= 2^24 (may be null)
};

struct TcArgs {
    TcProb p[kMaxBatch];
    int64_t T;             // hand-out positions over all products
    int32_t *err;          // error word (timeout)
    int32_t *next_tile;    // dynamic scheduler: next position (zeroed per launch)
    const int32_t *stop;   // set once an SP2 loop has stopped: nothing to do
    int32_t nprob;
    int32_t float_split;   // slices are a float split: C = sum_d S_d in FP64, no scaling
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

// The product owning hand-out position pos (products sorted by pos0).
__device__ __forceinline__ int find_prob(const TcArgs &g, int64_t pos)
{
    int lo = 0, hi = g.nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g.p[mid].pos0 <= pos) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int S, int E, int B, int W>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(const __grid_constant__ TcArgs g)
{
    constexpr int R = 128 / B;                  // leaf rows per tile
    constexpr uint32_t kSlice = B * B * E;      // one slice of one leaf (bytes)
    constexpr uint32_t kSBO = 8 * B * E;        // 8-row group stride
    constexpr uint32_t kAW = slice_atom_bytes<B, E>();  // swizzle atom width (bytes)
    constexpr int kMmaK = B * E / 32;           // instructions per slice pair
    constexpr uint32_t kColAcc = S * B;         // TMEM columns per output leaf column
    // two accumulators (columns 0 and kAccStride) when a tile's fit in half
    // of TMEM, else one
    constexpr int kNAcc = W * S * B <= (int)kAccStride ? 2 : 1;
    static_assert(W * S * B <= (int)kTmemCols, "accumulators exceed TMEM");
    static_assert(R * W <= 8, "the item's masks exceed 8 bits");
    static_assert((uint32_t)S * (R + W) * kSlice <= kRingBytes, "work item exceeds the ring");
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full_bar[kSlots], empty_bar[kSlots];
    __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2], done_bar;
    __shared__ uint32_t slot_off[kSlots];  // ring byte offset of each in-flight item
    __shared__ uint32_t slot_w[kSlots];    // its work-list entry
    __shared__ unsigned long long slot_end[kSlots];  // its end in the producer's cumulative ring pointer
    __shared__ int32_t tile_q[kTileRing];  // tiles handed out (product << 24 | tile), -1 = no more
    __shared__ int32_t tile_n[kTileRing];  // their work-item counts
    __shared__ int32_t tile_d[kTileRing];  // and least diagonals (4 bits per column)
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
            mbar_init(smem_u32(&acce_bar[q]), kEpiWarps);
        }
        mbar_init(smem_u32(&done_bar), 1);
        for (int q = 0; q < kTileRing; q++) {
            mbar_init(smem_u32(&tfull_bar[q]), 1);
            mbar_init(smem_u32(&tempty_bar[q]), 1 + kEpiWarps);  // MMA and the epilogue warps
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
    // the ring starts on a 1 KB boundary: swizzle atoms (up to 8 rows x 128 B)
    // must sit at addresses aligned to their repeat
    const uint32_t sraw = smem_u32(smem);
    const uint32_t sbase = (sraw + 1023u) & ~1023u;
    volatile int *abort_v = &abort_flag;

    if (warp == 0) {
        // ------------------------------ producer ------------------------------
        // The warp loads 32 work entries (and their B slots) at a time; lane 0
        // then allocates ring space and issues the copies item by item.
        // cumulative byte pointers (allocation incl. wrap padding, release)
        unsigned long long alloc_ptr = 0, free_ptr = 0;
        uint32_t ring_pos = 0;  // alloc_ptr modulo the ring size
        uint32_t issued = 0, released = 0;
        bool ok = true;
        uint32_t tq = 0, tph = 0;
        if (lane == 0)
            for (int mp = 0; mp < g.nprob; mp++)
                if (g.p[mp].tmB)
                    for (int h = 0; h < S; h++) tmap_acquire(static_cast<const uint8_t *>(g.p[mp].tmB) + 128 * h);
        for (;;) {
            // take the next tile and hand it to the MMA and epilogue warps
            int32_t tt = -1, tn = 0;
            int tgood = 1;
            if (lane == 0) {
                if (!mbar_wait(smem_u32(&tempty_bar[tq]), tph ^ 1, abort_v)) {
                    tgood = 0;
                } else {
                    for (;;) {
                        const int32_t pos = atomicAdd(g.next_tile, 1);
                        if (pos >= T) break;
                        const int mp = find_prob(g, pos);
                        const int32_t o = g.p[mp].order[pos - g.p[mp].pos0];
                        if (o >= 0) {
                            tt = (mp << 24) | o;
                            tn = g.p[mp].cnt[o];
                            tile_n[tq] = tn;
                            tile_d[tq] = g.p[mp].d0[o];
                            break;
                        }
                        // the rest of this product's order holds no tile with
                        // work: move the counter past it (positions only grow)
                        atomicMax(g.next_tile, (int32_t)(mp + 1 < g.nprob ? g.p[mp + 1].pos0 : T));
                    }
                    tile_q[tq] = tt;
                    mbar_arrive(smem_u32(&tfull_bar[tq]));
                }
            }
            tt = __shfl_sync(0xffffffffu, tt, 0);
            tn = __shfl_sync(0xffffffffu, tn, 0);
            if (!__shfl_sync(0xffffffffu, tgood, 0)) {
                ok = false;
                break;
            }
            if (++tq == kTileRing) {
                tq = 0;
                tph ^= 1;
            }
            if (tt < 0) break;
            const TcProb &P = g.p[tt >> 24];
            const int64_t t = tt & 0xFFFFFF;
            const int64_t nb = P.nb;
            const int64_t I = t / P.nbt, J = t % P.nbt;
            const int64_t e0 = t * nb, e1 = e0 + tn;
            for (int64_t base = e0; base < e1 && ok; base += 32) {
                const int cnt = (int)(e1 - base < 32 ? e1 - base : 32);
                uint32_t wl = 0;
                int64_t bl[W];
#pragma unroll
                for (int c = 0; c < W; c++) bl[c] = 0;
                if (lane < cnt) {
                    wl = P.list[base + lane];
                    const int64_t kk = item_k(wl);
#pragma unroll
                    for (int c = 0; c < W; c++) {
                        const int64_t j = W * J + c;
                        if (j < nb && item_mask_col<R, W>(wl, c) && !P.tmB)
                            bl[c] = P.sym ? P.slotA[j * nb + kk] : P.slotB[kk * nb + j];
                    }
                }
                // The whole warp runs the per-item bookkeeping (the values are
                // uniform across its lanes, so it never diverges); lane 0 alone
                // issues the copies.
                for (int q = 0; q < cnt; q++) {
                    const uint32_t w = __shfl_sync(0xffffffffu, wl, q);
                    int64_t bslot[W];
#pragma unroll
                    for (int c = 0; c < W; c++) bslot[c] = __shfl_sync(0xffffffffu, bl[c], q);
                    const int64_t k = item_k(w);
                    const int za = item_za(w);
                    int mc[W], mA = 0;
                    uint32_t need = 0;
#pragma unroll
                    for (int c = 0; c < W; c++) {
                        // slices needed from column c's B leaf (none: column absent)
                        mc[c] = item_mask_col<R, W>(w, c) ? S - za - item_zb_col(w, c) : 0;
                        mA = mc[c] > mA ? mc[c] : mA;
                        need += (uint32_t)mc[c] * kSlice;
                    }
                    need += (uint32_t)mA * R * kSlice;
                    if (ring_pos + need > kRingBytes) {  // the item does not fit before the end: wrap
                        alloc_ptr += kRingBytes - ring_pos;
                        ring_pos = 0;
                    }
                    const uint32_t pos = ring_pos;
                    const unsigned long long new_end = alloc_ptr + need;
                    // wait (in order) for released items until the region and a slot are free
                    for (;;) {
                        // nothing in flight: the wrap padding before the region holds
                        // nothing either (an item larger than the space left after the
                        // last wrap would otherwise wait for space that never frees)
                        if (released == issued) free_ptr = alloc_ptr;
                        if (new_end - free_ptr <= kRingBytes && issued - released < (uint32_t)kSlots) break;
                        const uint32_t rs = released % kSlots;
                        if (!mbar_wait(smem_u32(&empty_bar[rs]), (released / kSlots) & 1, abort_v)) {
                            ok = false;
                            break;
                        }
                        free_ptr = slot_end[rs];
                        released++;
                    }
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                    const uint32_t sl = issued % kSlots;
                    if (lane == 0) {
                        slot_off[sl] = pos;
                        slot_w[sl] = w;
                        slot_end[sl] = new_end;
                        const uint32_t fb = smem_u32(&full_bar[sl]);
                        uint32_t dst = sbase + pos;
                        mbar_expect_tx(fb, need);
                        // A: slices za..za+mA-1 of the R rows' leaves, one contiguous block
                        bulk_g2s(dst, P.slA + ((I * nb + k) * S + za) * (int64_t)(R * kSlice),
                                 (uint32_t)mA * R * kSlice, fb);
                        dst += (uint32_t)mA * R * kSlice;
                        // B: slices zb..S-1-za of leaf (k, j) per present column
                        // (symmetric: leaf (j, k), from the tile-major array
                        // when tensor maps are given)
#pragma unroll
                        for (int c = 0; c < W; c++) {
                            if (mc[c] <= 0) continue;
                            if (P.tmB) {
                                const int64_t j = W * J + c;
                                tma_load_5d(dst, static_cast<const uint8_t *>(P.tmB) + 128 * (mc[c] - 1), 0, 0,
                                            (int)(j % R), item_zb_col(w, c), (int)((j / R) * nb + k), fb);
                            } else {
                                bulk_g2s(dst,
                                         P.slB + bslot[c] * (int64_t)(S * kSlice) + item_zb_col(w, c) * kSlice,
                                         (uint32_t)mc[c] * kSlice, fb);
                            }
                            dst += (uint32_t)mc[c] * kSlice;
                        }
                    }
                    __syncwarp();
                    alloc_ptr = new_end;
                    ring_pos += need;
                    issued++;
                }
            }
            if (!ok) break;  // a wait gave up: no further tiles
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
        // Lane 0 alone: waits until an item has landed, then issues its MMAs
        // (per present column, with the TMEM lanes of that column's culled
        // leaf rows disabled) and commits them to the item's "empty" barrier
        // and, at the end of a tile, to the accumulator's "full" barrier.
        if (lane == 0) {
            uint32_t consumed = 0, acc = 0, aph = 0;
            bool ok = true;
            uint32_t tq = 0, tph = 0;
            for (;;) {
                if (!mbar_wait(smem_u32(&tfull_bar[tq]), tph, abort_v)) {
                    ok = false;
                    break;
                }
                const int32_t tt = tile_q[tq], tn = tile_n[tq];
                mbar_arrive(smem_u32(&tempty_bar[tq]));
                if (++tq == kTileRing) {
                    tq = 0;
                    tph ^= 1;
                }
                if (tt < 0) break;
                const TcProb &P = g.p[tt >> 24];
                const int64_t t = tt & 0xFFFFFF;
                // the accumulator was zeroed by the epilogue (phase u of its barrier)
                if (!mbar_wait(smem_u32(&acce_bar[acc]), aph, abort_v)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dacc = tmem + acc * kAccStride;
                const int64_t e1 = t * P.nb + tn;
                for (int64_t e = t * P.nb; e < e1; e++) {
                    const uint32_t sl = consumed % kSlots;
                    if (!mbar_wait(smem_u32(&full_bar[sl]), (consumed / kSlots) & 1, abort_v)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t w = slot_w[sl], pos = slot_off[sl];
                    const int za = item_za(w);
                    int mc[W], mA = 0;
#pragma unroll
                    for (int c = 0; c < W; c++) {
                        mc[c] = item_mask_col<R, W>(w, c) ? S - za - item_zb_col(w, c) : 0;
                        mA = mc[c] > mA ? mc[c] : mA;
                    }
                    const uint32_t sa = sbase + pos;                  // A slice za
                    uint32_t sb = sa + (uint32_t)mA * R * kSlice;     // B slices of the first present column
                    // descriptors advance by adding (bytes >> 4) to the address field
                    // (shared addresses stay below 256 KB, so the field never carries)
                    const uint64_t da0 = smem_desc<kAW>(sa, kSBO);
#pragma unroll
                    for (int c = 0; c < W; c++) {
                        if (mc[c] <= 0) continue;
                        const uint32_t mask = item_mask_col<R, W>(w, c);
                        const uint32_t dis[4] = {culled_lanes<B>(mask, 0), culled_lanes<B>(mask, 1),
                                                 culled_lanes<B>(mask, 2), culled_lanes<B>(mask, 3)};
                        const uint64_t db0 = smem_desc<kAW>(sb, kSBO);
                        uint32_t idesc = mma_idesc<E>(128, B * mc[c]);
                        uint32_t dcol = dacc + c * kColAcc + B * (za + item_zb_col(w, c));
                        for (int pp = 0; pp < mc[c]; pp++) {
                            const uint64_t da = da0 + (uint64_t)(pp * (R * kSlice / 16));
#pragma unroll
                            for (int h = 0; h < kMmaK; h++) {
                                // 32 bytes of K each: inside a swizzle atom the start
                                // address moves by 32 B, across atoms by 8 AW bytes
                                const uint32_t kb = (uint32_t)(32 * h);
                                const uint64_t adv = ((kb / kAW) * 8 * kAW + kb % kAW) >> 4;
                                mma_issue<E>(dcol, da + adv, db0 + adv, idesc, dis);
                            }
                            idesc -= (uint32_t)(B >> 3) << 17;  // N shrinks by b
                            dcol += B;
                        }
                        sb += (uint32_t)mc[c] * kSlice;
                    }
                    mma_commit(smem_u32(&empty_bar[sl]));
                    consumed++;
                }
                if (!ok) break;
                mma_commit(smem_u32(&accf_bar[acc]));
                if (++acc == (uint32_t)kNAcc) {
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
        // ------------------------------ epilogue (warps 2-9) ------------------------------
        // Two warps per TMEM lane quadrant (a warp may only access the lanes
        // 32 (warp % 4) .. + 31): member m of the quadrant handles the
        // 16-column groups h in [m HPM, (m + 1) HPM) of every tile column.
        constexpr int NH = B / 16, HPM = (NH + 1) / 2;
        const int m = (warp - 2) >> 2;
        const int h_lo = m * HPM, h_hi = min(NH, h_lo + HPM);
        const int quad = warp & 3;             // TMEM lane quadrant of this warp
        const int row = quad * 32 + lane;      // tile row 0..127
        const int L = row / B, r = row % B;    // leaf within tile, row within leaf
        const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
        // the accumulators start at zero (first phase of their "empty" barriers)
        for (int b = 0; b < kNAcc; b++) {
            for (int d = 0; d < W * S; d++)
                for (int h = h_lo; h < h_hi; h++) tmem_zero16(tmem + b * kAccStride + lane_off + B * d + 16 * h);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0)
            for (int b = 0; b < kNAcc; b++) mbar_arrive(smem_u32(&acce_bar[b]));
        uint32_t acc = 0, aph = 0;
        uint32_t tq = 0, tph = 0;
        for (;;) {
            int32_t tt = -1, tn = 0, td = 0;
            int tgood = 1;
            if (lane == 0) {
                tgood = mbar_wait(smem_u32(&tfull_bar[tq]), tph, abort_v);
                if (tgood) {
                    tt = tile_q[tq];
                    tn = tile_n[tq];
                    td = tile_d[tq];
                    mbar_arrive(smem_u32(&tempty_bar[tq]));
                }
            }
            tt = __shfl_sync(0xffffffffu, tt, 0);
            tn = __shfl_sync(0xffffffffu, tn, 0);
            td = __shfl_sync(0xffffffffu, td, 0);
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
            const TcProb &P = g.p[tt >> 24];
            const int64_t t = tt & 0xFFFFFF;
            const int64_t nb = P.nb;
            const int64_t I = t / P.nbt, J = t % P.nbt;
            const bool has_work = tn > 0;
            // the least diagonal any item of the tile touches per column (from
            // the tile cull): the diagonals below it were never written and
            // are still zero, so they are neither read, cleared nor combined
            int d0[W];
#pragma unroll
            for (int c = 0; c < W; c++) {
                d0[c] = g.float_split ? 0 : (td >> (4 * c)) & 15;
                if (d0[c] > S) d0[c] = S;
            }
            // the output leaves' slots and the scale, loaded while the tile's
            // products are still running
            const int64_t i = (int64_t)R * I + L;
            const int kexp = g.float_split ? 0 : *P.sigA + *P.sigB - 7 * S - 7;
            int32_t oslot[W];
#pragma unroll
            for (int c = 0; c < W; c++) {
                const int64_t j = W * J + c;
                oslot[c] = (i < nb && j < nb && (!P.sym || i <= j)) ? __ldg(P.slotC + i * nb + j) : 0;
            }
            if (!mbar_wait(smem_u32(&accf_bar[acc]), aph, abort_v)) {
                if (lane == 0) atomicExch(g.err, 1);
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            double diag = 0.0;
            bool on_diag = false;
            bool released = false;  // this warp has released the accumulator
#pragma unroll 1
            for (int c = 0; c < W; c++) {
                const int64_t j = W * J + c;
                if (j >= nb) break;  // no such column (nothing was accumulated there)
                // symmetric mode: leaf (i, j) is written only for i <= j, and for
                // i < j its transpose goes to leaf (j, i)
                const bool store_leaf = i < nb && (!P.sym || i <= j);
                int32_t osl = 0;  // oslot[c] (static indexing)
#pragma unroll
                for (int cc = 0; cc < W; cc++)
                    if (cc == c) osl = oslot[cc];
                // a leaf row that none of the column's items keeps has an
                // all-zero accumulator: it is not read (when its whole warp is
                // idle), and it is written as zeros or, when the caller knows
                // it from the tile masks, not at all
                const bool idle = !((td >> (8 + 8 * c + L)) & 1);
                const bool widle = __all_sync(0xffffffffu, idle);
                const bool store = store_leaf && !(idle && P.skip_idle);
                double *dst = store ? P.leafC + (int64_t)osl * (B * B) + r * B : nullptr;
                double *mir =
                    (store && P.sym && P.mirror && i < j) ? P.leafC + (int64_t)P.slotC[j * nb + i] * (B * B) + r
                                                          : nullptr;
                const uint32_t tbase = tmem + acc * kAccStride + c * kColAcc + lane_off;
                if (i == j) on_diag = true;
                int dc = S;  // d0 of column c (static indexing of d0[])
#pragma unroll
                for (int cc = 0; cc < W; cc++)
                    if (cc == c) dc = d0[cc];
#pragma unroll
                for (int hh = 0; hh < HPM; hh++) {
                    const int h = h_lo + hh;
                    if (h >= h_hi) break;  // warp-uniform
                    // the last group of the tile this warp handles: once its
                    // values are in registers and its columns cleared, the
                    // accumulator is released (the combination and the stores
                    // below need no tensor memory)
                    const bool last = (h + 1 >= h_hi) && (c + 1 >= W || W * J + c + 1 >= nb);
                    // the S diagonals of these 16 columns: all loads issued,
                    // one wait, the accumulator zeroed for the next tile
                    if (widle) {  // warp-uniform: every row of this warp is idle
                        if (last && !released) {
                            // (clears of an earlier column of the tile complete first)
                            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                            __syncwarp();
                            if (lane == 0) mbar_arrive(smem_u32(&acce_bar[acc]));
                            released = true;
                        }
                        if (store) {
                            const double2 z = make_double2(0.0, 0.0);
#pragma unroll
                            for (int q = 0; q < 16; q += 2) {
                                const int col = 16 * h + q;
                                reinterpret_cast<double2 *>(dst)[col >> 1] = z;
                                if (mir) {
                                    mir[col * B] = 0.0;
                                    mir[(col + 1) * B] = 0.0;
                                }
                            }
                        }
                        continue;
                    }
                    uint32_t v[S][16];
                    if (has_work) {
#pragma unroll
                        for (int d = 0; d < S; d++) {
                            if (d >= dc) tmem_ld16(tbase + B * d + 16 * h, v[d]);
                            else
#pragma unroll
                                for (int q = 0; q < 16; q++) v[d][q] = 0u;
                        }
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int d = 0; d < S; d++)
                            if (d >= dc) tmem_zero16(tbase + B * d + 16 * h);
                    } else {
#pragma unroll
                        for (int d = 0; d < S; d++)
#pragma unroll
                            for (int q = 0; q < 16; q++) v[d][q] = 0u;
                    }
                    if (last && !released) {
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(smem_u32(&acce_bar[acc]));
                        released = true;
                    }
                    // exact slices: integer combination; float split: FP64 sum
                    double res[16];
                    if (g.float_split) {
#pragma unroll
                        for (int q = 0; q < 16; q++) {
                            double a = 0.0;
#pragma unroll
                            for (int d = 0; d < S; d++) a += (double)__uint_as_float(v[d][q]);
                            res[q] = a;
                        }
                    } else {
                        const int nr = combine_exact16<S>(v, dc, kexp, res);
                        if (nr && P.rounded) atomicAdd(P.rounded, nr);  // rare: the slow path only
                    }
                    if (store) {
#pragma unroll
                        for (int q = 0; q < 16; q += 2) {
                            const int col = 16 * h + q;
                            double2 v;
                            v.x = res[q];
                            v.y = res[q + 1];
                            if (i == j && col == (r & ~1)) diag = (r & 1) ? v.y : v.x;
                            reinterpret_cast<double2 *>(dst)[col >> 1] = v;
                            if (mir) {
                                mir[col * B] = v.x;
                                mir[(col + 1) * B] = v.y;
                            }
                        }
                    }
                }
            }
            if (!released) {  // no group of this warp (e.g. every column past the matrix)
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&acce_bar[acc]));
            }
            if (++acc == (uint32_t)kNAcc) {
                acc = 0;
                aph ^= 1;
            }
            if (B <= 32 && P.tr_part) {
                // fixed butterfly over the B rows of a diagonal leaf (a warp
                // holds 32 / B whole leaves, each within one tile column; the
                // condition is uniform over each leaf's rows); member m holds
                // the diagonal elements in its column groups and writes its
                // partial trace to tr_part[2 i + m]
                for (int o = B / 2; o > 0; o >>= 1) diag += __shfl_xor_sync(0xffffffffu, diag, o);
                if (r == 0 && on_diag && i < nb) P.tr_part[2 * i + m] = diag;
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

// Output leaf columns per tile: two at leaf 32 when the tile's accumulators
// still fit twice in TMEM (s <= 4 slices: the A slab of an item serves both
// columns, and the epilogue of one tile runs under the MMAs of the next),
// one otherwise (measured: with a single accumulator the tile epilogue is
// exposed and costs more than the shared A slab saves).
constexpr int tile_width(int B, int S) { return (B == 32 && 2 * S * B <= (int)kAccStride) ? 2 : 1; }

template <int S, int E, int B>
int launch_k(const TcArgs &a, cudaStream_t s)
{
    constexpr int W = tile_width(B, S);
    for (int m = 0; m < a.nprob; m++)
        if (a.p[m].tw != W) {
            spamm_set_error("tensor-core kernel: work lists of %d-column tiles, kernel built for %d", a.p[m].tw, W);
            return SPAMM_E_INVAL;
        }
    const size_t smem = kRingBytes + 1024;  // + alignment slack of the ring
    static unsigned long long configured = 0;
    if (int rc = spamm_smem_attr(k_gemm_tc<S, E, B, W>, smem, configured)) return rc;
    int64_t grid = spamm_num_sms();
    if (grid > a.T) grid = a.T;
    if (grid < 1) grid = 1;
    k_gemm_tc<S, E, B, W><<<(unsigned)grid, kThreads, smem, s>>>(a);
    SPAMM_CK_LAUNCH();
    return SPAMM_OK;
}

// Launch for leaf B with S slices of E-byte elements; E_NOTSUP if that
// combination is not instantiated.
template <int B>
int launch_leaf(const TcArgs &a, int S, int E, cudaStream_t s)
{
#define SPAMM_TC_CASE(SS, EE)                                            \
    if constexpr (SS * B <= (int)kAccStride)                             \
        if (S == SS && E == EE) return launch_k<SS, EE, B>(a, s);
    SPAMM_TC_CASE(1, 2)
    SPAMM_TC_CASE(2, 2)
    SPAMM_TC_CASE(3, 2)
    SPAMM_TC_CASE(4, 2)
    SPAMM_TC_CASE(5, 2)
    SPAMM_TC_CASE(6, 2)
    SPAMM_TC_CASE(7, 2)
    SPAMM_TC_CASE(1, 4)
    SPAMM_TC_CASE(2, 4)
#undef SPAMM_TC_CASE
    spamm_set_error("tensor-core kernel: %d slices of %d-byte elements at leaf %d not built", S, E, B);
    return SPAMM_E_NOTSUP;
}

}  // namespace tc

// Per-leaf launchers (gemm_tc_b16.cu, gemm_tc.cu, gemm_tc_b64.cu).
int tc_launch_b16(const tc::TcArgs &a, int S, int E, cudaStream_t s);
int tc_launch_b32(const tc::TcArgs &a, int S, int E, cudaStream_t s);
int tc_launch_b64(const tc::TcArgs &a, int S, int E, cudaStream_t s);
