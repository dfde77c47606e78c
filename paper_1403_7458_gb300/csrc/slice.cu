// slice.cu -- exact integer slices of FP64 leaves for the tensor-core path.
//
// Every element x of a matrix is scaled by the matrix's global power of two
// 2^-sigma (sigma chosen so that max|x| < 2^sigma), rounded to the integer
// X = round(|x| 2^(7s - sigma)) <= 2^(7s), and cut into s base-128 digits,
//     X = sum_p d_p 128^(s-1-p),  d_0 in [0, 128], d_p in [0, 127] (p > 0),
// each carrying the sign of x.  Digits are integers of at most 8 bits, so
// BF16 holds them exactly and their pairwise products are exact in FP32;
// a sum of such products is exact while the absolute values of its terms
// add up to less than 2^24 (beyond that FP32 rounds it).
// (Error-free splitting after Ozaki, Ogita, Oishi and Rump, 2012.)
//
// Float splits instead store s_0 = round(x), s_1 = round(x - s_0), ... in
// BF16 or TF32 (round to nearest), for the low-precision modes.
//
// Two layouts per b x b leaf (b = 16, 32, 64), both slice-major and each
// slice in the tcgen05 K-major swizzled layout (slice_byte_offset: 8-row
// groups, 32/64/128-byte swizzle atoms along K); slice p occupies bytes
// [p b^2 e, (p+1) b^2 e) for e-byte elements:
//   A role : rows r of the leaf, K = columns l
//   B role : rows = columns c of the leaf (N), K = rows l
// The B-role image of leaf (k, j) equals the A-role image of its transpose,
// so for a symmetric matrix the A-role array serves both operands.  The
// tile-major A array puts the R = 128 / b leaves (i, k), i = R I .. R I + R-1,
// of one tile next to each other per slice: [I][k][p][L][slice].
//
// Leaves of squared norm 0 are skipped (no product reads their slices).
// Per leaf the number z of leading all-zero slices (every digit d_p, p < z,
// is 0) is recorded: slice pairs touching them contribute exactly nothing.
//
// Roofline: HBM-bound; per element 8 B read, 2 e s B written (both roles).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <string.h>

#include <type_traits>

#include "internal.cuh"

namespace {

// Threads of a slicing block (one leaf at a time): small blocks keep more
// leaves in flight per SM, the kernel being bound by each leaf's chain of
// dependent loads rather than by bandwidth.
constexpr int kSliceThreads = 128;

// max |x| over the stored leaves, as the IEEE bit pattern (monotone for
// non-negative doubles), by integer atomicMax: exact and order-free.
__global__ void k_absmax(const int32_t *__restrict__ stop, const double *__restrict__ leaf, int64_t count,
                         unsigned long long *__restrict__ out)
{
    if (stop && *stop) return;  // the SP2 loop has already stopped
    unsigned long long m = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride) {
        unsigned long long u = (unsigned long long)__double_as_longlong(leaf[q]) & 0x7FFFFFFFFFFFFFFFull;
        if (u > m && u < 0x7FF0000000000000ull) m = u;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// A fixed scale for callers that bound their matrix: max|x| is taken as 1.0,
// so sigma = 1 (|x| < 2).
__global__ void k_unit_scale(const int32_t *__restrict__ stop, unsigned long long *__restrict__ out)
{
    if (stop && *stop) return;
    *out = 0x3FF0000000000000ull;  // bits of 1.0
}

// sigma: the smallest integer with max|x| < 2^sigma (0 for an all-zero matrix)
__device__ __forceinline__ int sigma_of(unsigned long long maxbits)
{
    if (maxbits == 0) return 0;
    int E = (int)(maxbits >> 52);
    if (E == 0) return -1022;  // subnormal maximum
    return E - 1022;
}

// Round to the nearest TF32 (10 fraction bits, ties away from zero): the
// bit pattern of an FP32 value whose low 13 bits are zero.
__device__ __forceinline__ uint32_t to_tf32(float f)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
    return r;
}

// Slice p of element x as the stored element: exact digit (BF16) or the next
// term of a float split (BF16 or TF32); `rest` carries the unsplit remainder.
template <int E>
__device__ __forceinline__ uint32_t slice_elem(uint64_t X, bool neg, int p, int S, bool float_split, double &rest)
{
    if (E == 4) {
        const uint32_t t = to_tf32((float)rest);
        rest -= (double)__uint_as_float(t);
        return t;
    }
    if (float_split) {
        const __nv_bfloat16 t = __double2bfloat16(rest);
        rest -= (double)__bfloat162float(t);
        return __bfloat16_as_ushort(t);
    }
    return slice_digit_bf16(X, neg, p, S);
}

// One block per leaf position (i, k) of the rows = R * ceil(nb / R) padded
// leaf rows (R = 128 / B): slices of the leaf staged in shared memory in the
// core-matrix layout, then copied to the per-leaf and/or tile-major arrays.
template <int S, int E, int B>
__global__ void __launch_bounds__(kSliceThreads)
k_slice(const int32_t *__restrict__ stop, const double *__restrict__ leaf, const int32_t *__restrict__ slot,
        const double *__restrict__ n2, int64_t P, int64_t nb, int64_t rows,
        const unsigned long long *__restrict__ maxbits, int32_t *__restrict__ sigma_out,
        uint8_t *__restrict__ tileA, uint8_t *__restrict__ perleaf, int perleaf_transposed,
        uint8_t *__restrict__ zlead, int32_t *__restrict__ overflow, int float_split, int chunk,
        const double *__restrict__ keep_max, int keep_by_row, double tau2)
{
    using W = typename std::conditional<E == 4, uint32_t, uint16_t>::type;
    constexpr int R = 128 / B;               // leaf rows per tile
    constexpr int kU4 = B * B * E / 16;      // 16-byte chunks per slice
    constexpr int kThreads = kSliceThreads;  // the launch's block size
    constexpr int kPerThread = B * B / kThreads;
    static_assert(B * B % kThreads == 0, "leaf elements must be a multiple of the block size");
    __shared__ __align__(16) W sa[S * B * B];
    __shared__ unsigned long long s_xmax;
    __shared__ int64_t s_pos[kThreads];  // positions of the chunk that have a leaf to slice
    __shared__ int32_t s_slot[kThreads];
    __shared__ int s_wcount[kThreads / 32];
    if (stop && *stop) return;  // the SP2 loop has already stopped
    const int sigma = sigma_of(*maxbits);
    if (blockIdx.x == 0 && threadIdx.x == 0 && sigma_out) *sigma_out = sigma;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // chunks of `chunk` <= kThreads leaf positions: thread t tests position
    // t of the chunk (one round trip for the whole chunk), the block then
    // slices the chunk's listed leaves one after the other
    for (int64_t base = (int64_t)blockIdx.x * chunk; base < rows * nb; base += (int64_t)gridDim.x * chunk) {
        {
            const int64_t pos = base + threadIdx.x;
            const int64_t i = pos / nb, k = pos % nb;
            // slot and norm loads issued together (the norm does not wait for the slot)
            const bool in = threadIdx.x < chunk && pos < rows * nb && i < nb;
            const int32_t sl = in ? slot[i * nb + k] : -1;
            const double nrm = in ? n2[i * P + k] : 0.0;
            // a leaf of squared norm 0 (and a padding position) takes part in
            // no product: it is never in a work item's mask (A) and never a
            // listed B leaf, so its slices are never read unmasked; skip it
            // with keep_max, also a leaf whose norm fails Eq. 4 against every
            // partner (keep_max holds the largest partner norm per row or
            // column): no kept triple uses it, so no product reads its slices
            const bool need = sl >= 0 && nrm != 0.0 &&
                              (!keep_max || keep_product(nrm, keep_max[keep_by_row ? i : k], tau2));
            const unsigned bal = __ballot_sync(0xffffffffu, need);
            if (lane == 0) s_wcount[wid] = __popc(bal);
            __syncthreads();
            int at = __popc(bal & ((1u << lane) - 1u));
            for (int q = 0; q < wid; q++) at += s_wcount[q];
            if (need) {
                s_pos[at] = pos;
                s_slot[at] = sl;
            }
        }
        __syncthreads();
        int listed = 0;
        for (int q = 0; q < kThreads / 32; q++) listed += s_wcount[q];
        for (int li = 0; li < listed; li++) {
            const int64_t pos = s_pos[li];
            const int64_t i = pos / nb, k = pos % nb;
            const int32_t sl = s_slot[li];
            if (threadIdx.x == 0) s_xmax = 0;
            __syncthreads();
            unsigned long long xmax = 0;
            const double *src = leaf + (int64_t)sl * (B * B);
            if (perleaf && perleaf_transposed) {
                double xs[kPerThread];  // all loads of the leaf issued before any is used
#pragma unroll
                for (int u = 0; u < kPerThread; u++) xs[u] = src[threadIdx.x + kThreads * u];
#pragma unroll
                for (int u = 0; u < kPerThread; u++) {
                    const int q = threadIdx.x + kThreads * u;
                    const int r = q / B, l = q % B;
                    const double x = xs[u];
                    const uint64_t X = float_split ? 0 : slice_int(x, sigma, S);
                    const bool neg = x < 0.0;
                    xmax = X > xmax ? X : xmax;
                    // outside |x| < 2^sigma (possible only with a caller-fixed scale)
                    if (!float_split && (X > (1ull << (7 * S)) || !(fabs(x) <= 1e300))) atomicExch(overflow, 1);
                    double rest = x;  // float split: s_p = round(x - s_0 - ... - s_{p-1})
                    // [p][g][cc][8 x ce], element (r, l) stored as (l, r)
                    const int o = slice_byte_offset<B, E>(l, r) / E;
#pragma unroll
                    for (int p = 0; p < S; p++) sa[p * B * B + o] = (W)slice_elem<E>(X, neg, p, S, float_split, rest);
                }
            } else {
                // untransposed: elements (r, l) and (r, l + 1), l even, are
                // neighbours in every slice, so a thread takes such pairs and
                // stores both with one shared-memory store per slice
                using W2 = typename std::conditional<E == 4, uint2, uint32_t>::type;
                constexpr int kPairs = kPerThread / 2;
                double2 xs[kPairs];  // all loads of the leaf issued before any is used
#pragma unroll
                for (int u = 0; u < kPairs; u++) xs[u] = reinterpret_cast<const double2 *>(src)[threadIdx.x + kThreads * u];
#pragma unroll
                for (int u = 0; u < kPairs; u++) {
                    const int q = 2 * (threadIdx.x + kThreads * u);
                    const int r = q / B, l = q % B;
                    const double x0 = xs[u].x, x1 = xs[u].y;
                    const uint64_t X0 = float_split ? 0 : slice_int(x0, sigma, S);
                    const uint64_t X1 = float_split ? 0 : slice_int(x1, sigma, S);
                    xmax = X0 > xmax ? X0 : xmax;
                    xmax = X1 > xmax ? X1 : xmax;
                    if (!float_split && (X0 > (1ull << (7 * S)) || X1 > (1ull << (7 * S)) || !(fabs(x0) <= 1e300) ||
                                         !(fabs(x1) <= 1e300)))
                        atomicExch(overflow, 1);
                    double rest0 = x0, rest1 = x1;
                    W2 *sp = reinterpret_cast<W2 *>(reinterpret_cast<uint8_t *>(sa) + slice_byte_offset<B, E>(r, l));
#pragma unroll
                    for (int p = 0; p < S; p++) {
                        const uint32_t v0 = slice_elem<E>(X0, x0 < 0.0, p, S, float_split, rest0);
                        const uint32_t v1 = slice_elem<E>(X1, x1 < 0.0, p, S, float_split, rest1);
                        W2 pr;
                        if constexpr (E == 4) pr = make_uint2(v0, v1);
                        else pr = (v0 & 0xFFFFu) | (v1 << 16);
                        sp[p * (B * B * E / sizeof(W2))] = pr;
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long v = __shfl_xor_sync(0xffffffffu, xmax, o);
                xmax = v > xmax ? v : xmax;
            }
            if ((threadIdx.x & 31) == 0 && xmax) atomicMax(&s_xmax, xmax);
            __syncthreads();
            if (threadIdx.x == 0 && zlead) {
                // leading zero slices: X < 2^(7 (S - z)) for every element (float
                // splits have none)
                const unsigned long long xm = s_xmax;
                const int bits = xm ? 64 - __clzll((long long)xm) : 0;
                const int z = float_split ? 0 : S - (bits + 6) / 7;
                zlead[sl] = (uint8_t)(z < 0 ? 0 : z);
            }
            const uint4 *ss = reinterpret_cast<const uint4 *>(sa);
            if (perleaf) {
                uint4 *d = reinterpret_cast<uint4 *>(perleaf + (int64_t)sl * (S * B * B * E));
#pragma unroll
                for (int q = threadIdx.x; q < S * kU4; q += kThreads) d[q] = ss[q];
            }
            if (tileA && !perleaf_transposed) {
                // tile-major: block (I, k) holds [p][L][slice] for its R rows
                const int64_t I = i / R, L = i % R;
                uint4 *d = reinterpret_cast<uint4 *>(tileA + ((I * nb + k) * S * R + L) * (int64_t)(B * B * E));
#pragma unroll
                for (int q = threadIdx.x; q < S * kU4; q += kThreads) d[(q / kU4) * (R * kU4) + (q % kU4)] = ss[q];
            }
            __syncthreads();
        }
        // (the chunk's list and counts are rewritten only after the barrier
        // that ends its last leaf, or this one when it listed none)
        __syncthreads();
    }
}

}  // namespace

// Storage for the slices of matrix m (kept across calls while s and e are
// unchanged).
int slices_alloc(spamm_mat_t m, int s, int e, bool tile_a, bool per_leaf, cudaStream_t st)
{
    if (m->b != 16 && m->b != 32 && m->b != 64) {
        spamm_set_error("tensor-core path: leaf must be 16, 32 or 64 (got %d)", m->b);
        return SPAMM_E_NOTSUP;
    }
    int rc;
    const size_t per = (size_t)s * m->b * m->b * e;  // bytes per leaf
    const int64_t R = 128 / m->b;
    const int64_t rows = ((m->nb + R - 1) / R) * R;
    if (m->sl_s != s || m->sl_e != e) {
        spamm_release(m->slA, st);
        spamm_release(m->slB, st);
        spamm_release(m->zlead, st);
        spamm_release(m->tmapA, st);
        m->tmapA = nullptr;
        m->slA = m->slB = nullptr;
        m->zlead = nullptr;
        m->sl_s = s;
        m->sl_e = e;
        m->slB_transposed = -1;
    }
    if (!m->zlead && (rc = spamm_alloc((void **)&m->zlead, m->nslots, st))) return rc;
    if (!m->scale) {
        if ((rc = spamm_alloc((void **)&m->scale, 16, st))) return rc;
        SPAMM_CK(cudaMemsetAsync(m->scale, 0, 16, st));  // max bits, sigma, overflow flag
    }
    if (tile_a && !m->slA) {
        if ((rc = spamm_alloc((void **)&m->slA, per * rows * m->nb, st))) return rc;
    }
    if (per_leaf && !m->slB) {
        if ((rc = spamm_alloc((void **)&m->slB, per * m->nslots, st))) return rc;
    }
    return SPAMM_OK;
}

namespace {

constexpr int kMaxTmaps = 7;  // box heights 1..s, s <= 7
struct TmapSet {
    CUtensorMap t[kMaxTmaps];
};

__global__ void k_store_tmaps(const __grid_constant__ TmapSet src, int count, uint4 *dst)
{
    const uint4 *w = reinterpret_cast<const uint4 *>(&src.t[0]);
    for (int i = threadIdx.x; i < count * (int)(sizeof(CUtensorMap) / 16); i += blockDim.x) dst[i] = w[i];
}

}  // namespace

// The tile-major array as a 5-D tensor of 8-byte words: (word of a chunk of
// at most 2 KB, chunk of a slice, leaf L of the tile, slice q, block I nb + k),
// strides 8 B, chunk, slice, R slices, s R slices.  Map h - 1 has the box
// {chunk, chunks, 1, h, 1}: the slices q0 .. q0 + h - 1 of one leaf, which
// land in shared memory one after another, as the B operand wants them.
int slices_tmaps(spamm_mat_t m, cudaStream_t st)
{
    if (m->tmapA) return SPAMM_OK;
    const int S = m->sl_s, b = m->b, R = 128 / b;
    if (!m->slA || S < 1 || S > kMaxTmaps) {
        spamm_set_error("slices_tmaps: no tile-major slices (or %d slices) to map", S);
        return SPAMM_E_INVAL;
    }
    const uint64_t slice = (uint64_t)b * b * m->sl_e, words = slice / 8;
    const uint64_t c0 = words < 256 ? words : 256, nch = words / c0;
    const int64_t nI = (m->nb + R - 1) / R;
    cuuint64_t dim[5] = {(cuuint64_t)c0, (cuuint64_t)nch, (cuuint64_t)R, (cuuint64_t)S, (cuuint64_t)(nI * m->nb)};
    cuuint64_t stride[4] = {(cuuint64_t)(c0 * 8), (cuuint64_t)slice, (cuuint64_t)(slice * R),
                            (cuuint64_t)(slice * R * S)};
    cuuint32_t elem[5] = {1, 1, 1, 1, 1};
    // the driver's encoder, looked up through the runtime (the library does
    // not link the driver library directly)
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            spamm_set_error("cuTensorMapEncodeTiled is not available from the driver");
            return SPAMM_E_CUDA;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    TmapSet set;
    memset(&set, 0, sizeof(set));
    for (int h = 1; h <= S; h++) {
        cuuint32_t box[5] = {(cuuint32_t)c0, (cuuint32_t)nch, 1, (cuuint32_t)h, 1};
        const CUresult r = encode(&set.t[h - 1], CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, m->slA, dim,
                                                  stride, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            spamm_set_error("cuTensorMapEncodeTiled failed (%d) for the B-role view of the slices", (int)r);
            return SPAMM_E_CUDA;
        }
    }
    void *d = nullptr;
    if (int rc = spamm_alloc(&d, sizeof(CUtensorMap) * S, st)) return rc;
    k_store_tmaps<<<1, 64, 0, st>>>(set, S, reinterpret_cast<uint4 *>(d));
    SPAMM_CK_LAUNCH();
    m->tmapA = d;
    return SPAMM_OK;
}

namespace {

template <int S, int E, int B>
void slice_launch(unsigned grid, int chunk, cudaStream_t st, const int32_t *stop, spamm_mat_t m, int64_t rows,
                  unsigned long long *mx, int32_t *sig, uint8_t *ta, uint8_t *pl, int tr, uint8_t *zl,
                  int float_split, const double *keep_max, int keep_by_row, double tau2)
{
    k_slice<S, E, B><<<grid, kSliceThreads, 0, st>>>(stop, m->leaf, m->slot, m->n2 + tier_offset(m->depth), m->P, m->nb,
                                           rows, mx, sig, ta, pl, tr, zl, sig + 1, float_split, chunk, keep_max,
                                           keep_by_row, tau2);
}

template <int B>
bool slice_dispatch_b(int s, int e, unsigned grid, int chunk, cudaStream_t st, const int32_t *stop, spamm_mat_t m,
                      int64_t rows, unsigned long long *mx, int32_t *sig, uint8_t *ta, uint8_t *pl, int tr,
                      uint8_t *zl, int fs, const double *km, int kr, double tau2)
{
#define SPAMM_SLICE_CASE(SS, EE)                                              \
    if (s == SS && e == EE && SS * B <= 256) {                                \
        slice_launch<SS, EE, B>(grid, chunk, st, stop, m, rows, mx, sig, ta, pl, tr, zl, fs, km, kr, tau2); \
        return true;                                                          \
    }
    SPAMM_SLICE_CASE(1, 2)
    SPAMM_SLICE_CASE(2, 2)
    SPAMM_SLICE_CASE(3, 2)
    SPAMM_SLICE_CASE(4, 2)
    SPAMM_SLICE_CASE(5, 2)
    SPAMM_SLICE_CASE(6, 2)
    SPAMM_SLICE_CASE(7, 2)
    SPAMM_SLICE_CASE(1, 4)
    SPAMM_SLICE_CASE(2, 4)
#undef SPAMM_SLICE_CASE
    return false;
}

}  // namespace

// Slices of matrix m: `tile_a` asks for the tile-major A-operand array,
// `per_leaf` for the per-leaf array (transposed = B-operand layout).  A matrix
// that serves as both operands of a non-symmetric product needs the A array
// and the transposed per-leaf array; a symmetric product uses the untransposed
// per-leaf array of the transpose leaf as its B operand.
int launch_slices(spamm_mat_t m, int s, int e, bool tile_a, bool per_leaf, bool transposed, cudaStream_t st,
                  const int32_t *stop, bool unit_scale, bool float_split, const double *keep_a,
                  const double *keep_b, double tau2)
{
    int rc = slices_alloc(m, s, e, tile_a, per_leaf, st);
    if (rc) return rc;
    if (e == 4 && !float_split) {
        spamm_set_error("TF32 slices are float splits only");
        return SPAMM_E_NOTSUP;
    }
    const int64_t R = 128 / m->b;
    const int64_t rows = ((m->nb + R - 1) / R) * R;
    const int64_t count = m->nslots * m->b * m->b;
    const int blocks = spamm_num_sms() * 8;
    // the scale matters to exact slices only: float splits take no maximum;
    // a fixed unit scale is written once and kept while it stays in force
    if (unit_scale || float_split) {
        if (!m->scale_unit) {
            k_unit_scale<<<1, 1, 0, st>>>(nullptr, reinterpret_cast<unsigned long long *>(m->scale));
            SPAMM_CK_LAUNCH();
            m->scale_unit = true;
        }
    } else {
        SPAMM_CK(cudaMemsetAsync(m->scale, 0, sizeof(unsigned long long), st));  // max bits
        k_absmax<<<blocks, 256, 0, st>>>(stop, m->leaf, count, reinterpret_cast<unsigned long long *>(m->scale));
        SPAMM_CK_LAUNCH();
        m->scale_unit = false;
    }
    unsigned long long *mx = reinterpret_cast<unsigned long long *>(m->scale);
    int32_t *sig = reinterpret_cast<int32_t *>(m->scale + 1);
    const int64_t npos = rows * m->nb;
    // positions a block tests at once: up to kSliceThreads, fewer when that
    // would leave the GPU with too few blocks (about 16 per SM)
    int64_t chunk = npos / ((int64_t)spamm_num_sms() * 16);
    chunk = chunk < 1 ? 1 : (chunk > kSliceThreads ? kSliceThreads : chunk);
    const int64_t chunks = (npos + chunk - 1) / chunk;
    const unsigned grid = (unsigned)(chunks < 65535 * 4 ? chunks : 65535 * 4);
    // the tile-major array and a transposed per-leaf array need two passes
    const int passes = (tile_a && per_leaf && transposed) ? 2 : 1;
    for (int pass = 0; pass < passes; pass++) {
        uint8_t *ta = (tile_a && pass == 0) ? m->slA : nullptr;
        uint8_t *pl = (per_leaf && (passes == 1 || pass == 1)) ? m->slB : nullptr;
        const int tr = pl && transposed ? 1 : 0;
        uint8_t *zl = pass == 0 ? m->zlead : nullptr;
        const int fs = float_split ? 1 : 0;
        // leaves no product of this call uses are skipped: the tile-major
        // (A-role) pass tests against keep_a per column, the per-leaf
        // (B-role) pass against keep_b per row; a pass writing both arrays
        // skips nothing
        const double *km = (ta && pl) ? nullptr : ta ? keep_a : keep_b;
        const int kr = ta ? 0 : 1;
        bool ok = false;
        switch (m->b) {
        case 16: ok = slice_dispatch_b<16>(s, e, grid, (int)chunk, st, stop, m, rows, mx, sig, ta, pl, tr, zl, fs, km, kr,
                                            tau2);
            break;
        case 32: ok = slice_dispatch_b<32>(s, e, grid, (int)chunk, st, stop, m, rows, mx, sig, ta, pl, tr, zl, fs, km, kr,
                                            tau2);
            break;
        case 64: ok = slice_dispatch_b<64>(s, e, grid, (int)chunk, st, stop, m, rows, mx, sig, ta, pl, tr, zl, fs, km, kr,
                                            tau2);
            break;
        }
        if (!ok) {
            spamm_set_error("slices: %d slices of %d-byte elements at leaf %d not built", s, e, m->b);
            return SPAMM_E_NOTSUP;
        }
        SPAMM_CK_LAUNCH();
    }
    if (per_leaf) m->slB_transposed = transposed ? 1 : 0;
    return SPAMM_OK;
}
