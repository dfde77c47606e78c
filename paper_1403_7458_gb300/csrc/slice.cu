// slice.cu -- exact integer slices of FP64 leaves for the tensor-core path.
//
// Every element x of a matrix is scaled by the matrix's global power of two
// 2^-sigma (sigma chosen so that max|x| < 2^sigma), rounded to the integer
// X = round(|x| 2^(7s - sigma)) <= 2^(7s), and cut into s base-128 digits,
//     X = sum_p d_p 128^(s-1-p),  d_0 in [0, 128], d_p in [0, 127] (p > 0),
// each carrying the sign of x.  Digits are integers of at most 8 bits, so
// BF16 holds them exactly, their pairwise products are exact in FP32, and
// sums of such products stay exact while they are below 2^24.
// (Error-free splitting after Ozaki, Ogita, Oishi and Rump, 2012.)
//
// Two layouts per leaf (b = 32, 2s KB each), both slice-major and made of
// 8 x 8 "core matrices" of BF16 (16-byte rows) as the tcgen05 K-major
// operand wants; slice p occupies bytes [2048 p, 2048 (p + 1)):
//   A role : [p][g = r/8][cc = l/8][8 x 8]   rows r of the leaf, K = columns l
//   B role : [q][g = c/8][cc = l/8][8 x 8]   N = columns c, K = rows l
// The B-role image of leaf (k, j) equals the A-role image of its transpose,
// so for a symmetric matrix the A-role array serves both operands.
//
// Per leaf the number z of leading all-zero slices (every digit d_p, p < z,
// is 0) is recorded: slice pairs touching them contribute exactly nothing.
//
// Roofline: HBM-bound; per element 8 B read, 4s B written (both roles).
#include <cuda_bf16.h>

#include "internal.cuh"

namespace {

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

template <int S>
__global__ void __launch_bounds__(256)
k_slice(const int32_t *__restrict__ stop, const double *__restrict__ leaf, const int32_t *__restrict__ slot,
        int64_t nb, int64_t rows,
        const unsigned long long *__restrict__ maxbits, int32_t *__restrict__ sigma_out,
        uint16_t *__restrict__ tileA, uint16_t *__restrict__ perleaf, int perleaf_transposed,
        uint8_t *__restrict__ zlead, int32_t *__restrict__ overflow, int float_split)
{
    constexpr int B = 32;
    __shared__ __align__(16) uint16_t sa[S * 1024];
    __shared__ unsigned long long s_xmax;
    if (stop && *stop) return;  // the SP2 loop has already stopped
    const int sigma = sigma_of(*maxbits);
    if (blockIdx.x == 0 && threadIdx.x == 0 && sigma_out) *sigma_out = sigma;
    // positions (i, k) over rows = 4 * ceil(nb / 4) padded leaf rows
    for (int64_t pos = blockIdx.x; pos < rows * nb; pos += gridDim.x) {
        const int64_t i = pos / nb, k = pos % nb;
        const int32_t sl = i < nb ? slot[i * nb + k] : -1;
        if (threadIdx.x == 0) s_xmax = 0;
        __syncthreads();
        unsigned long long xmax = 0;
        const double *src = leaf + (int64_t)(sl < 0 ? 0 : sl) * (B * B);
        for (int q = threadIdx.x; q < B * B; q += blockDim.x) {
            const int r = q / B, l = q % B;
            const double x = sl >= 0 ? src[q] : 0.0;
            const uint64_t X = float_split ? 0 : slice_int(x, sigma, S);
            const bool neg = x < 0.0;
            xmax = X > xmax ? X : xmax;
            // outside |x| < 2^sigma (possible only with a caller-fixed scale)
            if (!float_split && (X > (1ull << (7 * S)) || !(fabs(x) <= 1e300))) atomicExch(overflow, 1);
            double rest = x;  // float split: s_p = bf16(x - s_0 - ... - s_{p-1})
#pragma unroll
            for (int p = 0; p < S; p++) {
                uint16_t h;
                if (float_split) {
                    const __nv_bfloat16 t = __double2bfloat16(rest);
                    h = __bfloat16_as_ushort(t);
                    rest -= (double)__bfloat162float(t);
                } else {
                    h = slice_digit_bf16(X, neg, p, S);
                }
                // [p][g][cc][8 x 8]; transposed: element (r, l) stored as (l, r)
                if (!perleaf_transposed || !perleaf)
                    sa[p * 1024 + slice_offset(r, l)] = h;
                else
                    sa[p * 1024 + slice_offset(l, r)] = h;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, xmax, o);
            xmax = v > xmax ? v : xmax;
        }
        if ((threadIdx.x & 31) == 0 && xmax) atomicMax(&s_xmax, xmax);
        __syncthreads();
        if (threadIdx.x == 0 && zlead && sl >= 0) {
            // leading zero slices: X < 2^(7 (S - z)) for every element (float
            // splits have none)
            const unsigned long long xm = s_xmax;
            const int bits = xm ? 64 - __clzll((long long)xm) : 0;
            const int z = float_split ? 0 : S - (bits + 6) / 7;
            zlead[sl] = (uint8_t)(z < 0 ? 0 : z);
        }
        const uint4 *ss = reinterpret_cast<const uint4 *>(sa);
        if (perleaf && sl >= 0) {
            uint4 *d = reinterpret_cast<uint4 *>(perleaf + (int64_t)sl * (S * 1024));
            for (int q = threadIdx.x; q < S * 128; q += blockDim.x) d[q] = ss[q];
        }
        if (tileA && !perleaf_transposed) {
            // tile-major: block (I, k) holds [p][L][2 KB] for its four rows
            const int64_t I = i >> 2, L = i & 3;
            uint4 *d = reinterpret_cast<uint4 *>(tileA + ((I * nb + k) * S * 4 + L) * 1024);
            for (int q = threadIdx.x; q < S * 128; q += blockDim.x) d[(q >> 7) * 512 + (q & 127)] = ss[q];
        }
        __syncthreads();
    }
}

}  // namespace

// Storage for the slices of matrix m (kept across calls while s is unchanged).
int slices_alloc(spamm_mat_t m, int s, bool tile_a, bool per_leaf, cudaStream_t st)
{
    if (m->b != 32) {
        spamm_set_error("tensor-core path is built for leaf 32 (got %d)", m->b);
        return SPAMM_E_NOTSUP;
    }
    int rc;
    const size_t per = (size_t)s * 1024;  // BF16 elements per leaf
    const int64_t rows = ((m->nb + 3) / 4) * 4;
    if (m->sl_s != s) {
        spamm_release(m->slA, st);
        spamm_release(m->slB, st);
        spamm_release(m->zlead, st);
        m->slA = m->slB = nullptr;
        m->zlead = nullptr;
        m->sl_s = s;
        m->slB_transposed = -1;
    }
    if (!m->zlead && (rc = spamm_alloc((void **)&m->zlead, m->nslots, st))) return rc;
    if (!m->scale) {
        if ((rc = spamm_alloc((void **)&m->scale, 16, st))) return rc;
        SPAMM_CK(cudaMemsetAsync(m->scale, 0, 16, st));  // max bits, sigma, overflow flag
    }
    if (tile_a && !m->slA) {
        if ((rc = spamm_alloc((void **)&m->slA, sizeof(uint16_t) * per * rows * m->nb, st))) return rc;
    }
    if (per_leaf && !m->slB) {
        if ((rc = spamm_alloc((void **)&m->slB, sizeof(uint16_t) * per * m->nslots, st))) return rc;
    }
    return SPAMM_OK;
}

// Slices of matrix m: `tile_a` asks for the tile-major A-operand array,
// `per_leaf` for the per-leaf array (transposed = B-operand layout).  A matrix
// that serves as both operands of a non-symmetric product needs the A array
// and the transposed per-leaf array; a symmetric product uses the untransposed
// per-leaf array of the transpose leaf as its B operand.
int launch_slices(spamm_mat_t m, int s, bool tile_a, bool per_leaf, bool transposed, cudaStream_t st,
                  const int32_t *stop, bool unit_scale, bool float_split)
{
    if (m->b != 32) {
        spamm_set_error("tensor-core path is built for leaf 32 (got %d)", m->b);
        return SPAMM_E_NOTSUP;
    }
    int rc = slices_alloc(m, s, tile_a, per_leaf, st);
    if (rc) return rc;
    const int64_t rows = ((m->nb + 3) / 4) * 4;
    SPAMM_CK(cudaMemsetAsync(m->scale, 0, sizeof(unsigned long long), st));  // max bits
    const int64_t count = m->nslots * 1024;
    const int blocks = spamm_num_sms() * 8;
    if (unit_scale)
        k_unit_scale<<<1, 1, 0, st>>>(stop, reinterpret_cast<unsigned long long *>(m->scale));
    else
        k_absmax<<<blocks, 256, 0, st>>>(stop, m->leaf, count, reinterpret_cast<unsigned long long *>(m->scale));
    SPAMM_CK_LAUNCH();
    unsigned long long *mx = reinterpret_cast<unsigned long long *>(m->scale);
    int32_t *sig = reinterpret_cast<int32_t *>(m->scale + 1);
    const int64_t npos = rows * m->nb;
    const unsigned grid = (unsigned)(npos < 65535 * 4 ? npos : 65535 * 4);
    // the tile-major array and a transposed per-leaf array need two passes
    const int passes = (tile_a && per_leaf && transposed) ? 2 : 1;
    for (int pass = 0; pass < passes; pass++) {
        uint16_t *ta = (tile_a && pass == 0) ? m->slA : nullptr;
        uint16_t *pl = (per_leaf && (passes == 1 || pass == 1)) ? m->slB : nullptr;
        const int tr = pl && transposed ? 1 : 0;
        uint8_t *zl = pass == 0 ? m->zlead : nullptr;
#define SPAMM_SLICE_CASE(SS)                                                                          \
    case SS:                                                                                          \
        k_slice<SS><<<grid, 256, 0, st>>>(stop, m->leaf, m->slot, m->nb, rows, mx, sig, ta, pl, tr, zl,    \
                                          sig + 1, float_split ? 1 : 0);                               \
        break;
        switch (s) {
            SPAMM_SLICE_CASE(1)
            SPAMM_SLICE_CASE(2)
            SPAMM_SLICE_CASE(3)
            SPAMM_SLICE_CASE(4)
            SPAMM_SLICE_CASE(5)
            SPAMM_SLICE_CASE(6)
            SPAMM_SLICE_CASE(7)
        default:
            spamm_set_error("slices must be in 3..7 (got %d)", s);
            return SPAMM_E_INVAL;
        }
#undef SPAMM_SLICE_CASE
        SPAMM_CK_LAUNCH();
    }
    if (per_leaf) m->slB_transposed = transposed ? 1 : 0;
    return SPAMM_OK;
}
