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
// Two layouts per leaf (b = 32, 2s KB each), both made of 8 x 8 "core
// matrices" of BF16 (16-byte rows) as the tcgen05 K-major operand wants:
//   A role : [g = r/8][p][cc = l/8][8 x 8]   rows r of the leaf, K = columns l
//   B role : [q][g = c/8][cc = l/8][8 x 8]   N = columns c, K = rows l
// so that a stage of four A leaves has a uniform 8-row stride of s*512 bytes
// for every slice p, and B slices 0..s-1-p are one contiguous N-prefix.
//
// Roofline: HBM-bound; per element 8 B read, 4s B written (both roles).
#include "internal.cuh"

namespace {

// max |x| over the stored leaves, as the IEEE bit pattern (monotone for
// non-negative doubles), by integer atomicMax: exact and order-free.
__global__ void k_absmax(const double *__restrict__ leaf, int64_t count,
                         unsigned long long *__restrict__ out)
{
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
k_slice(const double *__restrict__ leaf, int64_t nslots, const unsigned long long *__restrict__ maxbits,
        int32_t *__restrict__ sigma_out, uint16_t *__restrict__ slA, uint16_t *__restrict__ slB)
{
    constexpr int B = 32;
    __shared__ __align__(16) uint16_t sa[S * 1024];
    __shared__ __align__(16) uint16_t sb[S * 1024];
    const int sigma = sigma_of(*maxbits);
    if (blockIdx.x == 0 && threadIdx.x == 0 && sigma_out) *sigma_out = sigma;
    for (int64_t slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
        const double *src = leaf + slot * (B * B);
        for (int q = threadIdx.x; q < B * B; q += blockDim.x) {
            const int r = q / B, l = q % B;
            uint64_t m;
            int e;
            const double x = src[q];
            dbl_decompose(x, m, e);
            uint64_t X = 0;
            if (m) {
                const int sh = 1075 + sigma - 7 * S - e;
                if (sh <= 0) X = m << (-sh);
                else if (sh < 64) X = (m >> sh) + ((m >> (sh - 1)) & 1ull);
            }
            const bool neg = x < 0.0;
#pragma unroll
            for (int p = 0; p < S; p++) {
                uint32_t d = (uint32_t)(X >> (7 * (S - 1 - p)));
                if (p > 0) d &= 127u;
                // integer d <= 128 -> BF16 bits (exact): via float
                float f = neg ? -(float)d : (float)d;
                uint16_t h = (uint16_t)(__float_as_uint(f) >> 16);
                // A role: [g][p][cc][ri][li]
                sa[((r >> 3) * S + p) * 256 + (l >> 3) * 64 + (r & 7) * 8 + (l & 7)] = h;
                // B role: element (row r = K index, column l = N index)
                sb[(p * 4 + (l >> 3)) * 256 + (r >> 3) * 64 + (l & 7) * 8 + (r & 7)] = h;
            }
        }
        __syncthreads();
        uint4 *da = reinterpret_cast<uint4 *>(slA + slot * (S * 1024));
        uint4 *db = reinterpret_cast<uint4 *>(slB + slot * (S * 1024));
        const uint4 *ssa = reinterpret_cast<const uint4 *>(sa);
        const uint4 *ssb = reinterpret_cast<const uint4 *>(sb);
        for (int q = threadIdx.x; q < S * 1024 / 8; q += blockDim.x) {
            if (slA) da[q] = ssa[q];
            if (slB) db[q] = ssb[q];
        }
        __syncthreads();
    }
}

}  // namespace

int launch_slices(spamm_mat_t m, int s, cudaStream_t st)
{
    if (m->b != 32) {
        spamm_set_error("tensor-core path is built for leaf 32 (got %d)", m->b);
        return SPAMM_E_NOTSUP;
    }
    int rc;
    const size_t per = (size_t)s * 1024;  // BF16 elements per leaf per role
    if (!m->slA || m->sl_s != s) {
        spamm_release(m->slA, st);
        spamm_release(m->slB, st);
        m->slA = m->slB = nullptr;
        if ((rc = spamm_alloc((void **)&m->slA, sizeof(uint16_t) * per * m->nslots, st))) return rc;
        if ((rc = spamm_alloc((void **)&m->slB, sizeof(uint16_t) * per * m->nslots, st))) return rc;
        if (!m->scale) {
            if ((rc = spamm_alloc((void **)&m->scale, 16, st))) return rc;
        }
        m->sl_s = s;
    }
    SPAMM_CK(cudaMemsetAsync(m->scale, 0, sizeof(unsigned long long), st));
    const int64_t count = m->nslots * 1024;
    int blocks = spamm_num_sms() * 8;
    k_absmax<<<blocks, 256, 0, st>>>(m->leaf, count, reinterpret_cast<unsigned long long *>(m->scale));
    SPAMM_CK_LAUNCH();
    unsigned long long *mx = reinterpret_cast<unsigned long long *>(m->scale);
    int32_t *sig = reinterpret_cast<int32_t *>(m->scale + 1);
    unsigned grid = (unsigned)(m->nslots < 65535 * 4 ? m->nslots : 65535 * 4);
    switch (s) {
    case 3: k_slice<3><<<grid, 256, 0, st>>>(m->leaf, m->nslots, mx, sig, m->slA, m->slB); break;
    case 4: k_slice<4><<<grid, 256, 0, st>>>(m->leaf, m->nslots, mx, sig, m->slA, m->slB); break;
    case 5: k_slice<5><<<grid, 256, 0, st>>>(m->leaf, m->nslots, mx, sig, m->slA, m->slB); break;
    case 6: k_slice<6><<<grid, 256, 0, st>>>(m->leaf, m->nslots, mx, sig, m->slA, m->slB); break;
    case 7: k_slice<7><<<grid, 256, 0, st>>>(m->leaf, m->nslots, mx, sig, m->slA, m->slB); break;
    default:
        spamm_set_error("slices must be in 3..7 (got %d)", s);
        return SPAMM_E_INVAL;
    }
    SPAMM_CK_LAUNCH();
    return SPAMM_OK;
}
