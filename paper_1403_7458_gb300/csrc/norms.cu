// norms.cu -- the norm quadtree (Sec. 2, Eqs. 1-3).
//
// Leaf tier: one warp per leaf reads the b x b FP64 block (coalesced, 16-byte
// loads; once, kept in registers, for b <= 32), finds the largest exponent,
// and accumulates the squares in 128-bit fixed point (order-independent, see
// internal.cuh).  The squared norm
// is rounded once and written to the leaf grid and to its transpose.
// Upper tiers: each parent is the once-rounded exact sum of its four children
// (Eq. 3, squared); one kernel per group of up to five tiers.
//
// Roofline: HBM-bound; algorithmic bytes per leaf = 8 b^2 read (+16 B norms).
#include "internal.cuh"

namespace {

constexpr int kWarpsPerBlock = 8;

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_leaf_norms(const double *__restrict__ leaf, const int32_t *__restrict__ slot, int64_t nb,
             int64_t P, int bb, double *__restrict__ n2, double *__restrict__ n2T)
{
    int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (w >= P * P) return;
    int64_t I = w / P, K = w % P;
    double r = 0.0;
    int32_t s = (I < nb && K < nb) ? slot[I * nb + K] : -1;
    if (s >= 0) {
        const double2 *src = reinterpret_cast<const double2 *>(leaf + (int64_t)s * bb);
        int nv = bb >> 1;
        int emax = 0;
#pragma unroll 4
        for (int q = lane; q < nv; q += 32) {
            double2 v = __ldg(src + q);
            emax = max(emax, max(exp_key(v.x), exp_key(v.y)));
        }
        emax = warp_max_int(emax);
        u128 acc = 0;
        if (emax > 0) {
#pragma unroll 4
            for (int q = lane; q < nv; q += 32) {
                double2 v = __ldg(src + q);
                acc += sq_term(v.x, emax) + sq_term(v.y, emax);
            }
            acc = warp_sum_u128(acc);
            r = sq_sum_round(acc, emax);
        }
    }
    if (lane == 0) {
        n2[I * P + K] = r;
        n2T[K * P + I] = r;
    }
}

// The same for leaves of up to 32 x 32: each lane keeps its b^2 / 32 values
// in registers between the exponent pass and the accumulation, so every
// leaf is read from memory once.
template <int B>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 2)
k_leaf_norms_reg(const double *__restrict__ leaf, const int32_t *__restrict__ slot, int64_t nb, int64_t P,
                 double *__restrict__ n2, double *__restrict__ n2T)
{
    constexpr int NV = B * B / 64;  // 16-byte loads per lane
    static_assert(NV >= 1 && B * B % 64 == 0, "leaf too small");
    const int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= P * P) return;
    const int64_t I = w / P, K = w % P;
    double r = 0.0;
    const int32_t s = (I < nb && K < nb) ? slot[I * nb + K] : -1;
    if (s >= 0) {  // warp-uniform
        const double2 *src = reinterpret_cast<const double2 *>(leaf + (int64_t)s * (B * B));
        double2 v[NV];
#pragma unroll
        for (int u = 0; u < NV; u++) v[u] = __ldg(src + lane + 32 * u);
        int emax = 0;
#pragma unroll
        for (int u = 0; u < NV; u++) emax = max(emax, max(exp_key(v[u].x), exp_key(v[u].y)));
        emax = warp_max_int(emax);
        if (emax > 0) {
            u128 acc = 0;
#pragma unroll
            for (int u = 0; u < NV; u++) acc += sq_term(v[u].x, emax) + sq_term(v[u].y, emax);
            acc = warp_sum_u128(acc);
            r = sq_sum_round(acc, emax);
        }
    }
    if (lane == 0) {
        n2[I * P + K] = r;
        n2T[K * P + I] = r;
    }
}

// One block per 32 x 32 square of tier `t0` (or the whole tier if smaller);
// reduces up to `levels` tiers in shared memory.
__global__ void __launch_bounds__(256)
k_pyramid(double *__restrict__ tiers, int t0, int levels)
{
    __shared__ double buf[32 * 32];
    __shared__ double nxt[16 * 16];
    int W0 = 1 << t0;
    int side = W0 < 32 ? W0 : 32;
    int bx = blockIdx.x % (W0 / side), by = blockIdx.x / (W0 / side);
    const double *src = tiers + tier_offset(t0);
    for (int q = threadIdx.x; q < side * side; q += blockDim.x) {
        int r = q / side, c = q % side;
        buf[q] = src[(int64_t)(by * side + r) * W0 + bx * side + c];
    }
    __syncthreads();
    int cur = side;
    for (int lv = 1; lv <= levels && cur > 1; lv++) {
        int half = cur >> 1;
        int t = t0 - lv;
        int Wt = 1 << t;
        double *dst = tiers + tier_offset(t);
        for (int q = threadIdx.x; q < half * half; q += blockDim.x) {
            int r = q / half, c = q % half;
            double v[4] = {buf[(2 * r) * cur + 2 * c], buf[(2 * r) * cur + 2 * c + 1],
                           buf[(2 * r + 1) * cur + 2 * c], buf[(2 * r + 1) * cur + 2 * c + 1]};
            int emax = 0;
            for (int u = 0; u < 4; u++) emax = max(emax, exp_key(v[u]));
            double out = 0.0;
            if (emax > 0) {
                u128 acc = 0;
                for (int u = 0; u < 4; u++) acc += val_term(v[u], emax);
                out = val_sum_round(acc, emax);
            }
            nxt[q] = out;
            dst[(int64_t)(by * half + r) * Wt + bx * half + c] = out;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < half * half; q += blockDim.x) buf[q] = nxt[q];
        __syncthreads();
        cur = half;
    }
}

}  // namespace

int launch_leaf_norms(spamm_mat_t m, cudaStream_t s)
{
    int64_t leaves = m->P * m->P;
    int64_t blocks = (leaves + kWarpsPerBlock - 1) / kWarpsPerBlock;
    double *n2 = m->n2 + tier_offset(m->depth);
    if (m->b == 16)
        k_leaf_norms_reg<16><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(m->leaf, m->slot, m->nb, m->P, n2,
                                                                               m->n2T);
    else if (m->b == 32)
        k_leaf_norms_reg<32><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(m->leaf, m->slot, m->nb, m->P, n2,
                                                                               m->n2T);
    else  // 64 x 64 leaves: 128 values per lane would not stay in registers; two reads
        k_leaf_norms<<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(m->leaf, m->slot, m->nb, m->P, m->b * m->b,
                                                                      n2, m->n2T);
    SPAMM_CK_LAUNCH();
    return launch_pyramid(m, s);
}

int launch_pyramid(spamm_mat_t m, cudaStream_t s)
{
    int t = m->depth;
    while (t > 0) {
        int W = 1 << t;
        int side = W < 32 ? W : 32;
        int levels = 0;
        while ((side >> levels) > 1 && levels < t) levels++;
        int blocks = (W / side) * (W / side);
        k_pyramid<<<blocks, 256, 0, s>>>(m->n2, t, levels);
        SPAMM_CK_LAUNCH();
        t -= levels;
    }
    return SPAMM_OK;
}
