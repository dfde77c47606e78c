// sp2.cu -- the SP2 spectral projection loop (Niklasson 2002, the solver the
// paper drives with SpAMM in Sec. 4).
//
// Per solve:
//   gershgorin : one thread per matrix row sums |f_ij| (j != i) in column
//                order (chunked vector loads, the next chunk in flight while
//                the current one is summed); a one-block kernel takes
//                min / max of f_ii -/+ sum;
//   x0         : X0 = (emax I - F) / (emax - emin), fused with X0's leaf norms
//                and its trace.
// Per iteration (all on the device; the host enqueues iterations in batches
// and reads the state once per batch):
//   cull + leaf products : X2 = SpAMM(X, X, tau), diagonal leaves also emit
//                          their traces;
//   decide               : one block sums those traces in a fixed order and
//                          picks X2 or 2X - X2;
//   update               : one warp per leaf writes the new X in place, its
//                          exact squared norm, the partial ||X2 - X||_F^2 and
//                          the diagonal traces; the last block to finish
//                          reduces the partials in a fixed order, records the
//                          iteration's history row and applies the stopping
//                          rule; once it stops, every later kernel of the
//                          batch returns at once.
// Every reduction has a fixed order, so two runs give identical bits.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace {

struct Sp2State {
    double emin, emax;
    double t1;       // tr X
    double t2;       // tr X^2
    double e;        // ||X^2 - X||_F
    double tn;       // tr of the updated X
    int64_t tasks;   // surviving triples of this iteration's product
    int32_t branch;  // 1: X <- X^2
    int32_t done;    // last-block ticket
    int32_t stopped; // set by the stopping rule; later kernels return at once
    int32_t reason;  // SP2_STOP_*
    int32_t iter;    // iterations completed
    int32_t pad;
    double ehist[3]; // e of the last three iterations
    int64_t units;   // tensor path: slice pairs of surviving triples, summed
    unsigned long long nonzero;  // leaves of the updated X with nonzero norm
};

// Stopping rule parameters (same rule as the host-side description in spamm.h)
struct Sp2Rule {
    double Ne, trace_tol, idem_tol;
    int32_t fixed_iters, max_iter;
};

constexpr int kEwWarps = 8;        // elementwise pass: warps per block (one leaf per warp at a time)
constexpr int kEwBlocksPerSm = 4;  // and resident blocks per SM (register cap 64: more leaves in flight)
constexpr int kRedThreads = 1024;
constexpr int kBatch = 4;  // SP2 iterations enqueued between reads of the state

// Row sums of |f_ij| (j != i) in column order, one thread per matrix row
// (the same order as the plain sequential sum, so the bounds are bit-equal
// to it).  The row's segment of each stored leaf is read in chunks of up to
// 32 values with vector loads, and the next chunk's loads are issued before
// the current chunk is summed, so that many loads are in flight per thread
// (the kernel streams every stored leaf of F once: HBM-bound).  Absent
// leaves are zero and skipped (adding +0 leaves the sum unchanged).
template <int B>
__global__ void __launch_bounds__(128)
k_gershgorin_rows(const double *__restrict__ leaf, const int32_t *__restrict__ slot, int64_t n, int64_t nb,
                  double *__restrict__ lo, double *__restrict__ hi)
{
    constexpr int CH = B < 32 ? B : 32;  // values per chunk
    constexpr int NCH = B / CH;          // chunks per leaf row segment
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t I = r / B;
    const int rr = (int)(r % B);
    const int32_t *srow = slot + I * nb;
    auto next_stored = [&](int64_t K) {
        while (K < nb && __ldg(srow + K) < 0) K++;
        return K;
    };
    auto load = [&](int64_t K, int h, double2 (&v)[CH / 2]) {
        const double2 *p =
            reinterpret_cast<const double2 *>(leaf + (int64_t)__ldg(srow + K) * (B * B) + rr * B + h * CH);
#pragma unroll
        for (int u = 0; u < CH / 2; u++) v[u] = __ldg(p + u);
    };
    double s = 0.0, d = 0.0;
    int64_t K = next_stored(0);
    int h = 0;
    double2 cur[CH / 2], nxt[CH / 2];
    if (K < nb) load(K, 0, cur);
    while (K < nb) {
        int64_t K2 = K;
        int h2 = h + 1;
        if (h2 == NCH) {
            h2 = 0;
            K2 = next_stored(K + 1);
        }
        if (K2 < nb) load(K2, h2, nxt);
        const int64_t c0 = K * B + h * CH;
#pragma unroll
        for (int u = 0; u < CH; u++) {
            const int64_t col = c0 + u;
            const double v = (u & 1) ? cur[u >> 1].y : cur[u >> 1].x;
            if (col < n) {
                if (col == r) d = v;
                else s += fabs(v);
            }
        }
        K = K2;
        h = h2;
#pragma unroll
        for (int u = 0; u < CH / 2; u++) cur[u] = nxt[u];
    }
    lo[r] = d - s;
    hi[r] = d + s;
}

// Exact symmetry test of a leaf-stored matrix: one warp per leaf (I, K) with
// I <= K compares it with the transpose of leaf (K, I).
__global__ void k_symmetry(const double *__restrict__ leaf, const int32_t *__restrict__ slot, int64_t nb,
                           int b, int32_t *__restrict__ asym)
{
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= nb * nb) return;
    const int64_t I = w / nb, K = w % nb;
    if (I > K) return;
    const int32_t s1 = slot[I * nb + K], s2 = slot[K * nb + I];
    if ((s1 < 0) != (s2 < 0)) {
        if (lane == 0) atomicExch(asym, 1);
        return;
    }
    if (s1 < 0) return;
    const double *a = leaf + (int64_t)s1 * b * b, *t = leaf + (int64_t)s2 * b * b;
    bool bad = false;
    for (int q = lane; q < b * b; q += 32) {
        const int r = q / b, c = q % b;
        // compare bit patterns: exact equality, NaN-safe
        bad |= __double_as_longlong(a[q]) != __double_as_longlong(t[c * b + r]);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicExch(asym, 1);
}

// Cheap symmetry screen on the leaf norms: flags F when some pair of mirror
// leaves differs in squared norm by more than rel times the larger one.
__global__ void k_norm_symmetry(const double *__restrict__ n2, int64_t nb, int64_t P, double rel,
                                int32_t *__restrict__ flag)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nb * nb) return;
    const int64_t I = g / nb, K = g % nb;
    if (I >= K) return;
    const double a = n2[I * P + K], b = n2[K * P + I];
    if (fabs(a - b) > rel * fmax(a, b)) atomicExch(flag, 1);
}

__global__ void __launch_bounds__(kRedThreads)
k_gershgorin_bounds(const double *__restrict__ lo, const double *__restrict__ hi, int64_t n,
                    Sp2State *st)
{
    __shared__ double smin[kRedThreads], smax[kRedThreads];
    double a = INFINITY, z = -INFINITY;
    for (int64_t q = threadIdx.x; q < n; q += kRedThreads) {
        a = fmin(a, lo[q]);
        z = fmax(z, hi[q]);
    }
    smin[threadIdx.x] = a;
    smax[threadIdx.x] = z;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st->emin = smin[0];
        st->emax = smax[0];
        st->done = 0;
        st->stopped = 0;
        st->reason = SP2_STOP_MAXITER;
        st->iter = 0;
        st->ehist[0] = st->ehist[1] = st->ehist[2] = INFINITY;
    }
}

// Fixed-order sum of v[0..count) by one block: thread t adds v[t], v[t+T], ...
// in order, then a fixed binary tree.  Result valid in thread 0.
__device__ double block_sum_fixed(const double *v, int64_t count, double *sbuf)
{
    double a = 0.0;
    for (int64_t q = threadIdx.x; q < count; q += blockDim.x) a += __ldcg(v + q);
    sbuf[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sbuf[threadIdx.x] += sbuf[threadIdx.x + o];
        __syncthreads();
    }
    double r = sbuf[0];
    __syncthreads();
    return r;
}

// The last block to finish an elementwise pass reduces the per-leaf partials
// in a fixed order, records the iteration's history row and applies the
// stopping rule (mode 1).
__device__ void sp2_finish(int mode, const double *idem_part, int64_t idem_count, const double *diag_part,
                           int64_t nb, Sp2State *st, const Sp2Rule &rule, double *hist, double *sred, bool *s_last)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *s_last = atomicAdd(&st->done, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    double e2 = block_sum_fixed(idem_part, idem_count, sred);
    double tn = block_sum_fixed(diag_part, nb, sred);
    if (threadIdx.x == 0) {
        st->tn = tn;
        st->done = 0;
        if (mode == 1) {
            const double e = sqrt(e2);
            st->e = e;
            const int it = st->iter + 1;
            double *row = hist + (int64_t)(it - 1) * SP2_H_COLS;
            row[SP2_H_TR] = st->t1;
            row[SP2_H_TR2] = st->t2;
            row[SP2_H_IDEM] = e;
            row[SP2_H_BRANCH] = st->branch ? 1.0 : 0.0;
            row[SP2_H_TASKS] = (double)st->tasks;
            row[SP2_H_TRNEW] = tn;
            row[SP2_H_FILL] = (double)atomicAdd(&st->nonzero, 0ull) / (double)(nb * nb);
            st->ehist[0] = st->ehist[1];
            st->ehist[1] = st->ehist[2];
            st->ehist[2] = e;
            st->iter = it;
            if (rule.fixed_iters > 0) {
                if (it >= rule.fixed_iters) {
                    st->stopped = 1;
                    st->reason = SP2_STOP_FIXED;
                }
            } else if (fabs(tn - rule.Ne) < rule.trace_tol && e < rule.idem_tol) {
                st->stopped = 1;
                st->reason = SP2_STOP_CONVERGED;
            } else if (it >= 3 && e < 1e-3 && e > 0.5 * st->ehist[0]) {
                st->stopped = 1;
                st->reason = SP2_STOP_STAGNATED;
            } else if (it >= rule.max_iter) {
                st->stopped = 1;
                st->reason = SP2_STOP_MAXITER;
            }
        }
    }
}


// An FP64 value cut to FP32 (the fraction truncated to 23 bits; values
// below the FP32 normal range become 0) by integer operations alone: for the
// squares of the idempotency error, where a relative error below 2^-22 per
// term is immaterial and an FP64 multiply-add per element is not.  Values of
// magnitude 2^128 and beyond, infinities and NaNs become infinities.
__device__ __forceinline__ float f64_to_f32_trunc(double x)
{
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7FF) - 896;                 // FP32 biased exponent
    const uint32_t m = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;    // top 23 fraction bits
    if (e >= 255) return __int_as_float(0x7F800000);
    return e > 0 ? __uint_as_float((hi & 0x80000000u) | ((uint32_t)e << 23) | m) : 0.0f;
}

// Elementwise pass over all leaves of X, one warp per leaf (persistent
// warps stride over the leaves).
//   mode 0: X <- (emax I - F) / (emax - emin)          (src = F)
//   mode 1: X <- X2 if branch else 2 X - X2            (src = X2)
// In mode 1 with x2rows (the tensor path's per-tile words of X2's product,
// R leaf rows by tw leaf columns per tile, symmetric or not: bit 8 + 8 c + L
// set when leaf row L of tile column c had work), a leaf of X2 without work
// is zero and was not written: it is not read, and a leaf that is zero in
// both X (squared norm 0) and X2 stays zero without being touched.
// Writes the leaf's squared norm (exact, once rounded) and, for diagonal
// leaves, its trace.  Each warp adds the partial ||X2 - X||^2 of its leaves
// in leaf order, and the block adds its warps' sums in warp order into
// idem_part[block] (mode 1).  The last block reduces the partials and stores
// e and the new trace in the state.
// A lane handles elements lane + 32 u of the leaf, in chunks of kCh rows of
// 32 whose loads are all issued before any is used; the squares are summed
// in a second pass over the written leaf (from L2), once the leaf's largest
// exponent is known.
template <int B>
__global__ void __launch_bounds__(kEwWarps * 32, kEwBlocksPerSm)
k_sp2_elementwise(int mode, double *__restrict__ X, const double *__restrict__ src,
                  const int32_t *__restrict__ slot, const int32_t *__restrict__ src_slot, int64_t n, int64_t nb,
                  int64_t P, double *__restrict__ n2, double *__restrict__ n2T, double *__restrict__ idem_part,
                  double *__restrict__ diag_part, Sp2State *st, Sp2Rule rule, double *__restrict__ hist,
                  const int32_t *__restrict__ x2rows, int R, int tw, int sym, int tlow)
{
    constexpr int BB = B * B;
    constexpr int kPer = BB / 32;              // elements per lane
    constexpr int kCh = kPer < 8 ? kPer : 8;   // rows of 32 per chunk
    __shared__ double sred[kEwWarps * 32];
    __shared__ double s_idem[kEwWarps];
    __shared__ bool s_last;
    if (mode == 1 && *(volatile int32_t *)&st->stopped) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * kEwWarps;
    const bool take_sq = st->branch != 0;
    const double emax = st->emax, range = st->emax - st->emin;
    double idem_w = 0.0;  // lane 0: this warp's leaves, in order
    for (int64_t w = (int64_t)blockIdx.x * kEwWarps + warp; w < nb * nb; w += nwarps) {
        const int64_t I = w / nb, K = w % nb;
        double *x = X + (int64_t)slot[w] * BB;
        // the source in mode 0 is F, which may leave zero leaves unstored
        // mode 1 with tlow: X2 stores only its leaves I <= K, a lower leaf
        // is read as the transpose of leaf (K, I)
        const bool tr = mode == 1 && tlow && I > K;
        const int32_t ss = src_slot[tr ? K * nb + I : w];
        const double *y = src + (int64_t)(ss < 0 ? 0 : ss) * BB;
        const bool diag = I == K;
        bool y0 = ss < 0;  // source leaf known to be zero
        if (mode == 1 && x2rows) {
            const int64_t a = (sym && I > K) ? K : I, c = (sym && I > K) ? I : K;
            const int32_t word = x2rows[(a / R) * ((nb + tw - 1) / tw) + c / tw];
            y0 = !((word >> (8 + 8 * (c % tw) + a % R)) & 1);
        }
        // X_new = X2 or 2X - X2 = 0 with X = 0 = X2: nothing to read or write
        // (mode 0 writes every leaf of X: X0 = (emax I - F) / range)
        if (mode == 1 && y0 && n2[I * P + K] == 0.0) {  // warp-uniform
            if (lane == 0 && diag) diag_part[I] = 0.0;
            continue;
        }
        // X0 of an off-diagonal leaf that F does not store: (0 - 0) / range
        // = +0 in every element; written without the divisions
        if (mode == 0 && y0 && !diag) {  // warp-uniform
            const double2 z = make_double2(0.0, 0.0);
#pragma unroll 4
            for (int q = lane; q < BB / 2; q += 32) reinterpret_cast<double2 *>(x)[q] = z;
            if (lane == 0) {
                n2[I * P + K] = 0.0;
                n2T[K * P + I] = 0.0;
            }
            continue;
        }
        float idem = 0.0f;  // this lane's sum of d^2 over the leaf (see below)
        int ek = 0;
        // the update's kind is uniform over the launch: one loop per kind, so
        // that no FP64 operation of another kind is issued (the FP64 pipe is
        // this kernel's bottleneck)
        auto pass1 = [&](auto kind) {
            constexpr int K = decltype(kind)::value;  // 0: X0, 1: X <- X2, 2: X <- 2X - X2
#pragma unroll 1
            for (int c0 = 0; c0 < kPer; c0 += kCh) {
                double yv[kCh], xv[kCh];
#pragma unroll
                for (int u = 0; u < kCh; u++) {
                    const int q = lane + 32 * (c0 + u);
                    yv[u] = y0 ? 0.0 : y[tr ? (q % B) * B + q / B : q];
                    xv[u] = K != 0 ? x[q] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < kCh; u++) {
                    const int q = lane + 32 * (c0 + u);
                    double nv;
                    if constexpr (K == 0) {
                        // (emax [i == j] - f_ij) / range; an off-diagonal zero
                        // gives +0 (no division), a nonzero -f_ij / range
                        // (0 - f equals -f exactly for f != 0)
                        const int r = q / B;
                        if (diag && r == q % B && I * B + r < n) nv = (emax - yv[u]) / range;
                        else nv = yv[u] == 0.0 ? 0.0 : -yv[u] / range;
                    } else {
                        // d = x2 - x in FP64; d^2 summed in FP32 from d cut to
                        // FP32 by integer operations (no FP64 multiply-add:
                        // the FP64 pipe bounds this kernel)
                        const float df = f64_to_f32_trunc(yv[u] - xv[u]);
                        idem = fmaf(df, df, idem);
                        if constexpr (K == 1) nv = yv[u];
                        else nv = fma(2.0, xv[u], -yv[u]);
                    }
                    x[q] = nv;
                    ek = max(ek, exp_key(nv));
                }
            }
        };
        if (mode == 0) pass1(std::integral_constant<int, 0>());
        else if (take_sq) pass1(std::integral_constant<int, 1>());
        else pass1(std::integral_constant<int, 2>());
        ek = warp_max_int(ek);
        __syncwarp();
        u128 acc = 0;
        double dsum = 0.0;
        if (ek > 0) {
#pragma unroll 1
            for (int c0 = 0; c0 < kPer; c0 += kCh) {
                double v[kCh];
#pragma unroll
                for (int u = 0; u < kCh; u++) v[u] = x[lane + 32 * (c0 + u)];
#pragma unroll
                for (int u = 0; u < kCh; u++) acc += sq_term(v[u], ek);
            }
        }
        if (diag)
            for (int r = lane; r < B; r += 32) dsum += x[r * B + r];
        acc = warp_sum_u128(acc);
        double idem_d = (double)idem;
        for (int o = 16; o > 0; o >>= 1) {
            idem_d += __shfl_xor_sync(0xffffffffu, idem_d, o);
            dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        }
        if (lane == 0) {
            double r = ek > 0 ? sq_sum_round(acc, ek) : 0.0;
            n2[I * P + K] = r;
            n2T[K * P + I] = r;
            if (r > 0.0) atomicAdd(&st->nonzero, 1ull);  // fill statistics
            idem_w += idem_d;
            if (diag) diag_part[I] = dsum;
        }
        __syncwarp();
    }
    if (lane == 0) s_idem[warp] = idem_w;
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int q = 0; q < kEwWarps; q++) e += s_idem[q];
        idem_part[blockIdx.x] = e;
    }
    sp2_finish(mode, idem_part, gridDim.x, diag_part, nb, st, rule, hist, sred, &s_last);
}

// Blocks of the elementwise pass resident on the whole GPU at once (queried
// once per device; the grid, and so the order of the partial sums, is fixed
// for a device).
template <int B>
int64_t ew_grid_cap()
{
    static int per_sm[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    int occ = __atomic_load_n(&per_sm[dev & 63], __ATOMIC_ACQUIRE);
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sp2_elementwise<B>, kEwWarps * 32, 0) != cudaSuccess ||
            occ < 1)
            occ = 1;
        __atomic_store_n(&per_sm[dev & 63], occ, __ATOMIC_RELEASE);
    }
    return (int64_t)spamm_num_sms() * occ;
}

// Launch of the elementwise pass for leaf size b (16, 32 or 64): persistent
// blocks, as many as fit on the GPU at once (fewer when there are fewer
// leaves); idem_part needs one entry per block.
template <int B>
void launch_elementwise_b(cudaStream_t s, int mode, double *X, const double *src, const int32_t *slot,
                          const int32_t *src_slot, int64_t n, int64_t nb, int64_t P, double *n2, double *n2T,
                          double *idem_part, double *diag_part, Sp2State *st, Sp2Rule rule, double *hist,
                          const int32_t *x2rows, int R, int tw, int sym, int tlow)
{
    const int64_t cap = ew_grid_cap<B>();
    const int64_t need = (nb * nb + kEwWarps - 1) / kEwWarps;
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    k_sp2_elementwise<B><<<grid, kEwWarps * 32, 0, s>>>(mode, X, src, slot, src_slot, n, nb, P, n2, n2T, idem_part,
                                                    diag_part, st, rule, hist, x2rows, R, tw, sym, tlow);
}

void launch_elementwise(int b, cudaStream_t s, int mode, double *X, const double *src, const int32_t *slot,
                        const int32_t *src_slot, int64_t n, int64_t nb, int64_t P, double *n2, double *n2T,
                        double *idem_part, double *diag_part, Sp2State *st, Sp2Rule rule, double *hist,
                        const int32_t *x2rows, int R, int tw, int sym, int tlow = 0)
{
    if (b == 16)
        launch_elementwise_b<16>(s, mode, X, src, slot, src_slot, n, nb, P, n2, n2T, idem_part, diag_part, st,
                                 rule, hist, x2rows, R, tw, sym, tlow);
    else if (b == 32)
        launch_elementwise_b<32>(s, mode, X, src, slot, src_slot, n, nb, P, n2, n2T, idem_part, diag_part, st,
                                 rule, hist, x2rows, R, tw, sym, tlow);
    else
        launch_elementwise_b<64>(s, mode, X, src, slot, src_slot, n, nb, P, n2, n2T, idem_part, diag_part, st,
                                 rule, hist, x2rows, R, tw, sym, tlow);
}


__global__ void __launch_bounds__(kRedThreads)
k_sp2_decide(const double *__restrict__ tr_part, int64_t ntr, const int64_t *__restrict__ off_end,
             const int64_t *__restrict__ units, double Ne, int rule, Sp2State *st)
{
    __shared__ double sred[kRedThreads];
    if (*(volatile int32_t *)&st->stopped) return;
    double t2 = block_sum_fixed(tr_part, ntr, sred);  // diagonal-leaf (partial) traces
    if (threadIdx.x == 0) {
        double t1 = st->tn;
        int take;
        if (rule == SP2_RULE_TRACE_ABOVE) take = t1 > Ne;
        else take = fabs(t2 - Ne) < fabs(2.0 * t1 - t2 - Ne);
        st->t1 = t1;
        st->t2 = t2;
        st->branch = take;
        st->tasks = *off_end;
        st->nonzero = 0;  // counted again by this iteration's update
        if (units) st->units += *units;
    }
}

struct Sp2Scratch {
    Sp2State *st = nullptr;
    double *lo = nullptr, *hi = nullptr;
    double *idem_part = nullptr, *diag_part = nullptr, *tr_part = nullptr;
    double *hist = nullptr;
    int32_t *flag = nullptr;
    Sp2State *host = nullptr;
    void release(cudaStream_t s)
    {
        spamm_release(st, s);
        spamm_release(lo, s);
        spamm_release(hi, s);
        spamm_release(idem_part, s);
        spamm_release(diag_part, s);
        spamm_release(tr_part, s);
        spamm_release(flag, s);
        spamm_release(hist, s);
        if (host) cudaFreeHost(host);
    }
};

}  // namespace

extern "C" int sp2_solve(spamm_mat_t F, double Ne, double tau, const sp2_opts_t *opts,
                         spamm_mat_t *Pout, sp2_report_t *report, void *stream)
{
    if (!F || !Pout || !(Ne > 0.0) || !(Ne < (double)F->n) || !(tau >= 0.0) || tau > 1e300) {
        spamm_set_error("sp2_solve: bad arguments (Ne must be in (0, n), tau finite >= 0)");
        return SPAMM_E_INVAL;
    }
    sp2_opts_t o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = 100;
    if (o.trace_tol <= 0) o.trace_tol = 1e-10;
    if (o.idem_tol <= 0) o.idem_tol = 1e-8;
    if (o.leaf && o.leaf != F->b) {
        spamm_set_error("sp2_solve: opts.leaf (%d) differs from F's leaf size (%d)", o.leaf, F->b);
        return SPAMM_E_INVAL;
    }
    if (o.prec != SPAMM_FP64 && !(tc_mode_ok(o.prec, o.slices, F->b) && F->b <= 32)) {
        spamm_set_error("sp2_solve: precision mode %d (leaf %d, slices %d) not built", o.prec, F->b,
                        o.slices);
        return SPAMM_E_NOTSUP;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nb = F->nb, G = nb * nb;
    int rc;
    bool created = false;
    if (*Pout == nullptr) {
        spamm_mat_t m = new spamm_mat();
        if ((rc = spamm_mat_alloc(m, F->n, F->b, s))) {
            spamm_free(m);
            return rc;
        }
        *Pout = m;
        created = true;
    } else if (!spamm_mat_same_shape(*Pout, F) || *Pout == F || !spamm_mat_dense(*Pout)) {
        spamm_set_error("sp2_solve: P must match F's shape, store every leaf and not alias F");
        return SPAMM_E_INVAL;
    }
    spamm_mat_t X = *Pout;
    spamm_mat_t X2 = new spamm_mat();
    Sp2Scratch sc;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t evs[5 * kBatch] = {};
    const bool timing = (o.flags & SPAMM_F_TIMING) != 0;
    double ms_cull = 0.0, ms_gemm = 0.0, ms_update = 0.0;
    const int64_t launches0 = spamm_launch_count();
    bool sym = false;
    int it = 0, reason = SP2_STOP_MAXITER;
    int64_t tasks_total = 0;
    Sp2State h;
    memset(&h, 0, sizeof(h));
    spamm_opts_t mo;
    memset(&mo, 0, sizeof(mo));
    mo.leaf = F->b;
    mo.prec = o.prec;
    mo.slices = o.slices;
    mo.flags = kFlagUnitScale | (o.flags & SPAMM_F_HEAVIEST);  // iterates satisfy |x_ij| <= ||X||_2 < 2
    const int limit = o.fixed_iters > 0 ? o.fixed_iters : o.max_iter;
    const bool coarse = nb >= kCoarseMinNb;
    const bool tcpath = prec_is_tc(o.prec);  // X2's tiles without work are left unwritten
    bool use_graph = !(o.flags & SPAMM_F_NOGRAPH) && (tcpath || spamm_cull_never_waits(nb));
    cudaStream_t cs = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t graph_launches = 0;
    int graphed = 0;  // iterations run by graph replays

#define SP2_TRY(x)                 \
    do {                           \
        if ((rc = (x))) goto done; \
    } while (0)
#define SP2_LAUNCHED()                      \
    do {                                    \
        spamm_note_launches(1);             \
        SP2_CUDA(cudaGetLastError());       \
    } while (0)
#define SP2_CUDA(x)                                                           \
    do {                                                                      \
        cudaError_t e_ = (x);                                                 \
        if (e_ != cudaSuccess) {                                              \
            rc = spamm_cuda_fail(e_, #x, __FILE__, __LINE__);                 \
            goto done;                                                        \
        }                                                                     \
    } while (0)

    SP2_TRY(spamm_mat_alloc(X2, F->n, F->b, s));
    SP2_TRY(spamm_alloc((void **)&sc.st, sizeof(Sp2State), s));
    SP2_TRY(spamm_alloc((void **)&sc.lo, sizeof(double) * F->n, s));
    SP2_TRY(spamm_alloc((void **)&sc.hi, sizeof(double) * F->n, s));
    SP2_TRY(spamm_alloc((void **)&sc.idem_part, sizeof(double) * G, s));
    SP2_TRY(spamm_alloc((void **)&sc.diag_part, sizeof(double) * nb, s));
    SP2_TRY(spamm_alloc((void **)&sc.tr_part, sizeof(double) * 2 * nb, s));  // tensor path: two per leaf row
    SP2_TRY(spamm_alloc((void **)&sc.flag, sizeof(int32_t) * 4, s));
    SP2_TRY(spamm_alloc((void **)&sc.hist, sizeof(double) * SP2_H_COLS * limit, s));
    SP2_CUDA(cudaMallocHost((void **)&sc.host, sizeof(Sp2State)));
    SP2_CUDA(cudaMemsetAsync(sc.st, 0, sizeof(Sp2State), s));
    SP2_CUDA(cudaMemsetAsync(sc.flag, 0, sizeof(int32_t) * 4, s));
    if (X->scale)  // clear the slicing overflow flag left by an earlier solve into P
        SP2_CUDA(cudaMemsetAsync(reinterpret_cast<char *>(X->scale) + 12, 0, sizeof(int32_t), s));
    SP2_CUDA(cudaEventCreate(&ev0));
    SP2_CUDA(cudaEventCreate(&ev1));
    if (timing)
        for (int q = 0; q < 5 * kBatch; q++) SP2_CUDA(cudaEventCreate(&evs[q]));
    SP2_CUDA(cudaEventRecord(ev0, s));

    {
        // F must be symmetric: mirror leaves' norms agree to 1e-12 relative
        // (2e-12 on squared norms)
        SP2_CUDA(cudaMemsetAsync(sc.flag + 1, 0, sizeof(int32_t), s));
        k_norm_symmetry<<<(unsigned)((G + 255) / 256), 256, 0, s>>>(F->n2 + tier_offset(F->depth), nb, F->P, 2e-12,
                                                                   sc.flag + 1);
        SP2_LAUNCHED();
        int32_t asym_norms = 0;
        SP2_CUDA(cudaMemcpyAsync(&asym_norms, sc.flag + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SP2_CUDA(cudaStreamSynchronize(s));
        if (asym_norms) {
            spamm_set_error("sp2_solve: F is not symmetric (mirror leaf norms differ beyond 1e-12 relative)");
            rc = SPAMM_E_INVAL;
            goto done;
        }
    }
    if (!(o.flags & SPAMM_F_NOSYM)) {
        SP2_CUDA(cudaMemsetAsync(sc.flag, 0, sizeof(int32_t), s));
        k_symmetry<<<(unsigned)((G + 7) / 8), 256, 0, s>>>(F->leaf, F->slot, nb, F->b, sc.flag);
        SP2_LAUNCHED();
        int32_t asym = 1;
        SP2_CUDA(cudaMemcpyAsync(&asym, sc.flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SP2_CUDA(cudaStreamSynchronize(s));
        sym = asym == 0;
    }
    {
        const unsigned gb = (unsigned)((F->n + 127) / 128);
        if (F->b == 16) k_gershgorin_rows<16><<<gb, 128, 0, s>>>(F->leaf, F->slot, F->n, nb, sc.lo, sc.hi);
        else if (F->b == 32) k_gershgorin_rows<32><<<gb, 128, 0, s>>>(F->leaf, F->slot, F->n, nb, sc.lo, sc.hi);
        else k_gershgorin_rows<64><<<gb, 128, 0, s>>>(F->leaf, F->slot, F->n, nb, sc.lo, sc.hi);
    }
    SP2_LAUNCHED();
    k_gershgorin_bounds<<<1, kRedThreads, 0, s>>>(sc.lo, sc.hi, F->n, sc.st);
    SP2_LAUNCHED();
    launch_elementwise(X->b, s, 0, X->leaf, F->leaf, X->slot, F->slot, F->n, nb, X->P, X->n2 + tier_offset(X->depth),
                       X->n2T, sc.idem_part, sc.diag_part, sc.st, Sp2Rule{Ne, 0, 0, 0, 1}, sc.hist, nullptr, 1, 1, 0);
    SP2_LAUNCHED();
    // upper tiers of the iterate: the cull's early skip reads them (rebuilt
    // only where the skip pays; otherwise marked stale and not used)
    if (coarse) SP2_TRY(launch_pyramid(X, s));
    X->tiers_ok = coarse;

    // X2's product kernels return at once when the device rule has stopped
    X2->ws.stop = reinterpret_cast<const int32_t *>(reinterpret_cast<const char *>(sc.st) +
                                                    offsetof(Sp2State, stopped));
    {
        const Sp2Rule rule{Ne, o.trace_tol, o.idem_tol, o.fixed_iters, o.max_iter};
        // the launches of `batch` iterations on stream st
        auto enqueue = [&](cudaStream_t st, int batch) -> int {
            for (int q = 0; q < batch; q++) {
                cudaEvent_t *ev = timing ? evs + 5 * q : nullptr;
                // tensor path, symmetric: X2 keeps only its leaves i <= j (the
                // update reads a lower leaf as the transpose of its mirror)
                int r = spamm_multiply_into(X, X, tau, X2, &mo, sc.tr_part, st, false, nullptr, false, ev,
                                            sym ? 1 : 0, false, !tcpath, !(tcpath && sym));
                if (r) return r;
                const int32_t *x2rows = tcpath ? X2->ws.td0 : nullptr;
                k_sp2_decide<<<1, kRedThreads, 0, st>>>(sc.tr_part, tcpath ? 2 * nb : nb, X2->ws.task_total,
                                                        X2->ws.pair_units, Ne,
                                                        o.rule, sc.st);
                SPAMM_CK_LAUNCH();
                launch_elementwise(X->b, st, 1, X->leaf, X2->leaf, X->slot, X2->slot, F->n, nb, X->P,
                                   X->n2 + tier_offset(X->depth), X->n2T, sc.idem_part, sc.diag_part, sc.st, rule,
                                   sc.hist, x2rows, 128 / X->b, X2->ws.tw, sym ? 1 : 0, (tcpath && sym) ? 1 : 0);
                SPAMM_CK_LAUNCH();
                if (coarse && (r = launch_pyramid(X, st))) return r;
                if (timing) SPAMM_CK(spamm_event_record(ev[4], st));
            }
            return SPAMM_OK;
        };
        int enq = 0;
        while (enq < limit) {
            const int batch = limit - enq < kBatch ? limit - enq : kBatch;
            bool replayed = false;
            if (use_graph && batch == kBatch && enq > 0) {
                // the first batch ran directly (it allocated every workspace);
                // capture one batch on an internal stream, then replay it
                if (!gexec) {
                    cudaGraph_t gr = nullptr;
                    const int64_t l0 = spamm_launch_count();
                    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
                    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
                    if (e == cudaSuccess) {
                        const int r = enqueue(cs, kBatch);
                        e = cudaStreamEndCapture(cs, &gr);
                        if (r == SPAMM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&gexec, gr, 0);
                        else if (e == cudaSuccess) e = cudaErrorUnknown;
                    }
                    if (gr) cudaGraphDestroy(gr);
                    graph_launches = spamm_launch_count() - l0;
                    spamm_note_launches(-graph_launches);  // counted per replay instead
                    if (e != cudaSuccess || !gexec) {
                        cudaGetLastError();  // fall back to direct launches
                        use_graph = false;
                        gexec = nullptr;
                    }
                }
                if (gexec) {
                    SP2_CUDA(cudaGraphLaunch(gexec, s));
                    spamm_note_launches(graph_launches);
                    replayed = true;
                }
            }
            if (!replayed) SP2_TRY(enqueue(s, batch));
            enq += batch;
            const int before = h.iter;
            SP2_CUDA(cudaMemcpyAsync(sc.host, sc.st, sizeof(Sp2State), cudaMemcpyDeviceToHost, s));
            SP2_CUDA(cudaStreamSynchronize(s));
            h = *sc.host;
            if (replayed) graphed += h.iter - before;
            if (timing) {
                for (int q = 0; q < h.iter - before && q < batch; q++) {
                    float a = 0.f, b = 0.f, c = 0.f;
                    cudaEventElapsedTime(&a, evs[5 * q + 0], evs[5 * q + 1]);
                    cudaEventElapsedTime(&b, evs[5 * q + 1], evs[5 * q + 2]);
                    cudaEventElapsedTime(&c, evs[5 * q + 3], evs[5 * q + 4]);
                    ms_cull += a;
                    ms_gemm += b;
                    ms_update += c;
                }
            }
            if (h.stopped) break;
        }
    }
    X2->ws.stop = nullptr;
    it = h.iter;
    reason = h.stopped ? h.reason : SP2_STOP_MAXITER;
    if (it > 0) {
        std::vector<double> hrows((size_t)it * SP2_H_COLS);
        SP2_CUDA(cudaMemcpyAsync(hrows.data(), sc.hist, sizeof(double) * hrows.size(), cudaMemcpyDeviceToHost, s));
        SP2_CUDA(cudaStreamSynchronize(s));
        for (int q = 0; q < it; q++) tasks_total += (int64_t)hrows[(size_t)q * SP2_H_COLS + SP2_H_TASKS];
        if (report && report->history) {
            const int rows = it < report->history_cap ? it : report->history_cap;
            memcpy(report->history, hrows.data(), sizeof(double) * rows * SP2_H_COLS);
        }
    }
    SP2_TRY(ws_check_errors(&X2->ws, s));  // (also reads the rounded-sum count of the solve's products)
    SP2_TRY(launch_pyramid(X, s));
    X->tiers_ok = true;
    SP2_CUDA(cudaEventRecord(ev1, s));
    SP2_CUDA(cudaEventSynchronize(ev1));
    if (o.prec == SPAMM_OZAKI_BF16 && X->scale) {
        // the unit scale needs |x| < 2 in every iterate (spectrum in [0, 1])
        int32_t ovf = 0;
        SP2_CUDA(cudaMemcpy(&ovf, reinterpret_cast<const char *>(X->scale) + 12, sizeof(int32_t),
                            cudaMemcpyDeviceToHost));
        if (ovf) {
            spamm_set_error("sp2_solve: an iterate left the slicing range |x| < 2");
            rc = SPAMM_E_INVAL;
            goto done;
        }
    }

    if (report) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        report->iters = it;
        report->stop_reason = reason;
        report->trace_err = fabs(h.tn - Ne);
        report->idem_err = h.e;
        report->emin = h.emin;
        report->emax = h.emax;
        report->tasks_total = tasks_total;
        report->flops_useful = 2.0 * double(F->b) * F->b * F->b * double(tasks_total);
        report->flops_tensor = 2.0 * double(F->b) * F->b * F->b * double(h.units);
        report->ms_total = ms;
        report->ms_cull = ms_cull;
        report->ms_gemm = ms_gemm;
        report->ms_update = ms_update;
        report->launches = spamm_launch_count() - launches0;
        report->symmetric = sym ? 1 : 0;
        report->graphed = graphed;
        report->sums_rounded = X2->ws.last_rounded;
    }
    rc = reason == SP2_STOP_MAXITER ? SPAMM_E_NOCONV : SPAMM_OK;
    if (rc == SPAMM_E_NOCONV) spamm_set_error("sp2_solve: %d iterations without convergence", it);
done:
    if (gexec) cudaGraphExecDestroy(gexec);
    if (cs) cudaStreamDestroy(cs);
    for (int q = 0; q < 5 * kBatch; q++)
        if (evs[q]) cudaEventDestroy(evs[q]);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    sc.release(s);
    spamm_free(X2);
    if (rc && rc != SPAMM_E_NOCONV && created) {
        spamm_free(*Pout);
        *Pout = nullptr;
    }
    return rc;
#undef SP2_TRY
#undef SP2_CUDA
}
