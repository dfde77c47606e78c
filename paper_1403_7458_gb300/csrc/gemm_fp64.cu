// gemm_fp64.cu -- grouped FP64 leaf products C_ij = sum_{k in S_ij} A_ik B_kj
// (the dense leaf product of Algorithm 1, applied to every surviving triple).
//
// Symmetric products (A == B exactly symmetric, as in SP2) form only the
// output leaves i <= j and store each C_ij (i < j) also as C_ji = C_ij^T.
//
// Output-stationary: one CTA owns one output leaf (i, j) at a time, so no two
// CTAs write the same C leaf and no lock or atomic on C is needed (the paper's
// OpenMP lock on C has no counterpart here).  CTAs are persistent and pull
// output leaves from a device counter.  For each surviving k, the A_ik and
// B_kj leaves are staged into shared memory with cp.async (double-buffered)
// and multiplied with FP64 fused multiply-adds, k increasing.  The epilogue
// writes C_ij, its exact squared norm (leaf tier of C's quadtree), and for
// diagonal leaves the partial trace used by SP2.
//
// A launch serves a table of up to kMaxBatch independent products: output
// leaves of all of them are numbered consecutively (product by product) and
// pulled from the one counter.
//
// Roofline: FP64 pipe bound (2 b^3 FLOP per task; operands 16 b^2 bytes per
// task, mostly served from L2).
#include "internal.cuh"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

struct FpProb {
    const double *leafA;
    const int32_t *slotA;
    const double *leafB;
    const int32_t *slotB;
    double *leafC;
    const int32_t *slotC;
    int64_t nb;
    int64_t P;
    const int64_t *off;
    const uint32_t *klist;
    double *n2C;
    double *n2CT;
    double *tr_part;
    int64_t g0;  // first output-leaf number of this product
    int32_t sym; // A == B exactly symmetric: only leaves i <= j are formed, C_ji = C_ij^T
    int64_t *exec;  // leaf products formed (may be null)
};

struct GemmArgs {
    FpProb p[kMaxBatch];
    int64_t G;            // output leaves over all products
    int32_t nprob;
    int32_t *counter;
    const int32_t *stop;  // set once an SP2 loop has stopped: nothing to do
};

__device__ __forceinline__ int find_prob(const GemmArgs &g, int64_t x)
{
    int lo = 0, hi = g.nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g.p[mid].g0 <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int B>
struct Tile {
    // rows x cols of outputs per thread
    static constexpr int TR = B == 64 ? 4 : 1;
    static constexpr int TC = B == 16 ? 1 : 4;
    static constexpr int COLT = B / TC;  // threads along a row
};

template <int B>
__device__ __forceinline__ void stage_leaf(double *dst, const double *src, int tid)
{
    constexpr int chunks = B * B / 2;  // 16-byte chunks
    for (int q = tid; q < chunks; q += kThreads) cp_async16(dst + 2 * q, src + 2 * q);
}

// (i, j) of entry x of the upper block triangle (i <= j) in row-major order:
// row i starts at i nb - i (i - 1) / 2.
__device__ __forceinline__ void upper_pair(int64_t x, int64_t nb, int64_t &i, int64_t &j)
{
    const double b = 2.0 * (double)nb + 1.0;
    int64_t r = (int64_t)floor((b - sqrt(b * b - 8.0 * (double)x)) * 0.5);
    auto start = [nb](int64_t q) { return q * nb - q * (q - 1) / 2; };
    if (r < 0) r = 0;
    if (r > nb - 1) r = nb - 1;
    while (r > 0 && start(r) > x) r--;
    while (r + 1 < nb && start(r + 1) <= x) r++;
    i = r;
    j = x - start(r) + r;
}

template <int B>
__global__ void __launch_bounds__(kThreads) k_gemm_fp64(const __grid_constant__ GemmArgs g)
{
    using T = Tile<B>;
    extern __shared__ __align__(16) double smem[];
    double *As = smem;               // [2][B*B]
    double *Bs = smem + 2 * B * B;   // [2][B*B]
    __shared__ int64_t s_group;
    __shared__ int s_red_i[kThreads / 32];
    __shared__ u128 s_red_u[kThreads / 32];

    if (g.stop && *g.stop) return;
    const int tid = threadIdx.x;
    int64_t formed = 0;      // leaf products this CTA formed (thread 0)
    int64_t *exec_out = nullptr;
    const int r0 = (tid / T::COLT) * T::TR;
    const int c0 = (tid % T::COLT) * T::TC;
    const int64_t G = g.G;

    for (;;) {
        if (tid == 0) s_group = atomicAdd(g.counter, 1);
        __syncthreads();
        const int64_t gg = s_group;
        if (gg >= G) break;
        const FpProb &P = g.p[find_prob(g, gg)];
        int64_t i, j;
        if (P.sym) upper_pair(gg - P.g0, P.nb, i, j);
        else {
            i = (gg - P.g0) / P.nb;
            j = (gg - P.g0) % P.nb;
        }
        const int64_t grp = i * P.nb + j;
        const int64_t t0 = P.off[grp], t1 = P.off[grp + 1];
        formed += t1 - t0;
        exec_out = P.exec;

        double acc[T::TR][T::TC];
#pragma unroll
        for (int a = 0; a < T::TR; a++)
#pragma unroll
            for (int b = 0; b < T::TC; b++) acc[a][b] = 0.0;

        if (t1 > t0) {
            {
                uint32_t k = P.klist[t0];
                stage_leaf<B>(As, P.leafA + (int64_t)P.slotA[i * P.nb + k] * B * B, tid);
                stage_leaf<B>(Bs, P.leafB + (int64_t)P.slotB[(int64_t)k * P.nb + j] * B * B, tid);
                cp_async_commit();
            }
            for (int64_t t = t0; t < t1; t++) {
                const int st = (int)((t - t0) & 1);
                if (t + 1 < t1) {
                    uint32_t k = P.klist[t + 1];
                    stage_leaf<B>(As + (st ^ 1) * B * B,
                                  P.leafA + (int64_t)P.slotA[i * P.nb + k] * B * B, tid);
                    stage_leaf<B>(Bs + (st ^ 1) * B * B,
                                  P.leafB + (int64_t)P.slotB[(int64_t)k * P.nb + j] * B * B, tid);
                }
                cp_async_commit();
                cp_async_wait1();
                __syncthreads();
                const double *a_s = As + st * B * B;
                const double *b_s = Bs + st * B * B;
#pragma unroll 4
                for (int l = 0; l < B; l++) {
                    double av[T::TR], bv[T::TC];
#pragma unroll
                    for (int a = 0; a < T::TR; a++) av[a] = a_s[(r0 + a) * B + l];
#pragma unroll
                    for (int b = 0; b < T::TC; b++) bv[b] = b_s[l * B + c0 + b];
#pragma unroll
                    for (int a = 0; a < T::TR; a++)
#pragma unroll
                        for (int b = 0; b < T::TC; b++) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
                }
                __syncthreads();
            }
        }

        // ---- epilogue: store C_ij, its squared norm and (diagonal) trace ----
        double *Cs = As;  // reuse stage 0 of A
#pragma unroll
        for (int a = 0; a < T::TR; a++)
#pragma unroll
            for (int b = 0; b < T::TC; b++) Cs[(r0 + a) * B + c0 + b] = acc[a][b];
        __syncthreads();
        double *dst = P.leafC + (int64_t)P.slotC[grp] * B * B;
        int emax = 0;
        for (int q = tid; q < B * B / 2; q += kThreads) {
            double2 v = reinterpret_cast<const double2 *>(Cs)[q];
            reinterpret_cast<double2 *>(dst)[q] = v;
            emax = max(emax, max(exp_key(v.x), exp_key(v.y)));
        }
        if (P.sym && i < j) {
            // the mirror leaf C_ji = C_ij^T (bit-identical to forming it: the
            // same products in the same order, the factors swapped)
            double *mir = P.leafC + (int64_t)P.slotC[j * P.nb + i] * B * B;
            for (int q = tid; q < B * B / 2; q += kThreads) {
                const int rr = (2 * q) / B, cc = (2 * q) % B;
                reinterpret_cast<double2 *>(mir)[q] = make_double2(Cs[cc * B + rr], Cs[(cc + 1) * B + rr]);
            }
        }
        emax = warp_max_int(emax);
        if ((tid & 31) == 0) s_red_i[tid >> 5] = emax;
        __syncthreads();
        emax = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; w++) emax = max(emax, s_red_i[w]);
        u128 accn = 0;
        if (emax > 0)
            for (int q = tid; q < B * B; q += kThreads) accn += sq_term(Cs[q], emax);
        accn = warp_sum_u128(accn);
        if ((tid & 31) == 0) s_red_u[tid >> 5] = accn;
        __syncthreads();
        if (tid == 0) {
            u128 tot = 0;
            for (int w = 0; w < kThreads / 32; w++) tot += s_red_u[w];
            double r = emax > 0 ? sq_sum_round(tot, emax) : 0.0;
            P.n2C[i * P.P + j] = r;
            P.n2CT[j * P.P + i] = r;
            if (P.sym && i < j) {  // a transposed leaf has the same exact squared norm
                P.n2C[j * P.P + i] = r;
                P.n2CT[i * P.P + j] = r;
            }
            if (i == j && P.tr_part) {
                double tr = 0.0;
                for (int q = 0; q < B; q++) tr += Cs[q * B + q];
                P.tr_part[i] = tr;
            }
        }
        __syncthreads();
    }
    if (tid == 0 && exec_out && formed) atomicAdd(reinterpret_cast<unsigned long long *>(exec_out),
                                                  (unsigned long long)formed);
}

template <int B>
int launch_b(const GemmArgs &args, cudaStream_t s)
{
    size_t smem = sizeof(double) * 4 * B * B;
    static unsigned long long configured = 0;
    if (int rc = spamm_smem_attr(k_gemm_fp64<B>, smem, configured)) return rc;
    int per_sm = 0;
    SPAMM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemm_fp64<B>, kThreads, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)spamm_num_sms() * per_sm;
    if (grid > args.G) grid = args.G;
    if (grid < 1) grid = 1;
    k_gemm_fp64<B><<<(unsigned)grid, kThreads, smem, s>>>(args);
    SPAMM_CK_LAUNCH();
    return SPAMM_OK;
}

}  // namespace

static void fill_prob(FpProb &p, spamm_mat_t A, spamm_mat_t B, spamm_mat_t C, SpammWorkspace *ws,
                      double *tr_part, int64_t g0)
{
    p.leafA = A->leaf;
    p.slotA = A->slot;
    p.leafB = B->leaf;
    p.slotB = B->slot;
    p.leafC = C->leaf;
    p.slotC = C->slot;
    p.nb = A->nb;
    p.P = A->P;
    p.off = ws->off;
    p.klist = ws->klist;
    p.n2C = C->n2 + tier_offset(C->depth);
    p.n2CT = C->n2T;
    p.tr_part = tr_part;
    p.g0 = g0;
    p.sym = 0;
    p.exec = nullptr;
}

static int launch_args(GemmArgs &g, int leaf, cudaStream_t s)
{
    SPAMM_CK(cudaMemsetAsync(g.counter, 0, sizeof(int32_t), s));
    switch (leaf) {
    case 16: return launch_b<16>(g, s);
    case 32: return launch_b<32>(g, s);
    case 64: return launch_b<64>(g, s);
    default:
        spamm_set_error("leaf size %d not built", leaf);
        return SPAMM_E_NOTSUP;
    }
}

int launch_gemm_fp64(spamm_mat_t A, spamm_mat_t B, spamm_mat_t C, SpammWorkspace *ws,
                     double *tr_part, cudaStream_t s, int sym)
{
    thread_local GemmArgs g;  // large (one table entry used); host-side staging only
    fill_prob(g.p[0], A, B, C, ws, tr_part, 0);
    g.p[0].sym = sym ? 1 : 0;
    g.p[0].exec = ws->exec;
    if (ws->exec) SPAMM_CK(cudaMemsetAsync(ws->exec, 0, sizeof(int64_t), s));
    g.nprob = 1;
    g.G = sym ? A->nb * (A->nb + 1) / 2 : A->nb * A->nb;
    g.counter = ws->counter;
    g.stop = ws->stop;
    return launch_args(g, A->b, s);
}

int launch_gemm_fp64_batched(int count, const spamm_mat_t *A, const spamm_mat_t *B, const spamm_mat_t *C,
                             SpammWorkspace *const *ws, cudaStream_t s, int32_t *counter)
{
    if (count < 1 || count > kMaxBatch) return SPAMM_E_INVAL;
    thread_local GemmArgs g;
    int64_t g0 = 0;
    for (int m = 0; m < count; m++) {
        fill_prob(g.p[m], A[m], B[m], C[m], ws[m], nullptr, g0);
        g0 += A[m]->nb * A[m]->nb;
    }
    g.nprob = count;
    g.G = g0;
    g.counter = counter;
    g.stop = nullptr;
    return launch_args(g, A[0]->b, s);
}
