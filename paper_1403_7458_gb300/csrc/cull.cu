// cull.cu -- the SpAMM culling pass (Eq. 4; Algorithm 1's occlusion test).
//
// The recursive walk of Algorithm 1 reaches exactly the leaf triples
// (i, k, j) whose leaf norms pass the test (a parent's squared norm is the
// rounded sum of its children's and so never smaller), so the task set is
// decided flat on the leaf tier.  Output is grouped by output leaf
// g = i * nb + j: the surviving k of group g are klist[off[g] .. off[g+1])
// in increasing order.
//
// Three launches:
//   count : one warp per group; lanes walk k in steps of 32 and count the
//           passing candidates with a ballot + popcount; a step is skipped
//           whole when the quadtree tier whose blocks are 32 x 32 leaves
//           already fails the test for the block row of i and the block
//           column of j (Algorithm 1's early occlusion: a parent's squared
//           norm is never below a child's, so no leaf triple under a failing
//           parent pair can pass);
//   scan  : exclusive prefix sum of the counts (three launches over many
//           blocks, scan.cuh);
//   emit  : the warps re-test and write each passing k at its ballot rank.
// Roofline: ALU/latency bound on the candidate tests; HBM/L2 traffic is the
// two leaf-norm rows per group (16 nb bytes) plus 4 bytes per task written.
#include "internal.cuh"
#include "scan.cuh"

namespace {

constexpr int kWarps = 8;

// Squared norms of the tier whose blocks are 32 x 32 leaves (W x W grid),
// for the early skip; null when the quadtree has fewer than 5 tiers below
// the root.
struct Coarse {
    const double *a, *b;
    int64_t W;
};

__device__ __forceinline__ bool coarse_pass(const Coarse &c, int64_t i, int64_t k0, int64_t j, double tau2)
{
    return !c.a || keep_product(__ldg(c.a + (i >> 5) * c.W + (k0 >> 5)), __ldg(c.b + (k0 >> 5) * c.W + (j >> 5)),
                                tau2);
}

__global__ void __launch_bounds__(kWarps * 32)
k_cull_count(const int32_t *__restrict__ stop, const double *__restrict__ n2A,
             const double *__restrict__ n2BT, int64_t nb, int64_t P, double tau2, Coarse co,
             int32_t *__restrict__ counts)
{
    if (stop && *stop) return;  // the SP2 loop has already stopped
    int64_t g = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (g >= nb * nb) return;
    int64_t i = g / nb, j = g % nb;
    const double *ra = n2A + i * P;
    const double *rb = n2BT + j * P;
    int cnt = 0;
    for (int64_t k0 = 0; k0 < nb; k0 += 32) {
        if (!coarse_pass(co, i, k0, j, tau2)) continue;  // warp-uniform
        int64_t k = k0 + lane;
        bool p = k < nb && keep_product(__ldg(ra + k), __ldg(rb + k), tau2);
        cnt += __popc(__ballot_sync(0xffffffffu, p));
    }
    if (lane == 0) counts[g] = cnt;
}

__global__ void __launch_bounds__(kWarps * 32)
k_cull_emit(const int32_t *__restrict__ stop, const double *__restrict__ n2A,
            const double *__restrict__ n2BT, int64_t nb, int64_t P, double tau2, Coarse co,
            const int64_t *__restrict__ off, uint32_t *__restrict__ klist, int64_t cap,
            int32_t *__restrict__ err)
{
    if (stop && *stop) return;  // the SP2 loop has already stopped
    int64_t g = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (g >= nb * nb) return;
    int64_t i = g / nb, j = g % nb;
    const double *ra = n2A + i * P;
    const double *rb = n2BT + j * P;
    int64_t base = off[g];
    if (off[g + 1] > cap) {
        if (lane == 0) atomicExch(err, 1);
        return;
    }
    unsigned lt = (1u << lane) - 1u;
    for (int64_t k0 = 0; k0 < nb; k0 += 32) {
        if (!coarse_pass(co, i, k0, j, tau2)) continue;  // warp-uniform
        int64_t k = k0 + lane;
        bool p = k < nb && keep_product(__ldg(ra + k), __ldg(rb + k), tau2);
        unsigned m = __ballot_sync(0xffffffffu, p);
        if (p) klist[base + __popc(m & lt)] = (uint32_t)k;
        base += __popc(m);
    }
}

Coarse coarse_tier(spamm_mat_t A, spamm_mat_t B)
{
    Coarse c{nullptr, nullptr, 0};
    if (A->depth >= 5 && A->tiers_ok && B->tiers_ok) {
        c.a = A->n2 + tier_offset(A->depth - 5);
        c.b = B->n2 + tier_offset(B->depth - 5);
        c.W = int64_t(1) << (A->depth - 5);
    }
    return c;
}

}  // namespace

// Worst-case list sizes up to this many bytes are reserved without asking the
// device for the exact count.
static const int64_t kEagerListBytes = int64_t(512) << 20;

bool spamm_cull_never_waits(int64_t nb) { return nb * nb * nb * 4 <= kEagerListBytes; }

int spamm_cull(spamm_mat_t A, spamm_mat_t B, double tau, SpammWorkspace *ws, int64_t nb,
               int64_t P, cudaStream_t s, bool need_total, int64_t *total_host, bool worst_case)
{
    int64_t G = nb * nb;
    double tau2 = tau * tau;
    unsigned blocks = (unsigned)((G + kWarps - 1) / kWarps);
    const Coarse co = coarse_tier(A, B);
    k_cull_count<<<blocks, kWarps * 32, 0, s>>>(ws->stop, A->n2 + tier_offset(A->depth), B->n2T, nb, P, tau2, co,
                                                ws->counts);
    SPAMM_CK_LAUNCH();
    if (int rc = ws_reserve_scan(ws, G, s)) return rc;
    {
        const int64_t nch = (G + scan::kChunk - 1) / scan::kChunk > 0 ? (G + scan::kChunk - 1) / scan::kChunk : 1;
        scan::k_sums<false><<<(unsigned)nch, scan::kThreads, 0, s>>>(ws->stop, ws->counts, nullptr, nullptr, nullptr,
                                                                      G, ws->scan_part);
        SPAMM_CK_LAUNCH();
        scan::k_top<false><<<1, scan::kTopThreads, 0, s>>>(ws->stop, ws->scan_part, nch, ws->off + G, nullptr,
                                                           nullptr, nullptr);
        SPAMM_CK_LAUNCH();
        scan::k_apply<false><<<(unsigned)nch, scan::kThreads, 0, s>>>(ws->stop, ws->counts, G, ws->scan_part,
                                                                       ws->off, nullptr, nullptr);
        SPAMM_CK_LAUNCH();
    }
    int64_t worst = G * nb;
    int64_t total = -1;
    if (need_total || (!worst_case && ws->klist_cap < worst && worst * 4 > kEagerListBytes)) {
        SPAMM_CK(cudaMemcpyAsync(&total, ws->off + G, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SPAMM_CK(cudaStreamSynchronize(s));
    }
    int64_t want = total >= 0 ? total : worst;
    if (ws->klist_cap < want) {
        int64_t cap = want;
        if (worst_case || (total >= 0 && worst * 4 <= kEagerListBytes)) cap = worst;
        else if (total >= 0) cap = want + want / 4 < worst ? want + want / 4 : worst;
        spamm_release(ws->klist, s);
        ws->klist = nullptr;
        ws->klist_cap = 0;
        int rc = spamm_alloc((void **)&ws->klist, sizeof(uint32_t) * (cap > 0 ? cap : 1), s);
        if (rc) return rc;
        ws->klist_cap = cap;
    }
    k_cull_emit<<<blocks, kWarps * 32, 0, s>>>(ws->stop, A->n2 + tier_offset(A->depth), B->n2T, nb, P, tau2, co,
                                               ws->off, ws->klist, ws->klist_cap, ws->counter + 8);
    SPAMM_CK_LAUNCH();
    if (total_host) *total_host = total;
    return SPAMM_OK;
}
