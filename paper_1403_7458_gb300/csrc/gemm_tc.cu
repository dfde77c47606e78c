// gemm_tc.cu -- tile culling for the tensor-core leaf products (Eq. 4 on
// tiles of R = 128 / b output leaf rows) and the host side of the tcgen05
// kernel in tc_kernel.cuh (single products and batches); instantiates the
// kernel for leaf 32.
#include "tc_kernel.cuh"
#include "scan.cuh"

namespace {

// ---------------------------------------------------------------------------
// tile cull: work lists of items (k, masks, zA, zB); tile t = I * nbt + J
// (columns j = W J .. W J + W - 1, nbt = ceil(nb / W)) owns the list
// segment [t nb, t nb + count[t])
// ---------------------------------------------------------------------------
constexpr int kWarps = 8;

struct CullArgs {
    const double *n2A, *n2BT;
    // tier whose blocks are 32 x 32 leaves (W x W), for skipping a 32-wide
    // step of k at once (null when the quadtree is shallower)
    const double *cA, *cB;
    int64_t cW;
    // per coarse pair (block row of A, block column of B), the bit set of
    // the coarse k-blocks that pass (cwords words of 32 bits per pair; null
    // when the coarse tier is not used)
    const uint32_t *cmask;
    int64_t nc, cwords;
    int denseA, denseB;  // identity slot maps: leaf (i, k) is slot i nb + k
    const uint8_t *zA, *zB;        // leading zero slices per slot
    const int32_t *slotA, *slotB;  // slot maps (B: of the matrix whose slices serve as B)
    int64_t nb, P, nI, nbt;
    double tau2;
    int sym, S, R;  // R = 128 / b leaf rows per tile
    const int32_t *stop;  // set once an SP2 loop has stopped: nothing to do
    // per group g of kCullCols leaf columns and k: the largest squared norm
    // of the B leaves (k, j), j in the group (row g nb + k)
    const double *bgmax;
    int cols;  // leaf columns per warp of k_tile_count: kCullCols, or a divisor of it for small products
};

// The A side of the candidates k of one step (one per lane): the squared
// norms and leading-zero counts of the R leaves (i, k), i = R I .. R I + R-1,
// loaded once and tested against every tile column of the warp.
template <int R>
struct StepA {
    double a[R];
    int z[R];
    double amax;  // the largest of the a[r]: some row passes Eq. 4 iff this one does
};

template <int R>
__device__ __forceinline__ void load_step_a(const CullArgs &c, int64_t I, int64_t k, StepA<R> &s)
{
    // every load of the candidate issued before any is used (one round trip)
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int64_t i = (int64_t)R * I + r;
        const bool in = k < c.nb && i < c.nb;
        s.a[r] = in ? __ldg(c.n2A + i * c.P + k) : 0.0;
        s.z[r] = (in && c.denseA) ? c.zA[i * c.nb + k] : 0;
    }
    if (!c.denseA)
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int64_t i = (int64_t)R * I + r;
            // a leaf of nonzero norm is stored (its slot is valid)
            if (s.a[r] != 0.0) s.z[r] = c.zA[c.slotA[i * c.nb + k]];
        }
    s.amax = s.a[0];
#pragma unroll
    for (int r = 1; r < R; r++) s.amax = fmax(s.amax, s.a[r]);
}

// Leading-zero slices of the B operand leaf (k, j) (symmetric: its image is
// leaf (j, k)'s A role): from an identity slot map, else -1 (to be looked up
// through the slot map once the leaf is known to be stored).
__device__ __forceinline__ int zb_dense(const CullArgs &c, int64_t j, int64_t k)
{
    if (c.sym) return c.denseA ? c.zA[j * c.nb + k] : -1;
    return c.denseB ? c.zB[k * c.nb + j] : -1;
}
__device__ __forceinline__ int zb_slot(const CullArgs &c, int64_t j, int64_t k)
{
    return c.sym ? c.zA[c.slotA[j * c.nb + k]] : c.zB[c.slotB[k * c.nb + j]];
}

// Work item of tile (I, j) at k (tc::item_make), or 0 when no kept leaf has a
// nonzero product.  ntask += surviving triples (symmetric mode: of the whole
// product, see below); npair += slice pairs those triples need (p >= zA_i,
// q >= zB, p + q < S).
// b and zb: the squared norm of the B leaf and its zb_dense value.
template <int R>
__device__ __forceinline__ uint32_t tile_item(const CullArgs &c, const StepA<R> &s, int64_t I, int64_t j, int64_t k,
                                              double b, int zb, int &ntask, int &npair)
{
    if (k >= c.nb) return 0;
    if (b == 0.0) return 0;  // B leaf zero (or not stored): no triple of the step survives
    if (zb < 0) zb = zb_slot(c, j, k);
    uint32_t mask = 0;
    int za = c.S;
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int64_t i = (int64_t)R * I + r;
        if (i < c.nb && keep_product(s.a[r], b, c.tau2)) {
            // symmetric mode counts the whole product's triples from the
            // active tiles alone: (i, k, j) survives iff (j, k, i) does, so
            // a leaf above the diagonal stands for itself and its mirror
            ntask += !c.sym ? 1 : (i < j ? 2 : (i == j ? 1 : 0));
            const int z = s.z[r];
            if (z + zb < c.S) {
                const int mr = c.S - z - zb;
                npair += mr * (mr + 1) / 2;
                mask |= 1u << r;
                za = z < za ? z : za;
            }
        }
    }
    if (!mask) return 0;
    return tc::item_make((uint32_t)k, mask, za, zb);
}

// Slice pairs a one-column item issues.
__device__ __forceinline__ int item_pairs(uint32_t w, int S)
{
    const int m = S - tc::item_za(w) - tc::item_zb(w);
    return m * (m + 1) / 2;
}

// Work item of a two-column tile (I, J) at k (leaf 32, R = 4; tc::item_make2),
// or 0.  Symmetric mode keeps only the triples of stored leaves (i <= j): a
// leaf below the diagonal is the mirror of one above it.
// bn and zbl: the two columns' B norms and zb_dense values.
__device__ __forceinline__ uint32_t tile_item2(const CullArgs &c, const StepA<4> &s, int64_t I, int64_t J,
                                               int64_t k, const double (&bn)[2], const int (&zbl)[2], int &ntask,
                                               int &npair)
{
    if (k >= c.nb) return 0;
    uint32_t mask[2] = {0u, 0u};
    int zbv[2] = {7, 7};
    int za = c.S;
#pragma unroll
    for (int cc = 0; cc < 2; cc++) {
        const int64_t j = 2 * J + cc;
        const double b = bn[cc];
        if (j >= c.nb || b == 0.0) continue;
        const int zb = zbl[cc] >= 0 ? zbl[cc] : zb_slot(c, j, k);
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int64_t i = 4 * I + r;
            if (i < c.nb && (!c.sym || i <= j) && keep_product(s.a[r], b, c.tau2)) {
                ntask += !c.sym ? 1 : (i < j ? 2 : 1);
                const int zr = s.z[r];
                if (zr + zb < c.S) {
                    const int mr = c.S - zr - zb;
                    npair += mr * (mr + 1) / 2;
                    mask[cc] |= 1u << r;
                    za = zr < za ? zr : za;
                }
            }
        }
        if (mask[cc]) zbv[cc] = zb;
    }
    if (!(mask[0] | mask[1])) return 0;
    return tc::item_make2((uint32_t)k, mask[0], mask[1], za, zbv[0], zbv[1]);
}

// Slice pairs a two-column item issues (its columns share zA).
__device__ __forceinline__ int item_pairs2(uint32_t w, int S)
{
    int n = 0;
#pragma unroll
    for (int cc = 0; cc < 2; cc++) {
        if (!tc::item_mask_col<4, 2>(w, cc)) continue;
        const int m = S - tc::item_za(w) - tc::item_zb_col(w, cc);
        n += m * (m + 1) / 2;
    }
    return n;
}

// Early occlusion (Algorithm 1): the R rows of tile I lie in one block row
// of the 32 x 32-leaf tier (R divides 32) and its W columns in one block
// column, so when that block row of A and the block of B holding
// (k0 .. k0+31, j) fail the test, every triple of the step fails (a parent's
// squared norm is never below a child's).  The passing blocks of each coarse
// pair are found once (k_coarse_mask) and every tile of the pair reads them.
//
// Bit sets of the passing coarse k-blocks: one warp per coarse pair (block
// row ci of A, block column cj of B in the tier whose blocks are 32 x 32
// leaves); bit kc of the pair's set is the culling test of Eq. 4 on the
// blocks (ci, kc) and (kc, cj).
__global__ void k_coarse_mask(const int32_t *__restrict__ stop, const double *__restrict__ cA,
                              const double *__restrict__ cB, int64_t cW, int64_t nc, int64_t cwords, double tau2,
                              uint32_t *__restrict__ mask)
{
    if (stop && *stop) return;
    const int64_t pr = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (pr >= nc * nc) return;
    const int64_t ci = pr / nc, cj = pr % nc;
    for (int64_t wd = 0; wd < cwords; wd++) {
        const int64_t kc = wd * 32 + lane;
        const bool p = kc < nc && keep_product(__ldg(cA + ci * cW + kc), __ldg(cB + kc * cW + cj), tau2);
        const unsigned bal = __ballot_sync(0xffffffffu, p);
        if (lane == 0) mask[pr * cwords + wd] = bal;
    }
}

// Leaf columns of a tile row that one warp of k_tile_count culls (a divisor
// of the coarse tier's 32, so that they share one coarse block column).
constexpr int kCullCols = 16;

// bgmax[g nb + k] = max over the group's columns j of n2B[k, j] (B's
// transposed norms n2BT[j P + k]): when the largest A norm of a k-step fails
// Eq. 4 against it in every lane, no tile of the group has a triple there.
__global__ void k_group_bmax(const int32_t *__restrict__ stop, const double *__restrict__ n2BT, int64_t P,
                             int64_t nb, int64_t ng, double *__restrict__ bgmax)
{
    if (stop && *stop) return;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= ng * nb) return;
    const int64_t g = q / nb, k = q % nb;
    double m = 0.0;
#pragma unroll 4
    for (int jj = 0; jj < kCullCols; jj++) {
        const int64_t j = g * kCullCols + jj;
        if (j < nb) m = fmax(m, __ldg(n2BT + j * P + k));
    }
    bgmax[q] = m;
}

// One warp per tile row I and c.cols leaf columns (c.cols / W tiles; c.cols
// divides kCullCols): for each step of 32 candidates k (lane = k) it loads the A side once and
// tests it against every tile of the warp (ballot), writing each tile's work
// items into the tile's own segment of the list, [t nb, t nb + count), in
// increasing k.  Per tile it counts the items, the surviving triples and the
// slice pairs; d0[t] receives, per tile column c, the least zA + zB over the
// column's items (4 bits at 4 c: the lowest diagonal its products touch; S
// when it has none) and the leaf rows any of them keeps (R bits at 8 + 8 c:
// the output leaves with work).  Lane jt holds the counts of the warp's
// tile jt.
template <int W, int R>
__global__ void __launch_bounds__(kWarps * 32, R <= 4 ? 4 : 3)
k_tile_count(CullArgs c, int32_t *__restrict__ counts, int32_t *__restrict__ tasks,
             int32_t *__restrict__ pairs, int32_t *__restrict__ useful, int32_t *__restrict__ d0out,
             uint32_t *__restrict__ list)
{
    const int NT = c.cols / W;  // tiles per warp
    static_assert(kCullCols / W <= 32, "a lane holds the counts of one tile");
    static_assert(W == 1 || R == 4, "two-column tiles have four leaf rows");
    if (c.stop && *c.stop) return;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int64_t ncg = (c.nbt + NT - 1) / NT;  // tile groups per tile row
    if (gw >= c.nI * ncg) return;
    const int64_t I = gw / ncg, J0 = (gw % ncg) * NT;
    const int nt = (int)(c.nbt - J0 < NT ? c.nbt - J0 : NT);  // tiles of this warp
    // symmetric mode: a tile entirely below the block diagonal (its last
    // column left of its first row) is formed as a mirror; the active tiles
    // are jt >= jt0
    int jt0 = 0;
    if (c.sym) {
        const int64_t jmin = ((int64_t)R * I + 1 + W - 1) / W - 1;  // least J with W J + W - 1 >= R I
        jt0 = jmin <= J0 ? 0 : (int)(jmin - J0 < nt ? jmin - J0 : nt);
    }
    int cnt = 0, ntask = 0, npair = 0, nuse = 0;  // of tile J0 + lane
    uint32_t tbits = 0;  // OR of the items' row and diagonal bits (see below)
    const unsigned lt = (1u << lane) - 1u;
    if (jt0 < nt) {
        // the steps of 32 candidates k0 .. k0 + 31 to test: the coarse
        // blocks whose pair with the warp's block row and column passes
        // (precomputed bit sets), else every step
        const int64_t nsteps = (c.nb + 31) / 32;
        const uint32_t *cm =
            c.cmask ? c.cmask + (((int64_t)R * I >> 5) * c.nc + (((int64_t)W * J0) >> 5)) * c.cwords : nullptr;
        for (int64_t wd = 0; wd < (nsteps + 31) / 32; wd++) {
            uint32_t bits = cm ? __ldg(cm + wd) : 0xFFFFFFFFu;  // warp-uniform
            while (bits) {
                const int64_t kc = wd * 32 + (__ffs(bits) - 1);
                bits &= bits - 1;
                if (kc >= nsteps) break;
                const int64_t k = kc * 32 + lane;
                StepA<R> sa;
                load_step_a<R>(c, I, k, sa);
                // no triple of the step survives in any tile of the warp: the
                // largest A norm fails against the largest B norm of the group
                // (the warp's columns lie in one group of kCullCols)
                const double bg = k < c.nb ? __ldg(c.bgmax + ((int64_t)W * J0 / kCullCols) * c.nb + k) : 0.0;
                if (!__any_sync(0xffffffffu, keep_product(sa.amax, bg, c.tau2))) continue;
                for (int jt = jt0; jt < nt; jt++) {
                    const int64_t J = J0 + jt;
                    // the B side (norms and leading zeros loaded together), and
                    // first the largest A norm of the step against it: when no
                    // lane passes, no triple of the tile's step survives
                    double bn[W];
                    int zbl[W];
                    bool pass = false;
#pragma unroll
                    for (int cc = 0; cc < W; cc++) {
                        const int64_t j = W * J + cc;
                        const bool in = k < c.nb && j < c.nb;
                        bn[cc] = in ? __ldg(c.n2BT + j * c.P + k) : 0.0;
                        zbl[cc] = in ? zb_dense(c, j, k) : 0;
                    }
#pragma unroll
                    for (int cc = 0; cc < W; cc++) pass = pass || keep_product(sa.amax, bn[cc], c.tau2);
                    if (!__any_sync(0xffffffffu, pass)) continue;
                    int tk = 0, tp = 0;
                    uint32_t w;
                    if constexpr (W == 2) w = tile_item2(c, sa, I, J, k, bn, zbl, tk, tp);
                    else w = tile_item<R>(c, sa, I, J, k, bn[0], zbl[0], tk, tp);
                    const unsigned bal = __ballot_sync(0xffffffffu, w != 0);
                    // nothing survives and nothing is listed (a kept triple below
                    // the diagonal of a symmetric product counts 0 but may be listed)
                    if (!__any_sync(0xffffffffu, tk != 0 || w != 0)) continue;
                    const int base = __shfl_sync(0xffffffffu, cnt, jt);
                    // the item's kept rows per column (8 / W bits each, from bit 0)
                    // and its lowest diagonal per column (one-hot, 8 bits from
                    // bit 8 + 8 c): one OR over the warp gives both
                    int pr = 0;
                    uint32_t bits = 0;
                    if (w) {
                        list[(I * c.nbt + J) * c.nb + base + __popc(bal & lt)] = w;
                        if constexpr (W == 2) {
                            pr = item_pairs2(w, c.S);
#pragma unroll
                            for (int cc = 0; cc < 2; cc++) {
                                const uint32_t m = tc::item_mask_col<4, 2>(w, cc);
                                if (m) bits |= m << (4 * cc) | 1u << (8 + 8 * cc + tc::item_za(w) + tc::item_zb_col(w, cc));
                            }
                        } else {
                            pr = item_pairs(w, c.S);
                            bits = tc::item_mask(w) | 1u << (8 + tc::item_za(w) + tc::item_zb(w));
                        }
                    }
                    const int sk = __reduce_add_sync(0xffffffffu, tk);
                    const int su = __reduce_add_sync(0xffffffffu, tp);
                    const int sp = __reduce_add_sync(0xffffffffu, pr);
                    const uint32_t so = __reduce_or_sync(0xffffffffu, bits);
                    if (lane == jt) {
                        cnt += __popc(bal);
                        ntask += sk;
                        nuse += su;
                        npair += sp;
                        tbits |= so;
                    }
                }
            }
        }
    }
    if (lane < nt) {
        const int64_t t = I * c.nbt + J0 + lane;
        const bool active = lane >= jt0;
        int packed = 0;
#pragma unroll
        for (int cc = 0; cc < W; cc++) {
            const uint32_t dz = (tbits >> (8 + 8 * cc)) & 0xFFu;  // diagonals that are some item's lowest
            const uint32_t rows = (tbits >> (8 / W * cc)) & ((1u << (8 / W)) - 1u);
            packed |= (dz ? min(__ffs(dz) - 1, c.S) : c.S) << (4 * cc) | (int)(rows << (8 + 8 * cc));
        }
        counts[t] = active ? cnt : 0;
        tasks[t] = active ? ntask : 0;
        pairs[t] = active ? npair : 0;
        useful[t] = active ? nuse : 0;
        d0out[t] = active ? packed : (W == 2 ? (c.S | c.S << 4) : c.S);
    }
}

// Hand-out orders list only the tiles with work (the rest of the order array
// holds -1); tiles without work are never handed out.
// Heaviest-first order (counting sort on the work-list length):
// hist -> descending exclusive scan -> scatter.
__global__ void k_tile_hist(const int32_t *__restrict__ stop, const int32_t *__restrict__ counts, int64_t nb,
                            int64_t G, int sym, int R, int32_t *__restrict__ bins)
{
    if (stop && *stop) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < G && counts[t] > 0) atomicAdd(bins + counts[t], 1);
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

// Zeroes the output leaves of tiles without work (they are never handed
// out): one warp per (tile, leaf row, tile column); in symmetric mode leaf
// (i, j), i <= j, and its mirror (j, i) (a leaf below the diagonal is the
// mirror of one above it).
__global__ void __launch_bounds__(kWarps * 32)
k_tile_zero(const int32_t *__restrict__ stop, const int32_t *__restrict__ counts, int64_t nb, int64_t nI,
            int64_t nbt, int R, int W, int sym, int b, const int32_t *__restrict__ slotC, double *__restrict__ leafC)
{
    if (stop && *stop) return;
    const int64_t w = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= nI * nbt * R * W) return;
    const int64_t t = w / (R * W), L = (w / W) % R, cc = w % W;
    const int64_t I = t / nbt, j = W * (t % nbt) + cc, i = (int64_t)R * I + L;
    if (counts[t] > 0 || i >= nb || j >= nb || (sym && i > j)) return;
    const double2 z = make_double2(0.0, 0.0);
    double2 *d = reinterpret_cast<double2 *>(leafC + (int64_t)slotC[i * nb + j] * b * b);
    for (int q = lane; q < b * b / 2; q += 32) d[q] = z;
    if (sym && i < j) {
        d = reinterpret_cast<double2 *>(leafC + (int64_t)slotC[j * nb + i] * b * b);
        for (int q = lane; q < b * b / 2; q += 32) d[q] = z;
    }
}

__global__ void k_tile_scatter(const int32_t *__restrict__ stop, const int32_t *__restrict__ counts, int64_t nb,
                               int64_t G, int sym, int R, int32_t *__restrict__ bins, int32_t *__restrict__ order)
{
    if (stop && *stop) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < G && counts[t] > 0) order[atomicAdd(bins + counts[t], 1)] = (int32_t)t;
}


}  // namespace

int tc_launch_b32(const tc::TcArgs &a, int S, int E, cudaStream_t s) { return tc::launch_leaf<32>(a, S, E, s); }

namespace {

// Watchdog self-test: one thread waits, with the kernels' bounded wait, on an
// mbarrier that nothing arrives at; the wait gives up after `limit` cycles
// and the kernel reports it in *err (1 = gave up, 2 = the barrier completed).
__global__ void k_watchdog(long long limit, int32_t *err)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    abort_flag = 0;
    tc::mbar_init(tc::smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const bool done = tc::mbar_wait(tc::smem_u32(&bar), 0, &abort_flag, limit);
    *err = done ? 2 : 1;
}

}  // namespace

extern "C" int spamm_watchdog_selftest(int32_t ms, void *stream)
{
    if (ms < 1 || ms > 10000) {
        spamm_set_error("spamm_watchdog_selftest: ms must be in 1..10000");
        return SPAMM_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, khz = 0;
    SPAMM_CK(cudaGetDevice(&dev));
    SPAMM_CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    if (khz <= 0) khz = 2070000;
    int32_t *err = nullptr;
    int rc = spamm_alloc((void **)&err, sizeof(int32_t), s);
    if (rc) return rc;
    SPAMM_CK(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    k_watchdog<<<1, 32, 0, s>>>((long long)ms * khz, err);
    SPAMM_CK_LAUNCH();
    int32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    spamm_release(err, s);
    if (e != cudaSuccess) return spamm_cuda_fail(e, "watchdog self-test", __FILE__, __LINE__);
    if (h == 1) {
        spamm_set_error("watchdog self-test: the wait gave up after %d ms (expected)", ms);
        return SPAMM_E_TIMEOUT;
    }
    spamm_set_error("watchdog self-test: unexpected state %d", h);
    return SPAMM_E_CUDA;
}

int tc_mode_ok(int prec, int slices, int leaf)
{
    if (!prec_is_tc(prec) || (leaf != 16 && leaf != 32 && leaf != 64)) return 0;
    const int s = prec_slices(prec, slices);
    if (!prec_float_split(prec) && (s < 3 || s > 7)) return 0;
    return s * leaf <= (int)tc::kAccStride;
}

// Tile cull for the tensor-core path into ws: tile lists and the order in
// which tiles are handed out: row-major (consecutive tiles share their row
// of A leaves, which then stays in L2) or heaviest first (tiles are taken
// dynamically, so this is longest-processing-time-first scheduling);
// toff[T + 1] receives the number of surviving triples.
int tc_tile_cull(spamm_mat_t A, spamm_mat_t B, double tau, SpammWorkspace *ws, int sym, int slices,
                 cudaStream_t s, bool heaviest_first)
{
    const int R = 128 / A->b, W = tc::tile_width(A->b, slices);
    const int64_t nb = A->nb, P = A->P, nI = (nb + R - 1) / R, nbt = (nb + W - 1) / W, T = nI * nbt;
    if (W == 2 && R != 4) {  // tile_item2 builds the masks of 4-row tiles
        spamm_set_error("tensor-core path: two-column tiles need leaf 32 (got %d)", A->b);
        return SPAMM_E_NOTSUP;
    }
    if (T >= (int64_t(1) << 24)) {
        spamm_set_error("tensor-core path: %lld tiles exceed 2^24", (long long)T);
        return SPAMM_E_NOTSUP;
    }
    int rc;
    if (ws->tile_cap < T) {
        spamm_release(ws->tcounts, s);
        spamm_release(ws->ttasks, s);
        spamm_release(ws->tpairs, s);
        spamm_release(ws->toff, s);
        spamm_release(ws->torder, s);
        spamm_release(ws->tbins, s);
        spamm_release(ws->tuseful, s);
        spamm_release(ws->tnz, s);
        spamm_release(ws->td0, s);
        ws->tcounts = ws->ttasks = ws->tpairs = ws->tuseful = ws->torder = ws->tbins = ws->tnz = ws->td0 = nullptr;
        ws->toff = nullptr;
        ws->tile_cap = 0;
        if ((rc = spamm_alloc((void **)&ws->tcounts, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->ttasks, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->tpairs, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->tuseful, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->toff, sizeof(int64_t) * (T + 4), s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->torder, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->tnz, sizeof(int32_t) * T, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->td0, sizeof(int32_t) * T, s))) return rc;
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
    c.nbt = nbt;
    c.tau2 = tau * tau;
    c.sym = sym;
    c.S = slices;
    c.R = R;
    c.stop = ws->stop;
    c.cA = c.cB = nullptr;
    c.cW = 0;
    c.cmask = nullptr;
    c.nc = (nb + 31) / 32;
    c.cwords = (c.nc + 31) / 32;
    c.denseA = spamm_mat_dense(A);
    c.denseB = spamm_mat_dense(B);
    if (A->depth >= 5 && A->tiers_ok && B->tiers_ok) {
        c.cA = A->n2 + tier_offset(A->depth - 5);
        c.cB = B->n2 + tier_offset(B->depth - 5);
        c.cW = int64_t(1) << (A->depth - 5);
        const int64_t words = c.nc * c.nc * c.cwords;
        if (ws->cmask_cap < words) {
            spamm_release(ws->cmask, s);
            ws->cmask = nullptr;
            ws->cmask_cap = 0;
            if ((rc = spamm_alloc((void **)&ws->cmask, sizeof(uint32_t) * words, s))) return rc;
            ws->cmask_cap = words;
        }
        k_coarse_mask<<<(unsigned)((c.nc * c.nc + 7) / 8), 256, 0, s>>>(ws->stop, c.cA, c.cB, c.cW, c.nc, c.cwords,
                                                                         c.tau2, ws->cmask);
        SPAMM_CK_LAUNCH();
        c.cmask = ws->cmask;
    }
    // one warp per tile row and c.cols leaf columns: kCullCols (the A side
    // of a step then serves the most tiles), fewer when that would leave
    // the GPU with under 32 warps per SM
    c.cols = kCullCols;
    while (c.cols > W && nI * ((nbt + c.cols / W - 1) / (c.cols / W)) < (int64_t)spamm_num_sms() * 32) c.cols /= 2;
    const int64_t cull_warps = nI * ((nbt + c.cols / W - 1) / (c.cols / W));
    const unsigned blocks = (unsigned)((cull_warps + kWarps - 1) / kWarps);
    {
        const int64_t ng = (nb + kCullCols - 1) / kCullCols, need = ng * nb;
        if (ws->bgmax_cap < need) {
            spamm_release(ws->bgmax, s);
            ws->bgmax = nullptr;
            ws->bgmax_cap = 0;
            if ((rc = spamm_alloc((void **)&ws->bgmax, sizeof(double) * need, s))) return rc;
            ws->bgmax_cap = need;
        }
        k_group_bmax<<<(unsigned)((need + 255) / 256), 256, 0, s>>>(ws->stop, c.n2BT, P, nb, ng, ws->bgmax);
        SPAMM_CK_LAUNCH();
        c.bgmax = ws->bgmax;
    }
    const int64_t worst = T * nb;  // every tile owns a segment of nb items (one per k)
    if (ws->tlist_cap < worst) {
        spamm_release(ws->tlist, s);
        ws->tlist = nullptr;
        ws->tlist_cap = 0;
        if ((rc = spamm_alloc((void **)&ws->tlist, sizeof(uint32_t) * worst, s))) return rc;
        ws->tlist_cap = worst;
    }
    auto kern = W == 2 ? k_tile_count<2, 4> : R == 8 ? k_tile_count<1, 8> : R == 4 ? k_tile_count<1, 4>
                                                                                 : k_tile_count<1, 2>;
    kern<<<blocks, kWarps * 32, 0, s>>>(c, ws->tcounts, ws->ttasks, ws->tpairs, ws->tuseful, ws->td0, ws->tlist);
    SPAMM_CK_LAUNCH();
    // totals: toff[T] work items, toff[T+1] surviving triples, toff[T+2]
    // issued slice-pair work, toff[T+3] slice pairs the surviving triples need
    // (toff[0..T) the items' running count); the order of tiles with work
    ws->tsym = sym;
    ws->tw = W;
    ws->tT = T;
    // hand-out positions: the active tiles (symmetric: tile row I starts at
    // tile column floor(R I / W), the first whose last column reaches row R I)
    ws->tactive = T;
    if (sym) {
        ws->tactive = 0;
        for (int64_t I = 0; I < nI; I++) {
            const int64_t j0 = (int64_t)R * I / W;
            ws->tactive += nbt > j0 ? nbt - j0 : 0;
        }
    }
    SPAMM_CK(cudaMemsetAsync(ws->torder, 0xFF, sizeof(int32_t) * ws->tactive, s));  // -1: no tile
    // offsets, ranks among the tiles with work and the row-major order of
    // those; totals at toff[T .. T+3]
    if ((rc = ws_reserve_scan(ws, T, s))) return rc;
    {
        const int64_t nch = (T + scan::kChunk - 1) / scan::kChunk;
        scan::k_sums<true><<<(unsigned)nch, scan::kThreads, 0, s>>>(ws->stop, ws->tcounts, ws->ttasks, ws->tpairs,
                                                                     ws->tuseful, T, ws->scan_part);
        SPAMM_CK_LAUNCH();
        scan::k_top<true><<<1, scan::kTopThreads, 0, s>>>(ws->stop, ws->scan_part, nch, ws->toff + T,
                                                          ws->toff + T + 1, ws->toff + T + 2, ws->toff + T + 3);
        SPAMM_CK_LAUNCH();
        scan::k_apply<true><<<(unsigned)nch, scan::kThreads, 0, s>>>(ws->stop, ws->tcounts, T, ws->scan_part, ws->toff,
                                                                      ws->tnz, heaviest_first ? nullptr : ws->torder);
        SPAMM_CK_LAUNCH();
    }
    if (heaviest_first) {
        SPAMM_CK(cudaMemsetAsync(ws->tbins, 0, sizeof(int32_t) * (nb + 1), s));
        k_tile_hist<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(ws->stop, ws->tcounts, nb, T, sym, R, ws->tbins);
        SPAMM_CK_LAUNCH();
        k_tile_bins_scan<<<1, 32, 0, s>>>(ws->stop, ws->tbins, nb + 1);
        SPAMM_CK_LAUNCH();
        k_tile_scatter<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(ws->stop, ws->tcounts, nb, T, sym, R, ws->tbins,
                                                                     ws->torder);
        SPAMM_CK_LAUNCH();
    }
    return SPAMM_OK;
}

int tc_zero_empty_tiles(spamm_mat_t C, SpammWorkspace *ws, cudaStream_t s)
{
    const int R = 128 / C->b, W = ws->tw;
    const int64_t nb = C->nb, nI = (nb + R - 1) / R, nbt = (nb + W - 1) / W;
    const int64_t warps = nI * nbt * R * W;
    k_tile_zero<<<(unsigned)((warps + kWarps - 1) / kWarps), kWarps * 32, 0, s>>>(
        ws->stop, ws->tcounts, nb, nI, nbt, R, W, ws->tsym, C->b, C->slot, C->leaf);
    SPAMM_CK_LAUNCH();
    return SPAMM_OK;
}

static void fill_prob(tc::TcProb &p, spamm_mat_t A, spamm_mat_t B, spamm_mat_t C, SpammWorkspace *ws,
                      double *tr_part, int64_t pos0)
{
    p.slA = A->slA;
    p.slB = B->slB;  // per-leaf slices: B-role layout
    // symmetric product: the B leaves come from the tile-major array (A == B)
    p.tmB = ws->tsym ? B->tmapA : nullptr;
    p.slotA = A->slot;
    p.slotB = B->slot;
    p.slotC = C->slot;
    p.leafC = C->leaf;
    p.cnt = ws->tcounts;
    p.d0 = ws->td0;
    p.list = ws->tlist;
    p.order = ws->torder;
    p.sigA = reinterpret_cast<const int32_t *>(A->scale + 1);
    p.sigB = reinterpret_cast<const int32_t *>(B->scale + 1);
    p.tr_part = tr_part;
    p.nb = A->nb;
    p.nbt = (A->nb + ws->tw - 1) / ws->tw;
    p.pos0 = pos0;
    p.sym = ws->tsym;
    p.tw = ws->tw;
    p.mirror = ws->tmirror;
    p.rounded = ws->counter ? ws->counter + 11 : nullptr;
    p.skip_idle = ws->tskip_idle;
}

static int launch_args(tc::TcArgs &a, int leaf, int slices, int e, cudaStream_t s)
{
    SPAMM_CK(cudaMemsetAsync(a.next_tile, 0, sizeof(int32_t), s));
    switch (leaf) {
    case 16: return tc_launch_b16(a, slices, e, s);
    case 32: return tc_launch_b32(a, slices, e, s);
    case 64: return tc_launch_b64(a, slices, e, s);
    default: return SPAMM_E_NOTSUP;
    }
}

int launch_gemm_tc(spamm_mat_t A, spamm_mat_t B, spamm_mat_t C, SpammWorkspace *ws,
                   double *tr_part, int slices, int e, cudaStream_t s, bool float_split)
{
    if (tr_part && A->b > 32) {
        spamm_set_error("tensor-core path: diagonal traces need leaf 16 or 32 (got %d)", A->b);
        return SPAMM_E_NOTSUP;
    }
    // diagonal leaves of tiles without work are never handed out: their
    // traces are 0 (two partial traces per leaf row, see the epilogue)
    if (tr_part) SPAMM_CK(cudaMemsetAsync(tr_part, 0, sizeof(double) * 2 * A->nb, s));
    thread_local tc::TcArgs a;  // large (one table entry used); host-side staging only
    fill_prob(a.p[0], A, B, C, ws, tr_part, 0);
    a.nprob = 1;
    a.T = ws->tactive;
    a.err = ws->counter + 9;
    a.next_tile = ws->counter + 10;
    a.stop = ws->stop;
    a.float_split = float_split ? 1 : 0;
    return launch_args(a, A->b, slices, e, s);
}

int launch_gemm_tc_batched(int count, const spamm_mat_t *A, const spamm_mat_t *B, const spamm_mat_t *C,
                           SpammWorkspace *const *ws, int slices, int e, cudaStream_t s, bool float_split,
                           int32_t *counters)
{
    if (count < 1 || count > kMaxBatch) return SPAMM_E_INVAL;
    thread_local tc::TcArgs a;
    int64_t pos = 0;
    for (int m = 0; m < count; m++) {
        fill_prob(a.p[m], A[m], B[m], C[m], ws[m], nullptr, pos);
        pos += ws[m]->tactive;
    }
    a.nprob = count;
    a.T = pos;
    a.err = counters + 9;
    a.next_tile = counters + 10;
    a.stop = nullptr;
    a.float_split = float_split ? 1 : 0;
    return launch_args(a, A[0]->b, slices, e, s);
}
