// internal.cuh -- shared declarations of the CUDA SpAMM / SP2 library.
//
// Layout in HBM (one handle = one n x n matrix):
//   leaf   : nslots leaves, each b x b FP64 row-major and contiguous
//            (leaf (i, k) lives at slot[i * nb + k]; dense handles use
//            slot = i * nb + k, so a block row of leaves is contiguous);
//   slot   : nb x nb int32 slot map (-1 = absent leaf: a sparse input built
//            with a drop threshold; outputs store every leaf);
//   n2     : squared norms of the whole quadtree (Sec. 2, Eqs. 1-3), tiers
//            t = 0..d concatenated, tier t a 2^t x 2^t row-major grid at
//            offset (4^t - 1) / 3; the leaf tier is P x P, P = 2^d;
//   n2T    : the leaf tier transposed (n2T[j * P + k] = n2[k][j]) so that a
//            warp reading B's column of leaf norms reads contiguous memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "spamm.h"

// ---------------------------------------------------------------------------
// Handle and workspace
// ---------------------------------------------------------------------------
struct SpammWorkspace {
    // task list (grouped by output leaf g = i * nb + j)
    int32_t *counts = nullptr;   // nb*nb
    int64_t *off = nullptr;      // nb*nb + 1
    uint32_t *klist = nullptr;   // capacity entries
    int64_t klist_cap = 0;
    int64_t groups_cap = 0;
    int32_t *counter = nullptr;  // work counters and error flags (16 ints)
    int64_t *exec = nullptr;     // FP64 path: leaf products formed by the last product
    double *tr_part = nullptr;   // per leaf row partial traces (nb)
    int64_t tr_cap = 0;
    // tensor-core path: tile work lists (tile t = I * nbt + J: leaf rows
    // R I .. R I + R - 1, leaf columns tw J .. tw J + tw - 1, nbt = ceil(nb / tw))
    int32_t *tcounts = nullptr;  // work items per tile
    int32_t *ttasks = nullptr;   // surviving triples per tile
    int32_t *tpairs = nullptr;   // slice-pair work per tile (sum of m(m+1)/2)
    int32_t *tuseful = nullptr;  // slice pairs the tile's surviving triples need
    int32_t *td0 = nullptr;      // per tile and column c: least zA + zB over its items (4 bits at 4 c; S:
                                 // none), leaf rows with work (R bits at 8 + 8 c)
    int64_t *toff = nullptr;     // T + 2: offsets, then the triple total
    int32_t *torder = nullptr;   // tile hand-out order (row-major or heaviest first), tiles with work only, then -1
    int32_t *tnz = nullptr;      // rank of each tile among the tiles with work
    int32_t *tbins = nullptr;    // nb + 1 histogram bins
    uint32_t *tlist = nullptr;   // k | mask << 15 | zA << 23 | zB << 26 (two columns: tc::item_make2)
    int64_t tile_cap = 0, tlist_cap = 0;
    const int64_t *task_total = nullptr;  // device: surviving triples of the last cull
    const int64_t *pair_units = nullptr;  // device: slice pairs needed (tensor path), else null
    int64_t last_items = 0;               // host copy: tile work items of the last product
    int64_t last_pairs = 0;               // host copy: slice-pair MMA work (units of 128 x b x b)
    int32_t last_rounded = 0;             // host copy: output elements with a diagonal sum >= 2^24 (counter 11)
    int64_t tactive = 0;                  // tiles in the order list of the last tile cull
    const int32_t *stop = nullptr;        // device flag: when set, the product's kernels return at once
    int tsym = 0;                         // last tile cull was symmetric
    int tw = 1;                           // output leaf columns per tile of the last tile cull
    int tmirror = 1;                      // symmetric tensor-core product: also store C_ji = C_ij^T
    int tskip_idle = 0;                   // tensor-core product: leaves without work in tiles with work are
                                          // not written (the caller reads the tile masks), else zeroed
    int64_t tT = 0;                       // tiles of the last tile cull (totals at toff + tT)
    uint32_t *cmask = nullptr;            // tile cull: passing coarse k-blocks per coarse (row, column) pair
    int64_t cmask_cap = 0;                // uint32 words
    double *bgmax = nullptr;              // tile cull: per group of 16 leaf columns j and k, max_j n2B[k, j]
    int64_t bgmax_cap = 0;                // doubles
    double *lmax = nullptr;               // slicing: largest partner norm per row / column (2 nb)
    int64_t lmax_cap = 0;                 // doubles
    int64_t *scan_part = nullptr;         // chunk partials of the multi-block scans (scan.cuh)
    int64_t scan_cap = 0;                 // int64 words
};

struct spamm_mat {
    int64_t n = 0;
    int b = 0;
    int64_t nb = 0;
    int depth = 0;
    int64_t P = 0;
    int64_t nslots = 0;
    double *leaf = nullptr;
    int32_t *slot = nullptr;
    double *n2 = nullptr;
    double *n2T = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    // slices for the tensor-core path (slice.cu): BF16 (2-byte) or TF32
    // (4-byte) elements; R = 128 / b leaf rows per tile
    uint8_t *slA = nullptr;           // A operand, tile-major [I][k][p][L] (R leaf rows per block)
    uint8_t *slB = nullptr;           // per-leaf [p][..] array (B operand)
    int slB_transposed = -1;          // layout of slB: 1 = B-role (transposed), 0 = A-role
    // tensor maps (CUtensorMap, 128 B each) of slA seen from the B role of a
    // symmetric product: map m - 1 copies m consecutive slices of one leaf
    // (slice.cu); null when not built
    void *tmapA = nullptr;
    uint8_t *zlead = nullptr;         // leading all-zero slices per slot
    int sl_s = 0;
    int sl_e = 0;                     // bytes per slice element
    unsigned long long *scale = nullptr;  // [0] max |x| bits, [1] int32 sigma, int32 overflow flag
    bool scale_unit = false;              // scale[0] holds the fixed unit maximum (1.0)
    bool tiers_ok = true;  // upper norm tiers match the leaf tier (the cull's early skip reads them)
    SpammWorkspace ws;  // used when this handle is the output of a product
};

// ---------------------------------------------------------------------------
// Host helpers (api.cu)
// ---------------------------------------------------------------------------
void spamm_set_error(const char *fmt, ...);
int spamm_cuda_fail(cudaError_t e, const char *what, const char *file, int line);
int spamm_alloc(void **p, size_t bytes, cudaStream_t s);
void spamm_release(void *p, cudaStream_t s);

#define SPAMM_CK(call)                                                        \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return spamm_cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define SPAMM_CK_LAUNCH()          \
    do {                           \
        spamm_note_launches(1);    \
        SPAMM_CK(cudaGetLastError()); \
    } while (0)

#ifdef __CUDACC__
__host__ __device__
#endif
static inline int64_t tier_offset(int t) { return ((int64_t(1) << (2 * t)) - 1) / 3; }

int spamm_num_sms();

// Raise a kernel's dynamic shared-memory limit once per device (the
// attribute belongs to the device the call is made on).
template <class Kernel>
int spamm_smem_attr(Kernel kernel, size_t bytes, unsigned long long &done_mask)
{
    int dev = 0;
    SPAMM_CK(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(__atomic_load_n(&done_mask, __ATOMIC_ACQUIRE) & bit)) {
        SPAMM_CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        __atomic_fetch_or(&done_mask, bit, __ATOMIC_RELEASE);
    }
    return SPAMM_OK;
}
cudaError_t spamm_event_record(cudaEvent_t e, cudaStream_t s);
int spamm_mat_alloc(spamm_mat_t m, int64_t n, int b, cudaStream_t s);
int spamm_mat_same_shape(spamm_mat_t a, spamm_mat_t b);
// Every leaf stored, slot = i * nb + k (outputs of products and of SP2).
int spamm_mat_dense(spamm_mat_t m);

// The early skip of the cull (32 x 32-leaf tier) pays from this many leaf
// rows on; SP2 rebuilds its iterate's upper tiers only then.
constexpr int64_t kCoarseMinNb = 256;

// Norms (norms.cu)
int launch_leaf_norms(spamm_mat_t m, cudaStream_t s);
int launch_pyramid(spamm_mat_t m, cudaStream_t s);

// Cull (cull.cu): fills ws.off / ws.klist for SpAMM(A, B, tau) into C's workspace.
// On return *total_host is the number of tasks when `need_total` is set (blocking),
// otherwise -1.
// worst_case: reserve room for every candidate instead of asking the device
// for the count (never waits for the stream; for graph capture).
int spamm_cull(spamm_mat_t A, spamm_mat_t B, double tau, SpammWorkspace *ws,
               int64_t nb, int64_t P, cudaStream_t s, bool need_total, int64_t *total_host,
               bool worst_case = false);
int ws_reserve_groups(SpammWorkspace *ws, int64_t groups, int64_t nb, cudaStream_t s);
// Room for the chunk partials of a scan over G entries in ws->scan_part.
int ws_reserve_scan(SpammWorkspace *ws, int64_t G, cudaStream_t s);
// The FP64 cull of an nb x nb leaf grid reserves its worst-case list (and so
// never waits for the stream once reserved).
bool spamm_cull_never_waits(int64_t nb);

// C = SpAMM(A, B, tau) into an existing handle (api.cu).  ev (optional, 4
// events) is recorded before the cull, before the products, before and after
// C's upper norm tiers.
// sym: A == B is exactly symmetric; both paths then form only the upper
// block triangle of C and mirror it (bit-identical, half the work).
// mirror = false (symmetric tensor path): only the leaves i <= j are
// stored; the caller reads C_ji as the transpose of C_ij (SP2 does).
// zero_empty = false (tensor path): leaves of tiles without work are left
// unwritten; the caller treats them as zero through ws->toff (SP2 does).
int spamm_multiply_into(spamm_mat_t A, spamm_mat_t B, double tau, spamm_mat_t C,
                        const spamm_opts_t *opts, double *tr_part, cudaStream_t s,
                        bool need_total, int64_t *tasks_out, bool build_pyramid,
                        cudaEvent_t *ev, int sym = 0, bool slices_ready = false, bool zero_empty = true,
                        bool mirror = true);

// Read and clear the device-side error words of a product (blocking).
int ws_check_errors(SpammWorkspace *ws, cudaStream_t s);

// Count of kernels this library launched (for reports).
void spamm_note_launches(int64_t k);
int64_t spamm_launch_count();

// Tensor-core path (slice.cu, gemm_tc*.cu).  e = bytes per slice element:
// 2 (BF16, tcgen05 kind::f16) or 4 (TF32, kind::tf32).
// keep_a / keep_b (optional, nb entries): largest partner norm per column
// (A role) / per row (B role); leaves that fail Eq. 4 against it are not
// sliced (the slices then serve only the product they were made for).
int launch_slices(spamm_mat_t m, int s, int e, bool tile_a, bool per_leaf, bool transposed, cudaStream_t st,
                  const int32_t *stop = nullptr, bool unit_scale = false, bool float_split = false,
                  const double *keep_a = nullptr, const double *keep_b = nullptr, double tau2 = 0.0);

// Tensor-core precision modes: slices per operand, element size, and whether
// the slices are exact integer digits (Ozaki) or a float split.
static inline bool prec_is_tc(int prec)
{
    return prec == SPAMM_OZAKI_BF16 || prec == SPAMM_BF16 || prec == SPAMM_BF16X3 || prec == SPAMM_TF32 ||
           prec == SPAMM_TF32X3;
}
static inline int prec_slices(int prec, int slices)
{
    return (prec == SPAMM_BF16 || prec == SPAMM_TF32) ? 1
           : (prec == SPAMM_BF16X3 || prec == SPAMM_TF32X3) ? 2
                                                             : (slices ? slices : 7);
}
static inline bool prec_float_split(int prec) { return prec != SPAMM_OZAKI_BF16; }
static inline int prec_elem(int prec) { return (prec == SPAMM_TF32 || prec == SPAMM_TF32X3) ? 4 : 2; }

// Internal flag of spamm_opts_t.flags: slice with the fixed scale sigma = 1
// (the caller guarantees |x| < 2, as SP2 does for its iterates).
constexpr int32_t kFlagUnitScale = 1 << 30;
int slices_alloc(spamm_mat_t m, int s, int e, bool tile_a, bool per_leaf, cudaStream_t st);
// Tensor maps of m's tile-major array for B-role copies (built once per
// allocation of the array; a kernel writes them, so the call can be captured).
int slices_tmaps(spamm_mat_t m, cudaStream_t st);
int tc_tile_cull(spamm_mat_t A, spamm_mat_t B, double tau, SpammWorkspace *ws, int sym, int slices,
                 cudaStream_t s, bool heaviest_first = false);
// Zero the output leaves of tiles without work (never handed out).
int tc_zero_empty_tiles(spamm_mat_t C, SpammWorkspace *ws, cudaStream_t s);
int launch_gemm_tc(spamm_mat_t A, spamm_mat_t B, spamm_mat_t C, SpammWorkspace *ws,
                   double *tr_part, int slices, int e, cudaStream_t s, bool float_split = false);
// One launch over the products m < count (count <= kMaxBatch) whose tile
// lists are in ws[m]; products are taken in the given order.
constexpr int kMaxBatch = 64;
int launch_gemm_tc_batched(int count, const spamm_mat_t *A, const spamm_mat_t *B, const spamm_mat_t *C,
                           SpammWorkspace *const *ws, int slices, int e, cudaStream_t s, bool float_split,
                           int32_t *counters);
// A tensor-core mode is built for (prec, slices, leaf): exact slices 3..7
// (BF16), float splits 1 or 2 terms; slices x leaf <= 256 TMEM columns.
int tc_mode_ok(int prec, int slices, int leaf);

// FP64 leaf products of count independent products in one launch (gemm_fp64.cu)
int launch_gemm_fp64_batched(int count, const spamm_mat_t *A, const spamm_mat_t *B, const spamm_mat_t *C,
                             SpammWorkspace *const *ws, cudaStream_t s, int32_t *counter);

// Leaf products (gemm_fp64.cu)
int launch_gemm_fp64(spamm_mat_t A, spamm_mat_t B, spamm_mat_t C, SpammWorkspace *ws,
                     double *tr_part, cudaStream_t s, int sym = 0);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

typedef unsigned __int128 u128;

// Exponent key and integer significand of |x| (IEEE binary64):
// |x| = m * 2^(e - 1075) with e >= 1; m = 0 for x = 0.
__device__ __forceinline__ void dbl_decompose(double x, uint64_t &m, int &e)
{
    uint64_t u = (uint64_t)__double_as_longlong(x);
    int E = (int)((u >> 52) & 0x7ff);
    uint64_t f = u & 0xFFFFFFFFFFFFFull;
    if (E == 0) {
        m = f;
        e = 1;
    } else {
        m = f | (1ull << 52);
        e = E;
    }
}

// RN(S * 2^k) for an unsigned 128-bit integer S (round to nearest, ties to
// even).  Exact whenever the result is a normal double.
__device__ __forceinline__ double u128_round_scaled(u128 S, int k)
{
    if (S == 0) return 0.0;
    uint64_t hi = (uint64_t)(S >> 64), lo = (uint64_t)S;
    int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    uint64_t mant;
    if (msb <= 52) {
        mant = lo;
    } else {
        int sh = msb - 52;
        mant = (uint64_t)(S >> sh);
        u128 rem = S & ((((u128)1) << sh) - 1);
        u128 half = ((u128)1) << (sh - 1);
        if (rem > half || (rem == half && (mant & 1))) mant++;
        if (mant == (1ull << 53)) {
            mant >>= 1;
            sh++;
        }
        k += sh;
    }
    if (mant >= (1ull << 52)) {
        int be = k + 52 + 1023;
        if (be >= 1 && be <= 2046)
            return __longlong_as_double((long long)(((uint64_t)be << 52) | (mant & 0xFFFFFFFFFFFFFull)));
    }
    return ldexp((double)mant, k);
}

// Exact fixed-point accumulation of squares: with emax the largest exponent
// key in a set of doubles, x^2 contributes floor(m^2 * 2^10 / 4^(emax - e))
// units of 2^(2 emax - 2160).  Every term is truncated on its own, so the sum
// is independent of the order of accumulation; the truncation is below 2^-104
// of the result, far inside one FP64 rounding.
__device__ __forceinline__ u128 sq_term(double x, int emax)
{
    uint64_t m;
    int e;
    dbl_decompose(x, m, e);
    if (m == 0) return 0;
    int sh = 2 * (emax - e);
    if (sh >= 120) return 0;
    u128 t = ((u128)m * (u128)m) << 10;
    return t >> sh;
}

__device__ __forceinline__ int exp_key(double x)
{
    uint64_t m;
    int e;
    dbl_decompose(x, m, e);
    return m ? e : 0;
}

__device__ __forceinline__ double sq_sum_round(u128 S, int emax)
{
    return u128_round_scaled(S, 2 * emax - 2160);
}

// Same scheme for non-negative doubles themselves (a parent's four children).
__device__ __forceinline__ u128 val_term(double x, int emax)
{
    uint64_t m;
    int e;
    dbl_decompose(x, m, e);
    if (m == 0) return 0;
    int sh = emax - e;
    if (sh >= 120) return 0;
    u128 t = ((u128)m) << 63;
    return t >> sh;
}

__device__ __forceinline__ double val_sum_round(u128 S, int emax)
{
    return u128_round_scaled(S, emax - 1075 - 63);
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int mask)
{
    uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    lo = __shfl_xor_sync(0xffffffffu, lo, mask);
    hi = __shfl_xor_sync(0xffffffffu, hi, mask);
    return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u128 warp_sum_u128(u128 v)
{
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor_u128(v, o);
    return v;
}

__device__ __forceinline__ int warp_max_int(int v)
{
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Exact slicing (see slice.cu): X = round-half-up(|x| 2^(7S - sigma)) as an
// integer (X <= 2^(7S) whenever |x| < 2^sigma), and its base-128 digit p as
// BF16 bits carrying the sign of x (digit 0 unmasked: it may be 128).
__device__ __forceinline__ uint64_t slice_int(double x, int sigma, int S)
{
    uint64_t m;
    int e;
    dbl_decompose(x, m, e);
    if (!m) return 0;
    const int sh = 1075 + sigma - 7 * S - e;
    if (sh <= 0) return m << (-sh);
    if (sh < 64) return (m >> sh) + ((m >> (sh - 1)) & 1ull);
    return 0;
}

__device__ __forceinline__ uint16_t slice_digit_bf16(uint64_t X, bool neg, int p, int S)
{
    uint32_t d = (uint32_t)(X >> (7 * (S - 1 - p)));
    if (p > 0) d &= 127u;
    // the FP32 value d (exact: d <= 128 < 2^23) from the bits of 2^23 + d,
    // minus 2^23; d <= 128 is exact in BF16 too, so the top half is its BF16
    const uint32_t f = __float_as_uint(__int_as_float(0x4B000000 | (int)d) - 8388608.0f);
    return (uint16_t)((f >> 16) | (neg ? 0x8000u : 0u));
}

// Layout of one slice of a B x B leaf with E-byte elements, as the tcgen05
// K-major operand wants it: row r of the leaf (M or N index) holds its
// B E bytes of K (= columns c); rows come in groups of 8 (stride 8 B E
// bytes, the descriptor's stride offset); within a group the K bytes are cut
// into swizzle atoms of AW = min(B E, 128) bytes (8 rows x AW bytes each,
// atoms along K adjacent), and inside an atom the 16-byte chunk index of row
// r8 is XOR-permuted by the row bits (the 32-, 64- and 128-byte swizzle
// modes).  Byte offset of element (r, c):
template <int B, int E>
__host__ __device__ constexpr int slice_atom_bytes() { return B * E < 128 ? B * E : 128; }

template <int B, int E>
__device__ __forceinline__ int slice_byte_offset(int r, int c)
{
    constexpr int RB = B * E, AW = slice_atom_bytes<B, E>();
    const int cb = c * E, katom = cb / AW, inb = cb % AW;
    const int chunk = inb >> 4, r8 = r & 7;
    int sw;
    if (AW == 128) sw = chunk ^ r8;                 // 128-byte swizzle
    else if (AW == 64) sw = chunk ^ ((r8 >> 1) & 3);  // 64-byte swizzle
    else sw = chunk ^ ((r8 >> 2) & 1);              // 32-byte swizzle
    return (r >> 3) * (8 * RB) + katom * (8 * AW) + r8 * AW + sw * 16 + (inb & 15);
}

// The culling predicate of Eq. 4 on squared norms, n2a * n2b > tau2, decided
// exactly as the FP64 expression would be.  Most candidates are settled from
// the exponent fields alone (integer work); the FP64 product is formed only
// when the exponents leave the outcome open.
__device__ __forceinline__ bool keep_product(double n2a, double n2b, double tau2)
{
    uint64_t ua = (uint64_t)__double_as_longlong(n2a);
    uint64_t ub = (uint64_t)__double_as_longlong(n2b);
    uint64_t ut = (uint64_t)__double_as_longlong(tau2);
    int ea = (int)(ua >> 52) & 0x7ff, eb = (int)(ub >> 52) & 0x7ff, et = (int)(ut >> 52) & 0x7ff;
    if (ua == 0 || ub == 0) return false;  // +0 norm: product is 0, never > tau2 >= 0
    if (ea != 0 && eb != 0 && et != 0 && ea != 0x7ff && eb != 0x7ff && et != 0x7ff) {
        // n2a in [2^(ea-1023), 2^(ea-1022)), same for n2b, tau2 in [2^(et-1023), ...)
        int lo = ea + eb - 2046;  // product in [2^lo, 2^(lo+2))
        int tl = et - 1023;
        if (lo + 2 <= tl) return false;  // RN(product) <= 2^(lo+2) <= tau2
        if (lo >= tl + 1) return true;   // RN(product) >= 2^lo > tau2
    }
    return n2a * n2b > tau2;
}

#endif  // __CUDACC__
