// api.cu -- C ABI entry points: handles, leaf storage, export, errors, and
// the SpAMM product driver (cull -> leaf products -> output norms).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "internal.cuh"
#include "scan.cuh"

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512];

void spamm_set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int spamm_cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    spamm_set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    if (e == cudaErrorMemoryAllocation) return SPAMM_E_NOMEM;
    return SPAMM_E_CUDA;
}

extern "C" const char *spamm_strerror(int status)
{
    switch (status) {
    case SPAMM_OK: return "ok";
    case SPAMM_E_INVAL: return "invalid argument";
    case SPAMM_E_NOMEM: return "out of memory";
    case SPAMM_E_CUDA: return "CUDA runtime error";
    case SPAMM_E_CAPACITY: return "buffer too small";
    case SPAMM_E_TIMEOUT: return "device-side wait timed out";
    case SPAMM_E_NOCONV: return "SP2 did not converge within max_iter";
    case SPAMM_E_NOTSUP: return "option not supported";
    default: return "unknown status";
    }
}

extern "C" const char *spamm_last_error(void) { return g_err; }

static thread_local int64_t g_launches = 0;
void spamm_note_launches(int64_t k) { g_launches += k; }
int64_t spamm_launch_count() { return g_launches; }

// ---------------------------------------------------------------------------
// Memory (stream-ordered allocator)
// ---------------------------------------------------------------------------
// The library's own stream-ordered pool on each device, created on first
// use.  It keeps freed memory for the library's next allocations instead of
// returning it to the driver at every synchronisation (mapping tens of GB
// anew for every SP2 solve costs tens of milliseconds); spamm_trim() hands
// the unused part back.
static cudaMemPool_t g_pools[64] = {};
static std::mutex g_pool_mu;

static cudaError_t pool_of_current(cudaMemPool_t *pool)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> l(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if ((e = cudaMemPoolCreate(&p, &props)) != cudaSuccess) return e;
        uint64_t keep = ~uint64_t(0);
        if ((e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pools[dev] = p;
    }
    *pool = g_pools[dev];
    return cudaSuccess;
}

int spamm_alloc(void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = pool_of_current(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        spamm_set_error("cudaMallocFromPoolAsync(%zu bytes): %s", bytes, cudaGetErrorString(e));
        return SPAMM_E_NOMEM;
    }
    return SPAMM_OK;
}

extern "C" int spamm_trim(void)
{
    cudaMemPool_t pool = nullptr;
    cudaError_t e = pool_of_current(&pool);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
    if (e != cudaSuccess) return spamm_cuda_fail(e, "spamm_trim", __FILE__, __LINE__);
    return SPAMM_OK;
}

void spamm_release(void *p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

// Record an event on s; inside a stream capture as an external event node
// (a plain record there only orders the captured work and is never timed).
cudaError_t spamm_event_record(cudaEvent_t e, cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaError_t err = cudaStreamIsCapturing(s, &st);
    if (err != cudaSuccess) return err;
    return st == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                               : cudaEventRecord(e, s);
}

int spamm_num_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

static bool valid_leaf(int b) { return b == 16 || b == 32 || b == 64; }

static int depth_of(int64_t nb)
{
    int d = 0;
    while ((int64_t(1) << d) < nb) d++;
    return d;
}

namespace {

__global__ void k_iota_slots(int32_t *slot, int64_t count)
{
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < count) slot[g] = (int32_t)g;
}

// Dense row-major n x n (leading dimension lda) -> leaf storage, zero-filling
// the ragged edge.  One thread per element of the padded nb*b square.
// Dense <-> leaf layout.  Rows r of the padded Np x Np matrix are taken by
// blockIdx.y (strided), columns c by the x threads, so that consecutive
// threads touch consecutive doubles; b = 2^lb (16, 32 or 64).
// Rows r0 .. r0 + rows - 1 of the padded matrix; row r of the input is
// a[(r - r0) lda ...] (a holds those rows only).
__global__ void k_pack(const double *__restrict__ a, int64_t n, int64_t lda, int lb, int64_t nb,
                       const int32_t *__restrict__ slot, double *__restrict__ leaf, int64_t r0, int64_t rows)
{
    const int b = 1 << lb;
    const int64_t Np = nb * b;
    for (int64_t r = r0 + blockIdx.y; r < r0 + rows; r += gridDim.y) {
        const int64_t I = r >> lb, rr = r & (b - 1);
        for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < Np; c += (int64_t)gridDim.x * blockDim.x) {
            const double v = (r < n && c < n) ? a[(r - r0) * lda + c] : 0.0;
            const int32_t s = slot[I * nb + (c >> lb)];
            if (s >= 0) leaf[((int64_t)s << (2 * lb)) + (rr << lb) + (c & (b - 1))] = v;
        }
    }
}

// Rows r0 .. r0 + rows - 1 of the matrix into dst[(r - r0) ld ...].
__global__ void k_unpack(const double *__restrict__ leaf, const int32_t *__restrict__ slot,
                         int64_t n, int lb, int64_t nb, double *__restrict__ dst, int64_t ld, int64_t r0,
                         int64_t rows)
{
    const int b = 1 << lb;
    for (int64_t r = r0 + blockIdx.y; r < r0 + rows; r += gridDim.y) {
        const int64_t I = r >> lb, rr = r & (b - 1);
        for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
            const int32_t s = slot[I * nb + (c >> lb)];
            dst[(r - r0) * ld + c] = s >= 0 ? leaf[((int64_t)s << (2 * lb)) + (rr << lb) + (c & (b - 1))] : 0.0;
        }
    }
}

// Launch shape of k_pack / k_unpack over `rows` x `cols` elements.
static dim3 pack_grid(int64_t rows, int64_t cols)
{
    const int64_t gx = (cols + 255) / 256, gy = rows < 4096 ? rows : 4096;
    return dim3((unsigned)(gx < 1024 ? gx : 1024), (unsigned)(gy < 1 ? 1 : gy));
}

static int log2_leaf(int b) { return b == 16 ? 4 : b == 32 ? 5 : 6; }

// ---------------------------------------------------------------------------
// Host transfers of dense matrices in row blocks: the copies of one block run
// on a library-owned copy stream of the device while the caller's stream
// packs (or unpacks) the block before, through two device buffers of one
// block each (so the transfer overlaps the layout change, and the staging
// takes two blocks, not the whole matrix).  The lock keeps one such transfer
// per device at a time (its events are shared).
// ---------------------------------------------------------------------------
struct CopyLane {
    cudaStream_t st;
    cudaEvent_t start, copied[2], used[2];
};

static CopyLane *copy_lane(std::unique_lock<std::mutex> *lock)
{
    static std::mutex mu;
    static std::map<int, CopyLane *> lanes;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::unique_lock<std::mutex> l(mu);
    auto it = lanes.find(dev);
    if (it == lanes.end()) {
        CopyLane *c = new CopyLane();
        bool ok = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&c->start, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; i < 2 && ok; i++)
            ok = cudaEventCreateWithFlags(&c->copied[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c->used[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            spamm_set_error("copy stream: creation failed");
            return nullptr;
        }
        it = lanes.emplace(dev, c).first;
    }
    *lock = std::move(l);
    return it->second;
}

// Rows per block: a multiple of the leaf edge b, about a quarter of the
// matrix for small ones and at most 2048 rows.
static int64_t copy_block_rows(int64_t n, int b)
{
    const int64_t r = ((n + 3) / 4 + b - 1) / b * b;
    const int64_t cap = (2048 / b) * b;
    return r < b ? b : (r > cap ? cap : r);
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

unsigned blocks_for(int64_t count, int threads) { return (unsigned)((count + threads - 1) / threads); }

}  // namespace

int spamm_mat_alloc(spamm_mat_t m, int64_t n, int b, cudaStream_t s)
{
    m->n = n;
    m->b = b;
    m->nb = (n + b - 1) / b;
    m->depth = depth_of(m->nb);
    m->P = int64_t(1) << m->depth;
    m->nslots = m->nb * m->nb;
    m->stream = s;
    cudaGetDevice(&m->device);
    int rc;
    if ((rc = spamm_alloc((void **)&m->leaf, sizeof(double) * m->nslots * b * b, s))) return rc;
    if ((rc = spamm_alloc((void **)&m->slot, sizeof(int32_t) * m->nb * m->nb, s))) return rc;
    if ((rc = spamm_alloc((void **)&m->n2, sizeof(double) * tier_offset(m->depth + 1), s))) return rc;
    if ((rc = spamm_alloc((void **)&m->n2T, sizeof(double) * m->P * m->P, s))) return rc;
    SPAMM_CK(cudaMemsetAsync(m->n2, 0, sizeof(double) * tier_offset(m->depth + 1), s));
    SPAMM_CK(cudaMemsetAsync(m->n2T, 0, sizeof(double) * m->P * m->P, s));
    k_iota_slots<<<blocks_for(m->nb * m->nb, 256), 256, 0, s>>>(m->slot, m->nb * m->nb);
    SPAMM_CK_LAUNCH();
    return SPAMM_OK;
}

int spamm_mat_same_shape(spamm_mat_t a, spamm_mat_t b)
{
    return a && b && a->n == b->n && a->b == b->b;
}

int spamm_mat_dense(spamm_mat_t m) { return m && m->nslots == m->nb * m->nb; }

static void ws_free(SpammWorkspace *ws, cudaStream_t s)
{
    spamm_release(ws->tcounts, s);
    spamm_release(ws->ttasks, s);
    spamm_release(ws->tpairs, s);
    spamm_release(ws->tuseful, s);
    spamm_release(ws->td0, s);
    spamm_release(ws->toff, s);
    spamm_release(ws->torder, s);
    spamm_release(ws->tnz, s);
    spamm_release(ws->tbins, s);
    spamm_release(ws->tlist, s);
    spamm_release(ws->counts, s);
    spamm_release(ws->off, s);
    spamm_release(ws->klist, s);
    spamm_release(ws->counter, s);
    spamm_release(ws->tr_part, s);
    spamm_release(ws->exec, s);
    spamm_release(ws->scan_part, s);
    spamm_release(ws->cmask, s);
    spamm_release(ws->bgmax, s);
    spamm_release(ws->lmax, s);
    *ws = SpammWorkspace();
}

extern "C" void spamm_free(spamm_mat_t m)
{
    if (!m) return;
    cudaStream_t s = m->stream;
    spamm_release(m->leaf, s);
    spamm_release(m->slot, s);
    spamm_release(m->n2, s);
    spamm_release(m->n2T, s);
    spamm_release(m->slA, s);
    spamm_release(m->slB, s);
    spamm_release(m->tmapA, s);
    spamm_release(m->zlead, s);
    spamm_release(m->scale, s);
    ws_free(&m->ws, s);
    delete m;
}

extern "C" void spamm_release_scratch(spamm_mat_t m, void *stream)
{
    if (!m) return;
    cudaStream_t s = (cudaStream_t)stream;
    spamm_release(m->slA, s);
    spamm_release(m->slB, s);
    spamm_release(m->tmapA, s);
    spamm_release(m->zlead, s);
    m->slA = m->slB = nullptr;
    m->tmapA = nullptr;
    m->zlead = nullptr;
    m->sl_s = m->sl_e = 0;
    m->slB_transposed = -1;
    const int32_t *stop = m->ws.stop;
    ws_free(&m->ws, s);
    m->ws.stop = stop;
}

// Sparse storage: flags of the leaves kept (squared norm > drop2), their
// exclusive prefix count (one block), the compacted leaf array.
// Leaves kept by a drop threshold: flag[q] = 1 when leaf q's squared norm
// exceeds drop2 (scanned by scan.cuh into slots).
__global__ void k_keep_flags(const double *__restrict__ n2, int64_t nb, int64_t P, double drop2,
                             int32_t *__restrict__ flag)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb * nb) return;
    flag[q] = n2[(q / nb) * P + q % nb] > drop2 ? 1 : 0;
}

// slot[q] = rank of leaf q among the kept ones, or -1; a dropped leaf's
// squared norm (and its transposed copy) becomes 0.
__global__ void k_keep_slots(const int32_t *__restrict__ flag, const int64_t *__restrict__ off, int64_t nb,
                             int64_t P, int32_t *__restrict__ slot, double *__restrict__ n2, double *__restrict__ n2T)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb * nb) return;
    const int64_t i = q / nb, k = q % nb;
    if (flag[q]) {
        slot[q] = (int32_t)off[q];
    } else {
        slot[q] = -1;
        n2[i * P + k] = 0.0;
        n2T[k * P + i] = 0.0;
    }
}

__global__ void k_gather_leaves(const double *__restrict__ dense, const int32_t *__restrict__ slot, int64_t G,
                                int bb, double *__restrict__ packed)
{
    const int64_t g = blockIdx.x;
    if (g >= G || slot[g] < 0) return;
    const double2 *s = reinterpret_cast<const double2 *>(dense + g * bb);
    double2 *d = reinterpret_cast<double2 *>(packed + (int64_t)slot[g] * bb);
    for (int q = threadIdx.x; q < bb / 2; q += blockDim.x) d[q] = s[q];
}

// Keep only the leaves with squared norm > drop2 (dense handle in, sparse
// out): dropped leaves get norm 0 and the pyramid is rebuilt.
static int compact_leaves(spamm_mat_t m, double drop2, cudaStream_t s)
{
    const int64_t G = m->nb * m->nb, nch = (G + scan::kChunk - 1) / scan::kChunk;
    int32_t *flag = nullptr, *slot = nullptr;
    int64_t *off = nullptr, *part = nullptr;
    auto release = [&]() {
        spamm_release(flag, s);
        spamm_release(off, s);
        spamm_release(part, s);
    };
    int rc;
    if ((rc = spamm_alloc((void **)&flag, sizeof(int32_t) * G, s)) ||
        (rc = spamm_alloc((void **)&off, sizeof(int64_t) * (G + 1), s)) ||
        (rc = spamm_alloc((void **)&part, sizeof(int64_t) * scan::part_words(G), s)) ||
        (rc = spamm_alloc((void **)&slot, sizeof(int32_t) * G, s))) {
        release();
        return rc;
    }
    double *n2 = m->n2 + tier_offset(m->depth);
    k_keep_flags<<<blocks_for(G, 256), 256, 0, s>>>(n2, m->nb, m->P, drop2, flag);
    scan::k_sums<false><<<(unsigned)nch, scan::kThreads, 0, s>>>(nullptr, flag, nullptr, nullptr, nullptr, G, part);
    scan::k_top<false><<<1, scan::kTopThreads, 0, s>>>(nullptr, part, nch, off + G, nullptr, nullptr, nullptr);
    scan::k_apply<false><<<(unsigned)nch, scan::kThreads, 0, s>>>(nullptr, flag, G, part, off, nullptr, nullptr);
    spamm_note_launches(4);
    int64_t kept = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&kept, off + G, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        release();
        spamm_release(slot, s);
        return spamm_cuda_fail(e, "sparse leaf count", __FILE__, __LINE__);
    }
    if (kept == G) {  // nothing dropped: stay dense
        release();
        spamm_release(slot, s);
        return SPAMM_OK;
    }
    k_keep_slots<<<blocks_for(G, 256), 256, 0, s>>>(flag, off, m->nb, m->P, slot, n2, m->n2T);
    spamm_note_launches(1);
    release();
    if ((e = cudaGetLastError()) != cudaSuccess) {
        spamm_release(slot, s);
        return spamm_cuda_fail(e, "k_keep_slots", __FILE__, __LINE__);
    }
    const int bb = m->b * m->b;
    double *packed = nullptr;
    if ((rc = spamm_alloc((void **)&packed, sizeof(double) * (kept > 0 ? kept : 1) * bb, s))) {
        spamm_release(slot, s);
        return rc;
    }
    if (kept > 0) {
        k_gather_leaves<<<(unsigned)G, 256, 0, s>>>(m->leaf, slot, G, bb, packed);
        spamm_note_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            spamm_release(slot, s);
            spamm_release(packed, s);
            return spamm_cuda_fail(e, "k_gather_leaves", __FILE__, __LINE__);
        }
    }
    spamm_release(m->leaf, s);
    spamm_release(m->slot, s);
    m->leaf = packed;
    m->slot = slot;
    m->nslots = kept;
    // the leaf norms are those of the matrix as stored (a kept leaf's data
    // is unchanged, a dropped leaf's norm was set to 0): rebuild the tiers
    return launch_pyramid(m, s);
}

extern "C" int spamm_tree_build(const double *a, int64_t n, int64_t lda, double drop, const spamm_opts_t *opts,
                                void *stream, spamm_mat_t *out)
{
    if (!out) {
        spamm_set_error("spamm_tree_build: out is NULL");
        return SPAMM_E_INVAL;
    }
    *out = nullptr;
    int b = opts && opts->leaf ? opts->leaf : 32;
    if (!a || n < 1 || lda < n || !valid_leaf(b) || (n + b - 1) / b > (int64_t(1) << 15) || !(drop < 1e300)) {
        spamm_set_error("spamm_tree_build: bad arguments (n=%lld lda=%lld leaf=%d)", (long long)n,
                        (long long)lda, b);
        return SPAMM_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    spamm_mat_t m = new spamm_mat();
    int rc = spamm_mat_alloc(m, n, b, s);
    if (rc) {
        spamm_free(m);
        return rc;
    }
    const int64_t Np = m->nb * b;
    const bool host = !is_device_ptr(a);
    if (!host) {
        k_pack<<<pack_grid(Np, Np), 256, 0, s>>>(a, n, lda, log2_leaf(b), m->nb, m->slot, m->leaf, 0, Np);
        spamm_note_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            spamm_free(m);
            return spamm_cuda_fail(e, "k_pack", __FILE__, __LINE__);
        }
    } else {
        // row blocks: H2D on the copy stream, packing on s
        std::unique_lock<std::mutex> lk;
        CopyLane *cl = copy_lane(&lk);
        if (!cl) {
            spamm_free(m);
            return SPAMM_E_CUDA;
        }
        const int64_t R = copy_block_rows(n, b);
        double *buf[2] = {nullptr, nullptr};
        for (int i = 0; i < 2 && rc == SPAMM_OK; i++) rc = spamm_alloc((void **)&buf[i], sizeof(double) * R * n, s);
        cudaError_t e = cudaSuccess;
        if (rc == SPAMM_OK) {
            e = cudaEventRecord(cl->start, s);  // the buffers exist (stream-ordered allocation)
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cl->st, cl->start, 0);
            for (int64_t r0 = 0, q = 0; r0 < Np && e == cudaSuccess; r0 += R, q++) {
                const int i = (int)(q & 1);
                const int64_t rows = Np - r0 < R ? Np - r0 : R;
                if (q >= 2) e = cudaStreamWaitEvent(cl->st, cl->used[i], 0);  // block q - 2 packed
                if (e == cudaSuccess && r0 < n)
                    e = cudaMemcpy2DAsync(buf[i], sizeof(double) * n, a + r0 * lda, sizeof(double) * lda,
                                          sizeof(double) * n, (n - r0 < rows ? n - r0 : rows),
                                          cudaMemcpyHostToDevice, cl->st);
                if (e == cudaSuccess) e = cudaEventRecord(cl->copied[i], cl->st);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s, cl->copied[i], 0);
                if (e == cudaSuccess) {
                    k_pack<<<pack_grid(rows, Np), 256, 0, s>>>(buf[i], n, n, log2_leaf(b), m->nb, m->slot, m->leaf,
                                                              r0, rows);
                    spamm_note_launches(1);
                    e = cudaGetLastError();
                }
                if (e == cudaSuccess) e = cudaEventRecord(cl->used[i], s);
            }
        }
        for (int i = 0; i < 2; i++) spamm_release(buf[i], s);  // after the packs that read them (on s)
        if (rc == SPAMM_OK && e != cudaSuccess) rc = spamm_cuda_fail(e, "host-to-device blocks", __FILE__, __LINE__);
        if (rc) {
            spamm_free(m);
            return rc;
        }
    }
    if ((rc = launch_leaf_norms(m, s))) {
        spamm_free(m);
        return rc;
    }
    if (drop >= 0.0 && (rc = compact_leaves(m, drop * drop, s))) {
        spamm_free(m);
        return rc;
    }
    if (host) {
        // the caller may reuse its host buffer as soon as we return (s
        // waited for every block's copy)
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            spamm_free(m);
            return spamm_cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
        }
    }
    *out = m;
    return SPAMM_OK;
}

extern "C" int spamm_to_dense(spamm_mat_t m, double *dst, int64_t ld, void *stream)
{
    if (!m || !dst || ld < m->n) {
        spamm_set_error("spamm_to_dense: bad arguments");
        return SPAMM_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int64_t n = m->n;
    if (is_device_ptr(dst)) {
        k_unpack<<<pack_grid(n, n), 256, 0, s>>>(m->leaf, m->slot, n, log2_leaf(m->b), m->nb, dst, ld, 0, n);
        SPAMM_CK_LAUNCH();
        return SPAMM_OK;
    }
    // row blocks: unpacking on s, D2H on the copy stream
    std::unique_lock<std::mutex> lk;
    CopyLane *cl = copy_lane(&lk);
    if (!cl) return SPAMM_E_CUDA;
    const int64_t R = copy_block_rows(n, m->b);
    double *buf[2] = {nullptr, nullptr};
    int rc = SPAMM_OK;
    for (int i = 0; i < 2 && rc == SPAMM_OK; i++) rc = spamm_alloc((void **)&buf[i], sizeof(double) * R * n, s);
    cudaError_t e = cudaSuccess;
    if (rc == SPAMM_OK) {
        for (int64_t r0 = 0, q = 0; r0 < n && e == cudaSuccess; r0 += R, q++) {
            const int i = (int)(q & 1);
            const int64_t rows = n - r0 < R ? n - r0 : R;
            if (q >= 2) e = cudaStreamWaitEvent(s, cl->used[i], 0);  // block q - 2 copied out
            if (e == cudaSuccess) {
                k_unpack<<<pack_grid(rows, n), 256, 0, s>>>(m->leaf, m->slot, n, log2_leaf(m->b), m->nb, buf[i], n,
                                                            r0, rows);
                spamm_note_launches(1);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaEventRecord(cl->copied[i], s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cl->st, cl->copied[i], 0);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(dst + r0 * ld, sizeof(double) * ld, buf[i], sizeof(double) * n,
                                      sizeof(double) * n, rows, cudaMemcpyDeviceToHost, cl->st);
            if (e == cudaSuccess) e = cudaEventRecord(cl->used[i], cl->st);
        }
        // s continues once every block is on the host
        if (e == cudaSuccess) e = cudaEventRecord(cl->start, cl->st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, cl->start, 0);
    }
    for (int i = 0; i < 2; i++) spamm_release(buf[i], s);
    if (e == cudaSuccess && rc == SPAMM_OK) e = cudaStreamSynchronize(s);
    if (rc == SPAMM_OK && e != cudaSuccess) rc = spamm_cuda_fail(e, "spamm_to_dense copy", __FILE__, __LINE__);
    return rc;
}

extern "C" int spamm_norms(spamm_mat_t m, int32_t tier, double *dst, void *stream)
{
    if (!m || !dst || tier < 0 || tier > m->depth) {
        spamm_set_error("spamm_norms: bad arguments");
        return SPAMM_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int64_t W = int64_t(1) << tier;
    SPAMM_CK(cudaMemcpyAsync(dst, m->n2 + tier_offset(tier), sizeof(double) * W * W,
                             cudaMemcpyDefault, s));
    if (!is_device_ptr(dst)) SPAMM_CK(cudaStreamSynchronize(s));
    return SPAMM_OK;
}

extern "C" int spamm_info(spamm_mat_t m, int64_t *n, int32_t *leaf, int64_t *nb, int32_t *depth, int64_t *stored)
{
    if (!m) {
        spamm_set_error("spamm_info: NULL handle");
        return SPAMM_E_INVAL;
    }
    if (n) *n = m->n;
    if (leaf) *leaf = m->b;
    if (nb) *nb = m->nb;
    if (depth) *depth = m->depth;
    if (stored) *stored = m->nslots;
    return SPAMM_OK;
}

// ---------------------------------------------------------------------------
// SpAMM product
// ---------------------------------------------------------------------------
static int check_tau(double tau)
{
    if (!(tau >= 0.0) || tau > 1e300) {
        spamm_set_error("tau must be finite and >= 0 (got %g)", tau);
        return SPAMM_E_INVAL;
    }
    return SPAMM_OK;
}

int ws_reserve_groups(SpammWorkspace *ws, int64_t groups, int64_t nb, cudaStream_t s)
{
    int rc;
    if (ws->groups_cap < groups) {
        spamm_release(ws->counts, s);
        spamm_release(ws->off, s);
        ws->counts = nullptr;
        ws->off = nullptr;
        ws->groups_cap = 0;
        if ((rc = spamm_alloc((void **)&ws->counts, sizeof(int32_t) * groups, s))) return rc;
        if ((rc = spamm_alloc((void **)&ws->off, sizeof(int64_t) * (groups + 1), s))) return rc;
        ws->groups_cap = groups;
    }
    if (!ws->counter) {
        if ((rc = spamm_alloc((void **)&ws->counter, sizeof(int32_t) * 16, s))) return rc;
        SPAMM_CK(cudaMemsetAsync(ws->counter, 0, sizeof(int32_t) * 16, s));
    }
    if (!ws->exec && (rc = spamm_alloc((void **)&ws->exec, sizeof(int64_t), s))) return rc;
    if (ws->tr_cap < nb) {
        spamm_release(ws->tr_part, s);
        ws->tr_part = nullptr;
        ws->tr_cap = 0;
        if ((rc = spamm_alloc((void **)&ws->tr_part, sizeof(double) * nb, s))) return rc;
        ws->tr_cap = nb;
    }
    return SPAMM_OK;
}

int ws_reserve_scan(SpammWorkspace *ws, int64_t G, cudaStream_t s)
{
    const int64_t words = scan::part_words(G);
    if (ws->scan_cap >= words) return SPAMM_OK;
    spamm_release(ws->scan_part, s);
    ws->scan_part = nullptr;
    ws->scan_cap = 0;
    if (int rc = spamm_alloc((void **)&ws->scan_part, sizeof(int64_t) * words, s)) return rc;
    ws->scan_cap = words;
    return SPAMM_OK;
}

// Slices of the operands of A x B (tensor-core path): A's tile-major array
// and B's per-leaf array (B-role layout).  A symmetric product A == B reads
// its B leaves (the A-role layout of the transpose leaves) from the
// tile-major array itself, through tensor maps: no per-leaf array.
// out[r] = the largest of x[r P + j] (and of y[r P + j] when given) over the
// nb leaf columns j: one warp per row r.
__global__ void k_line_max(const int32_t *__restrict__ stop, const double *__restrict__ x,
                           const double *__restrict__ y, int64_t nb, int64_t P, double *__restrict__ out)
{
    if (stop && *stop) return;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= nb) return;
    double m = 0.0;
    for (int64_t j = lane; j < nb; j += 32) {
        m = fmax(m, x[r * P + j]);
        if (y) m = fmax(m, y[r * P + j]);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) out[r] = m;
}

// Slices of the operands of one product.  With prune (the slices serve this
// product alone), leaves that fail Eq. 4 against their largest partner are
// not sliced: an A leaf (i, k) against max_j ||B_kj||^2, a B leaf (k, j)
// against max_i ||A_ik||^2 (symmetric: both, from the norms and their
// transposes).  No kept triple involves such a leaf (the product of its norm
// with any partner's is at most the product with the largest).
static int slice_operands(spamm_mat_t A, spamm_mat_t B, int sl, int el, int symm, cudaStream_t s,
                          const int32_t *stop, bool unit, bool fsplit, SpammWorkspace *ws = nullptr,
                          double tau = 0.0)
{
    const double *keep_a = nullptr, *keep_b = nullptr;
    const double tau2 = tau * tau;
    // (A == B without symmetry: one leading-zero count per leaf serves both
    // roles, so every leaf either role needs must be sliced: no pruning)
    if (ws && !(A == B && !symm)) {
        const int64_t nb = A->nb;
        int rc;
        if (ws->lmax_cap < 2 * nb) {
            spamm_release(ws->lmax, s);
            ws->lmax = nullptr;
            ws->lmax_cap = 0;
            if ((rc = spamm_alloc((void **)&ws->lmax, sizeof(double) * 2 * nb, s))) return rc;
            ws->lmax_cap = 2 * nb;
        }
        const unsigned blocks = (unsigned)((nb + 7) / 8);
        const double *nB = B->n2 + tier_offset(B->depth);
        if (A == B && symm) {
            k_line_max<<<blocks, 256, 0, s>>>(stop, nB, B->n2T, nb, B->P, ws->lmax);
            SPAMM_CK_LAUNCH();
            keep_a = ws->lmax;
        } else {
            k_line_max<<<blocks, 256, 0, s>>>(stop, nB, nullptr, nb, B->P, ws->lmax);  // rows of B
            SPAMM_CK_LAUNCH();
            k_line_max<<<blocks, 256, 0, s>>>(stop, A->n2T, nullptr, nb, A->P, ws->lmax + nb);  // columns of A
            SPAMM_CK_LAUNCH();
            keep_a = ws->lmax;
            keep_b = ws->lmax + nb;
        }
    }
    if (A == B && symm) {
        if (int rc = launch_slices(A, sl, el, true, false, false, s, stop, unit, fsplit, keep_a, nullptr, tau2))
            return rc;
        return slices_tmaps(A, s);
    }
    if (A == B) return launch_slices(A, sl, el, true, true, true, s, stop, unit, fsplit);
    int rc = launch_slices(A, sl, el, true, false, false, s, stop, unit, fsplit, keep_a, nullptr, tau2);
    if (rc) return rc;
    return launch_slices(B, sl, el, false, true, true, s, stop, unit, fsplit, nullptr, keep_b, tau2);
}

// Device-side error words of a product's workspace (blocking read): list
// overflow of the cull (counter 8) and a bounded wait that gave up in the
// tensor-core kernel (counter 9).  Both are cleared after reading, and so is
// counter 11, the tensor-core products' count of output elements with a
// diagonal sum at or beyond 2^24 (kept in ws->last_rounded).
int ws_check_errors(SpammWorkspace *ws, cudaStream_t s)
{
    if (!ws->counter) return SPAMM_OK;
    int32_t w[4] = {0, 0, 0, 0};
    SPAMM_CK(cudaMemcpyAsync(w, ws->counter + 8, sizeof(w), cudaMemcpyDeviceToHost, s));
    SPAMM_CK(cudaStreamSynchronize(s));
    ws->last_rounded = w[3];
    if (w[3]) SPAMM_CK(cudaMemsetAsync(ws->counter + 11, 0, sizeof(int32_t), s));
    if (!w[0] && !w[1]) return SPAMM_OK;
    SPAMM_CK(cudaMemsetAsync(ws->counter + 8, 0, sizeof(int32_t) * 2, s));
    if (w[1]) {
        spamm_set_error("tensor-core leaf products: a device-side wait timed out");
        return SPAMM_E_TIMEOUT;
    }
    spamm_set_error("task list overflow in the cull");
    return SPAMM_E_CAPACITY;
}

int spamm_multiply_into(spamm_mat_t A, spamm_mat_t B, double tau, spamm_mat_t C,
                        const spamm_opts_t *opts, double *tr_part, cudaStream_t s,
                        bool need_total, int64_t *tasks_out, bool build_pyramid,
                        cudaEvent_t *ev, int sym, bool slices_ready, bool zero_empty, bool mirror)
{
    int prec = opts ? opts->prec : SPAMM_FP64;
    if (ev) SPAMM_CK(spamm_event_record(ev[0], s));
    SpammWorkspace *ws = &C->ws;
    int rc = ws_reserve_groups(ws, A->nb * A->nb, A->nb, s);
    if (rc) return rc;
    int64_t total = -1;
    if (prec == SPAMM_FP64) {
        rc = spamm_cull(A, B, tau, ws, A->nb, A->P, s, need_total, &total);
        if (rc) return rc;
        ws->task_total = ws->off + A->nb * A->nb;
        ws->pair_units = ws->exec;  // leaf products formed (half of them when symmetric)
        if (ev) SPAMM_CK(spamm_event_record(ev[1], s));
        rc = launch_gemm_fp64(A, B, C, ws, tr_part, s, (sym && A == B) ? 1 : 0);
    } else if (prec_is_tc(prec)) {
        const int sl = prec_slices(prec, opts ? opts->slices : 0);
        const int el = prec_elem(prec);
        const bool fsplit = prec_float_split(prec);
        const int symm = (sym && A == B) ? 1 : 0;
        const bool unit = opts && (opts->flags & kFlagUnitScale);
        // slices first: the tile cull reads each leaf's leading zero slices
        if (slices_ready) {
            // the caller already wrote A's slices
        } else if ((rc = slice_operands(A, B, sl, el, symm, s, ws->stop, unit, fsplit, ws, tau))) {
            return rc;
        }
        const bool heavy = opts && (opts->flags & SPAMM_F_HEAVIEST);
        if ((rc = tc_tile_cull(A, B, tau, ws, symm, sl, s, heavy))) return rc;
        if (zero_empty && (rc = tc_zero_empty_tiles(C, ws, s))) return rc;
        ws->tmirror = mirror ? 1 : 0;
        ws->tskip_idle = zero_empty ? 0 : 1;
        if (ev) SPAMM_CK(spamm_event_record(ev[1], s));
        rc = launch_gemm_tc(A, B, C, ws, tr_part, sl, el, s, fsplit);
        if (rc) return rc;
        const int64_t T = ws->tT;
        ws->task_total = ws->toff + T + 1;
        ws->pair_units = ws->toff + T + 3;
        if (need_total) {
            int64_t both[3];
            SPAMM_CK(cudaMemcpyAsync(both, ws->toff + T, sizeof(int64_t) * 3, cudaMemcpyDeviceToHost, s));
            SPAMM_CK(cudaStreamSynchronize(s));
            total = both[1];
            ws->last_items = both[0];
            ws->last_pairs = both[2];
        }
    } else {
        spamm_set_error("precision mode %d not built", prec);
        rc = SPAMM_E_NOTSUP;
    }
    if (rc) return rc;
    if (ev) SPAMM_CK(spamm_event_record(ev[2], s));
    C->tiers_ok = build_pyramid;
    if (build_pyramid) {
        // the FP64 epilogue already wrote C's leaf norms; the tensor-core
        // epilogue does not, so they are formed from the stored leaves
        rc = prec == SPAMM_FP64 ? launch_pyramid(C, s) : launch_leaf_norms(C, s);
        if (rc) return rc;
    }
    if (ev) SPAMM_CK(spamm_event_record(ev[3], s));
    if (tasks_out) *tasks_out = total;
    return SPAMM_OK;
}

extern "C" int spamm_multiply(spamm_mat_t A, spamm_mat_t B, double tau, spamm_mat_t *C,
                              const spamm_opts_t *opts, spamm_stats_t *stats, void *stream)
{
    if (!A || !B || !C || !spamm_mat_same_shape(A, B)) {
        spamm_set_error("spamm_multiply: NULL handle or shape mismatch");
        return SPAMM_E_INVAL;
    }
    int rc = check_tau(tau);
    if (rc) return rc;
    int prec = opts ? opts->prec : SPAMM_FP64;
    if (prec != SPAMM_FP64 && !prec_is_tc(prec)) {
        spamm_set_error("spamm_multiply: unknown precision mode %d", prec);
        return SPAMM_E_NOTSUP;
    }
    if (prec_is_tc(prec) && !tc_mode_ok(prec, opts ? opts->slices : 0, A->b)) {
        spamm_set_error("spamm_multiply: tensor-core mode %d with %d slices at leaf %d not built (exact "
                        "slices 3..7, slices x leaf <= 256)",
                        prec, opts ? opts->slices : 0, A->b);
        return SPAMM_E_NOTSUP;
    }
    cudaStream_t s = (cudaStream_t)stream;
    bool created = false;
    if (*C == nullptr) {
        spamm_mat_t m = new spamm_mat();
        if ((rc = spamm_mat_alloc(m, A->n, A->b, s))) {
            spamm_free(m);
            return rc;
        }
        *C = m;
        created = true;
    } else if (!spamm_mat_same_shape(*C, A) || *C == A || *C == B || !spamm_mat_dense(*C)) {
        spamm_set_error("spamm_multiply: C must match A's shape, store every leaf and not alias A or B");
        return SPAMM_E_INVAL;
    }
    bool timing = stats && opts && (opts->flags & SPAMM_F_TIMING);
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (timing)
        for (int q = 0; q < 4 && rc == SPAMM_OK; q++)
            if (cudaEventCreate(&ev[q]) != cudaSuccess) rc = SPAMM_E_CUDA;
    int64_t total = -1;
    if (rc == SPAMM_OK)
        rc = spamm_multiply_into(A, B, tau, *C, opts, nullptr, s, stats != nullptr, &total, true,
                                 timing ? ev : nullptr);
    if (rc == SPAMM_OK && stats) {
        int64_t nb = A->nb;
        double b3 = double(A->b) * A->b * A->b;
        stats->tasks = total;
        stats->candidates = nb * nb * nb;
        stats->flops_useful = 2.0 * b3 * double(total);
        stats->flops_issued = stats->flops_useful;
        if (prec_is_tc(prec)) {
            stats->flops_issued = 2.0 * 128 * double(A->b) * A->b * double((*C)->ws.last_pairs);
        }
        stats->ms_cull = stats->ms_gemm = stats->ms_norm = 0.f;
        rc = ws_check_errors(&(*C)->ws, s);
        stats->sums_rounded = (*C)->ws.last_rounded;
        if (timing && rc == SPAMM_OK) {
            cudaError_t e = cudaEventSynchronize(ev[3]);
            if (e != cudaSuccess) rc = spamm_cuda_fail(e, "cudaEventSynchronize", __FILE__, __LINE__);
            cudaEventElapsedTime(&stats->ms_cull, ev[0], ev[1]);
            cudaEventElapsedTime(&stats->ms_gemm, ev[1], ev[2]);
            cudaEventElapsedTime(&stats->ms_norm, ev[2], ev[3]);
        }
    }
    for (int q = 0; q < 4; q++)
        if (ev[q]) cudaEventDestroy(ev[q]);
    if (rc && created) {
        spamm_free(*C);
        *C = nullptr;
    }
    return rc;
}

// ---------------------------------------------------------------------------
// Auxiliary streams of the current device for the per-product preparation of
// batched products (created once, kept for the life of the process).  The
// returned lock serialises batched calls on the device while they enqueue.
// ---------------------------------------------------------------------------
constexpr int kAuxStreams = 4;
struct AuxStreams {
    cudaStream_t st[kAuxStreams];
    cudaEvent_t fork;
    cudaEvent_t join[kAuxStreams];
};

static AuxStreams *aux_streams(std::unique_lock<std::mutex> *lock)
{
    static std::mutex mu;
    static std::map<int, AuxStreams *> sets;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::unique_lock<std::mutex> l(mu);
    auto it = sets.find(dev);
    if (it == sets.end()) {
        AuxStreams *a = new AuxStreams();
        bool ok = cudaEventCreateWithFlags(&a->fork, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; i < kAuxStreams && ok; i++) {
            ok = cudaStreamCreateWithFlags(&a->st[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&a->join[i], cudaEventDisableTiming) == cudaSuccess;
        }
        if (!ok) {
            spamm_set_error("auxiliary streams: creation failed");
            return nullptr;  // (what was created stays; only on a failing device)
        }
        it = sets.emplace(dev, a).first;
    }
    *lock = std::move(l);
    return it->second;
}

// ---------------------------------------------------------------------------
// Batched products: per product slicing / cull, then ONE leaf-product launch
// per group of at most kMaxBatch products, then per product output norms.
// ---------------------------------------------------------------------------
extern "C" int spamm_multiply_batched(int32_t count, const spamm_mat_t *A, const spamm_mat_t *B,
                                      const double *tau, spamm_mat_t *C, const spamm_opts_t *opts,
                                      spamm_stats_t *stats, void *stream)
{
    if (count < 0 || (count > 0 && (!A || !B || !tau || !C))) {
        spamm_set_error("spamm_multiply_batched: bad arguments");
        return SPAMM_E_INVAL;
    }
    if (stats) memset(stats, 0, sizeof(*stats));
    if (count == 0) return SPAMM_OK;
    const int prec = opts ? opts->prec : SPAMM_FP64;
    const int leaf = A[0] ? A[0]->b : 0;
    int rc;
    for (int m = 0; m < count; m++) {
        if (!A[m] || !B[m] || !spamm_mat_same_shape(A[m], B[m]) || A[m]->b != leaf) {
            spamm_set_error("spamm_multiply_batched: product %d: NULL handle, shape mismatch or a leaf size "
                            "other than the batch's",
                            m);
            return SPAMM_E_INVAL;
        }
        if ((rc = check_tau(tau[m]))) return rc;
        if (C[m] && (!spamm_mat_same_shape(C[m], A[m]) || C[m] == A[m] || C[m] == B[m] || !spamm_mat_dense(C[m]))) {
            spamm_set_error("spamm_multiply_batched: C[%d] must match A[%d]'s shape and not alias A or B", m, m);
            return SPAMM_E_INVAL;
        }
        for (int q = 0; q < count && C[m]; q++) {
            if (q != m && (C[q] == C[m] || A[q] == C[m] || B[q] == C[m])) {
                spamm_set_error("spamm_multiply_batched: C[%d] is also another product's input or output", m);
                return SPAMM_E_INVAL;
            }
        }
    }
    if (prec != SPAMM_FP64 && !tc_mode_ok(prec, opts ? opts->slices : 0, leaf)) {
        spamm_set_error("spamm_multiply_batched: precision mode %d (leaf %d, slices %d) not built", prec, leaf,
                        opts ? opts->slices : 0);
        return SPAMM_E_NOTSUP;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<char> created(count, 0);
    for (int m = 0; m < count && rc == SPAMM_OK; m++) {
        if (C[m]) continue;
        spamm_mat_t c = new spamm_mat();
        if ((rc = spamm_mat_alloc(c, A[m]->n, leaf, s))) {
            spamm_free(c);
            break;
        }
        C[m] = c;
        created[m] = 1;
    }
    // larger products first: with tiles handed out dynamically this is
    // longest-processing-time-first scheduling across the batch
    std::vector<int> ord(count);
    for (int m = 0; m < count; m++) ord[m] = m;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return A[x]->nb > A[y]->nb; });
    const bool timing = stats && opts && (opts->flags & SPAMM_F_TIMING);
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (timing)
        for (int q = 0; q < 4 && rc == SPAMM_OK; q++)
            if (cudaEventCreate(&ev[q]) != cudaSuccess) rc = SPAMM_E_CUDA;
    const bool tcp = prec != SPAMM_FP64;
    const int sl = tcp ? prec_slices(prec, opts ? opts->slices : 0) : 0;
    const int el = tcp ? prec_elem(prec) : 0;
    const bool fsplit = tcp && prec_float_split(prec);
    const bool unit = opts && (opts->flags & kFlagUnitScale);
    std::vector<spamm_mat_t> a(count), b(count), c(count);
    std::vector<SpammWorkspace *> w(count);
    for (int q = 0; q < count; q++) {
        a[q] = A[ord[q]];
        b[q] = B[ord[q]];
        c[q] = C[ord[q]];
        w[q] = &C[ord[q]]->ws;
    }
    if (rc == SPAMM_OK && timing && spamm_event_record(ev[0], s) != cudaSuccess) rc = SPAMM_E_CUDA;
    // per product: slicing and culling, spread over the auxiliary streams
    // (forked from s and joined back before the leaf products); products that
    // share an input handle stay on one stream (they write the same slices)
    std::unique_lock<std::mutex> aux_lock;
    AuxStreams *aux = rc == SPAMM_OK ? aux_streams(&aux_lock) : nullptr;
    if (rc == SPAMM_OK && !aux) rc = SPAMM_E_CUDA;
    std::vector<int> lane_of(count, 0);
    if (rc == SPAMM_OK) {
        std::vector<int> root(count), lane_of_root(count, -1);
        int next = 0;
        for (int q = 0; q < count; q++) {
            root[q] = q;
            for (int p2 = 0; p2 < q; p2++)
                if (a[q] == a[p2] || a[q] == b[p2] || b[q] == a[p2] || b[q] == b[p2]) {
                    root[q] = root[p2];
                    break;
                }
            if (lane_of_root[root[q]] < 0) lane_of_root[root[q]] = next++ % kAuxStreams;
            lane_of[q] = lane_of_root[root[q]];
        }
        if (cudaEventRecord(aux->fork, s) != cudaSuccess) rc = SPAMM_E_CUDA;
        for (int i = 0; i < kAuxStreams && rc == SPAMM_OK; i++)
            if (cudaStreamWaitEvent(aux->st[i], aux->fork, 0) != cudaSuccess) rc = SPAMM_E_CUDA;
    }
    for (int q = 0; q < count && rc == SPAMM_OK; q++) {
        const int64_t nb = a[q]->nb;
        cudaStream_t sq = aux->st[lane_of[q]];
        if ((rc = ws_reserve_groups(w[q], nb * nb, nb, sq))) break;
        if (!tcp) {
            rc = spamm_cull(a[q], b[q], tau[ord[q]], w[q], nb, a[q]->P, sq, false, nullptr, true);
            w[q]->task_total = w[q]->off + nb * nb;
            w[q]->pair_units = nullptr;
        } else {
            rc = slice_operands(a[q], b[q], sl, el, 0, sq, nullptr, unit, fsplit);
            if (rc == SPAMM_OK)
                rc = tc_tile_cull(a[q], b[q], tau[ord[q]], w[q], 0, sl, sq,
                                  opts && (opts->flags & SPAMM_F_HEAVIEST));
            if (rc == SPAMM_OK) rc = tc_zero_empty_tiles(c[q], w[q], sq);
            w[q]->tskip_idle = 0;  // every output leaf is written
        }
    }
    if (aux) {
        // join (also after a failure, so that no forked stream is left dangling)
        for (int i = 0; i < kAuxStreams; i++) {
            cudaEventRecord(aux->join[i], aux->st[i]);
            cudaStreamWaitEvent(s, aux->join[i], 0);
        }
    }
    if (rc == SPAMM_OK && timing && spamm_event_record(ev[1], s) != cudaSuccess) rc = SPAMM_E_CUDA;
    for (int q0 = 0; q0 < count && rc == SPAMM_OK; q0 += kMaxBatch) {
        const int k = count - q0 < kMaxBatch ? count - q0 : kMaxBatch;
        int32_t *ctr = w[q0]->counter;
        rc = tcp ? launch_gemm_tc_batched(k, &a[q0], &b[q0], &c[q0], &w[q0], sl, el, s, fsplit, ctr)
                 : launch_gemm_fp64_batched(k, &a[q0], &b[q0], &c[q0], &w[q0], s, ctr);
    }
    if (rc == SPAMM_OK && timing && spamm_event_record(ev[2], s) != cudaSuccess) rc = SPAMM_E_CUDA;
    // output norms per product, again spread over the auxiliary streams
    if (rc == SPAMM_OK) {
        if (cudaEventRecord(aux->fork, s) != cudaSuccess) rc = SPAMM_E_CUDA;
        for (int i = 0; i < kAuxStreams && rc == SPAMM_OK; i++)
            if (cudaStreamWaitEvent(aux->st[i], aux->fork, 0) != cudaSuccess) rc = SPAMM_E_CUDA;
        for (int q = 0; q < count && rc == SPAMM_OK; q++) {
            cudaStream_t sq = aux->st[lane_of[q]];
            rc = tcp ? launch_leaf_norms(c[q], sq) : launch_pyramid(c[q], sq);
        }
        for (int i = 0; i < kAuxStreams; i++) {
            cudaEventRecord(aux->join[i], aux->st[i]);
            cudaStreamWaitEvent(s, aux->join[i], 0);
        }
    }
    if (rc == SPAMM_OK && timing && spamm_event_record(ev[3], s) != cudaSuccess) rc = SPAMM_E_CUDA;
    if (rc == SPAMM_OK && stats) {
        // totals (one blocking read per product) and the device error words
        for (int q = 0; q < count && rc == SPAMM_OK; q++) {
            const int64_t nb = a[q]->nb;
            int64_t v[4] = {0, 0, 0, 0};
            cudaError_t e;
            if (tcp) {
                e = cudaMemcpyAsync(v, w[q]->toff + w[q]->tT, sizeof(int64_t) * 4, cudaMemcpyDeviceToHost, s);
            } else {
                e = cudaMemcpyAsync(v + 1, w[q]->off + nb * nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                rc = spamm_cuda_fail(e, "batched totals", __FILE__, __LINE__);
                break;
            }
            const double b3 = double(leaf) * leaf * leaf;
            stats->tasks += v[1];
            stats->candidates += nb * nb * nb;
            stats->flops_useful += 2.0 * b3 * double(v[1]);
            stats->flops_issued += tcp ? 2.0 * 128 * double(leaf) * leaf * double(v[2]) : 2.0 * b3 * double(v[1]);
            rc = ws_check_errors(w[q], s);
            const int64_t r = (int64_t)stats->sums_rounded + w[q]->last_rounded;
            stats->sums_rounded = (int32_t)(r < INT32_MAX ? r : INT32_MAX);
        }
        if (rc == SPAMM_OK && timing) {
            cudaError_t e = cudaEventSynchronize(ev[3]);
            if (e != cudaSuccess) rc = spamm_cuda_fail(e, "cudaEventSynchronize", __FILE__, __LINE__);
            cudaEventElapsedTime(&stats->ms_cull, ev[0], ev[1]);
            cudaEventElapsedTime(&stats->ms_gemm, ev[1], ev[2]);
            cudaEventElapsedTime(&stats->ms_norm, ev[2], ev[3]);
        }
    }
    for (int q = 0; q < 4; q++)
        if (ev[q]) cudaEventDestroy(ev[q]);
    if (rc) {
        for (int m = 0; m < count; m++)
            if (created[m]) {
                spamm_free(C[m]);
                C[m] = nullptr;
            }
    }
    return rc;
}

extern "C" int spamm_task_list(spamm_mat_t A, spamm_mat_t B, double tau, int64_t *off_host,
                               uint32_t *k_host, int64_t cap, int64_t *ntasks, void *stream)
{
    if (!A || !B || !spamm_mat_same_shape(A, B) || !off_host || !ntasks || cap < 0 ||
        (cap > 0 && !k_host)) {
        spamm_set_error("spamm_task_list: bad arguments");
        return SPAMM_E_INVAL;
    }
    int rc = check_tau(tau);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    SpammWorkspace ws;
    int64_t G = A->nb * A->nb;
    if ((rc = ws_reserve_groups(&ws, G, A->nb, s)) == SPAMM_OK) {
        int64_t total = -1;
        rc = spamm_cull(A, B, tau, &ws, A->nb, A->P, s, true, &total);
        if (rc == SPAMM_OK) {
            *ntasks = total;
            cudaError_t e = cudaMemcpyAsync(off_host, ws.off, sizeof(int64_t) * (G + 1),
                                            cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && total <= cap && total > 0)
                e = cudaMemcpyAsync(k_host, ws.klist, sizeof(uint32_t) * total,
                                    cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = spamm_cuda_fail(e, "task list copy", __FILE__, __LINE__);
            else if (total > cap) {
                spamm_set_error("spamm_task_list: %lld tasks, capacity %lld", (long long)total,
                                (long long)cap);
                rc = SPAMM_E_CAPACITY;
            }
        }
    }
    ws_free(&ws, s);
    return rc;
}
