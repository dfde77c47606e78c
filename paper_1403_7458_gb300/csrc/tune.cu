// tune.cu -- autotuner for batched SpAMM: leaf size (16, 32, 64; the tile of
// the tensor path is 128 / b leaf rows by one leaf column, so this also picks
// the tile shape) and tile schedule (heaviest first or row-major), chosen by
// timing spamm_multiply_batched on the caller's own matrices.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace {

struct Handles {
    std::vector<spamm_mat_t> A, B, C;
    explicit Handles(int count) : A(count, nullptr), B(count, nullptr), C(count, nullptr) {}
    ~Handles()
    {
        for (size_t m = 0; m < A.size(); m++) {
            if (B[m] && B[m] != A[m]) spamm_free(B[m]);
            if (A[m]) spamm_free(A[m]);
            if (C[m]) spamm_free(C[m]);
        }
    }
};

}  // namespace

extern "C" int spamm_autotune_batched(int32_t count, const double *const *a, const double *const *b,
                                      const int64_t *n, const double *tau, const spamm_opts_t *opts,
                                      int32_t reps, spamm_tune_t *out, void *stream)
{
    if (count < 1 || !a || !b || !n || !tau || !out || reps < 1) {
        spamm_set_error("spamm_autotune_batched: bad arguments");
        return SPAMM_E_INVAL;
    }
    for (int m = 0; m < count; m++) {
        if (!a[m] || !b[m] || n[m] < 1) {
            spamm_set_error("spamm_autotune_batched: product %d: NULL matrix or n < 1", m);
            return SPAMM_E_INVAL;
        }
    }
    memset(out, 0, sizeof(*out));
    spamm_opts_t o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    const int prec = o.prec;
    const int base_flags = o.flags & ~(SPAMM_F_TIMING | SPAMM_F_HEAVIEST);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        spamm_set_error("spamm_autotune_batched: cudaEventCreate failed");
        return SPAMM_E_CUDA;
    }
    int rc = SPAMM_OK;
    float best = INFINITY;
    const int leaves[3] = {16, 32, 64};
    for (int li = 0; li < 3 && rc == SPAMM_OK; li++) {
        const int leaf = leaves[li];
        const bool built = prec == SPAMM_FP64 || tc_mode_ok(prec, o.slices, leaf);
        const int nsched = prec == SPAMM_FP64 ? 1 : 2;
        if (!built) {
            for (int sc = 0; sc < nsched && out->tried < SPAMM_TUNE_MAX; sc++) {
                out->cand_leaf[out->tried] = leaf;
                out->cand_flags[out->tried] = sc ? SPAMM_F_HEAVIEST : 0;
                out->cand_ms[out->tried] = -1.f;
                out->tried++;
            }
            continue;
        }
        Handles h(count);
        spamm_opts_t bo = o;
        bo.leaf = leaf;
        for (int m = 0; m < count && rc == SPAMM_OK; m++) {
            rc = spamm_tree_build(a[m], n[m], n[m], 0.0, &bo, stream, &h.A[m]);
            if (rc == SPAMM_OK) {
                if (b[m] == a[m]) h.B[m] = h.A[m];
                else rc = spamm_tree_build(b[m], n[m], n[m], 0.0, &bo, stream, &h.B[m]);
            }
        }
        for (int sc = 0; sc < nsched && rc == SPAMM_OK; sc++) {
            bo.flags = base_flags | (sc ? SPAMM_F_HEAVIEST : 0);
            spamm_stats_t st;
            rc = spamm_multiply_batched(count, h.A.data(), h.B.data(), tau, h.C.data(), &bo, &st, stream);
            std::vector<float> ts;
            for (int r = 0; r < reps && rc == SPAMM_OK; r++) {
                if (cudaEventRecord(e0, s) != cudaSuccess) rc = SPAMM_E_CUDA;
                if (rc == SPAMM_OK)
                    rc = spamm_multiply_batched(count, h.A.data(), h.B.data(), tau, h.C.data(), &bo, nullptr,
                                                stream);
                if (rc == SPAMM_OK && cudaEventRecord(e1, s) != cudaSuccess) rc = SPAMM_E_CUDA;
                if (rc == SPAMM_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = SPAMM_E_CUDA;
                float ms = 0.f;
                if (rc == SPAMM_OK) cudaEventElapsedTime(&ms, e0, e1);
                ts.push_back(ms);
            }
            if (rc != SPAMM_OK) break;
            std::sort(ts.begin(), ts.end());
            const float med = ts[ts.size() / 2];
            if (out->tried < SPAMM_TUNE_MAX) {
                out->cand_leaf[out->tried] = leaf;
                out->cand_flags[out->tried] = bo.flags & SPAMM_F_HEAVIEST;
                out->cand_ms[out->tried] = med;
                out->cand_tasks[out->tried] = st.tasks;
                out->tried++;
            }
            if (med < best) {
                best = med;
                out->leaf = leaf;
                out->flags = bo.flags & SPAMM_F_HEAVIEST;
                out->ms = med;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == SPAMM_OK && out->leaf == 0) {
        spamm_set_error("spamm_autotune_batched: precision mode %d is built for no leaf size", prec);
        rc = SPAMM_E_NOTSUP;
    }
    return rc;
}
