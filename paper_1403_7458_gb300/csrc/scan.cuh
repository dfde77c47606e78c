// scan.cuh -- exclusive prefix sums of per-group (or per-tile) counts over
// many blocks, for the culling passes (the offsets of the compacted task
// lists, Sec. 3.1 / Algorithm 1's task set laid out group by group).
//
// Three launches, every sum an integer (exact, so the result does not depend
// on the order of the additions):
//   sums  : block b adds the counts of its chunk of kChunk entries (and, in
//           the full form, the nonzero entries and three more per-entry
//           totals) into part[b];
//   top   : one block turns part[] into exclusive chunk prefixes and writes
//           the grand totals;
//   apply : block b scans its own chunk from its prefix and writes the
//           offsets (full form: also the rank of every entry among the
//           nonzero ones and, optionally, the ascending list of those).
// Roofline: HBM / L2; per entry 4 B read in `sums`, 4 B read and 8 (+4) B
// written in `apply`.
#pragma once

#include "internal.cuh"

namespace scan {

constexpr int kThreads = 256;
constexpr int kPer = 16;                   // consecutive entries per thread in `apply`
constexpr int kChunk = kThreads * kPer;    // entries per block
constexpr int kTopThreads = 1024;
constexpr int kFields = 5;                 // count, nonzero, and three totals

// Fields of part[b * kFields + f]: 0 sum of counts, 1 nonzero entries, 2-4
// sums of the extra arrays (full form).
template <bool kFull>
__global__ void __launch_bounds__(kThreads)
k_sums(const int32_t *__restrict__ stop, const int32_t *__restrict__ counts, const int32_t *__restrict__ x0,
       const int32_t *__restrict__ x1, const int32_t *__restrict__ x2, int64_t G, int64_t *__restrict__ part)
{
    __shared__ int64_t sh[kThreads / 32][kFields];
    if (stop && *stop) return;
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    int64_t v[kFields] = {0, 0, 0, 0, 0};
#pragma unroll 4
    for (int u = 0; u < kPer; u++) {
        const int64_t q = base + threadIdx.x + (int64_t)kThreads * u;  // coalesced
        if (q < G) {
            const int32_t c = counts[q];
            v[0] += c;
            if constexpr (kFull) {
                v[1] += c > 0;
                v[2] += x0[q];
                v[3] += x1[q];
                v[4] += x2[q];
            }
        }
    }
#pragma unroll
    for (int f = 0; f < kFields; f++)
        for (int o = 16; o > 0; o >>= 1) v[f] += __shfl_xor_sync(0xffffffffu, v[f], o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int f = 0; f < kFields; f++) sh[w][f] = v[f];
    __syncthreads();
    if (threadIdx.x < kFields) {
        int64_t s = 0;
        for (int q = 0; q < kThreads / 32; q++) s += sh[q][threadIdx.x];
        part[(int64_t)blockIdx.x * kFields + threadIdx.x] = s;
    }
}

// Exclusive prefixes of fields 0 and 1 over the chunks, in place; totals:
// *off_end = sum of counts; full form: tot[0..2] = sums of the extra arrays.
template <bool kFull>
__global__ void __launch_bounds__(kTopThreads)
k_top(const int32_t *__restrict__ stop, int64_t *__restrict__ part, int64_t nchunks, int64_t *__restrict__ off_end,
      int64_t *__restrict__ tot0, int64_t *__restrict__ tot1, int64_t *__restrict__ tot2)
{
    __shared__ int64_t sc[kTopThreads], sz[kTopThreads];
    __shared__ int64_t sx[3][kTopThreads / 32];
    if (stop && *stop) return;
    const int t = threadIdx.x;
    const int64_t per = (nchunks + kTopThreads - 1) / kTopThreads;
    const int64_t lo = t * per, hi = lo + per < nchunks ? lo + per : nchunks;
    int64_t c = 0, z = 0, x[3] = {0, 0, 0};
    for (int64_t b = lo; b < hi; b++) {
        c += part[b * kFields + 0];
        z += part[b * kFields + 1];
        if constexpr (kFull)
            for (int f = 0; f < 3; f++) x[f] += part[b * kFields + 2 + f];
    }
    sc[t] = c;
    sz[t] = z;
    __syncthreads();
    for (int o = 1; o < kTopThreads; o <<= 1) {  // inclusive scan of the per-thread sums
        const int64_t a = t >= o ? sc[t - o] : 0, bz = t >= o ? sz[t - o] : 0;
        __syncthreads();
        sc[t] += a;
        sz[t] += bz;
        __syncthreads();
    }
    int64_t rc = sc[t] - c, rz = sz[t] - z;
    for (int64_t b = lo; b < hi; b++) {
        const int64_t vc = part[b * kFields + 0], vz = part[b * kFields + 1];
        part[b * kFields + 0] = rc;
        part[b * kFields + 1] = rz;
        rc += vc;
        rz += vz;
    }
    if (t == kTopThreads - 1) *off_end = sc[t];
    if constexpr (kFull) {
        for (int f = 0; f < 3; f++)
            for (int o = 16; o > 0; o >>= 1) x[f] += __shfl_xor_sync(0xffffffffu, x[f], o);
        if ((t & 31) == 0)
            for (int f = 0; f < 3; f++) sx[f][t >> 5] = x[f];
        __syncthreads();
        if (t < 3) {
            int64_t s = 0;
            for (int q = 0; q < kTopThreads / 32; q++) s += sx[t][q];
            int64_t *dst = t == 0 ? tot0 : t == 1 ? tot1 : tot2;
            *dst = s;
        }
    }
}

// off[q] = exclusive prefix of counts; full form: nz[q] = rank of entry q
// among the nonzero entries, and order[rank] = q for nonzero entries (when
// order is given).
template <bool kFull>
__global__ void __launch_bounds__(kThreads)
k_apply(const int32_t *__restrict__ stop, const int32_t *__restrict__ counts, int64_t G,
        const int64_t *__restrict__ part, int64_t *__restrict__ off, int32_t *__restrict__ nz,
        int32_t *__restrict__ order)
{
    __shared__ int64_t wc[kThreads / 32], wz[kThreads / 32];
    if (stop && *stop) return;
    const int64_t q0 = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kPer;
    int32_t v[kPer];
#pragma unroll
    for (int u = 0; u < kPer; u++) v[u] = q0 + u < G ? counts[q0 + u] : 0;
    int64_t c = 0, z = 0;
#pragma unroll
    for (int u = 0; u < kPer; u++) {
        c += v[u];
        z += v[u] > 0;
    }
    // exclusive scan over the block's threads (warp shuffles, then warps)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t ic = c, iz = z;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t a = __shfl_up_sync(0xffffffffu, ic, o), b = __shfl_up_sync(0xffffffffu, iz, o);
        if (lane >= o) {
            ic += a;
            iz += b;
        }
    }
    if (lane == 31) {
        wc[w] = ic;
        wz[w] = iz;
    }
    __syncthreads();
    int64_t pc = part[(int64_t)blockIdx.x * kFields + 0], pz = part[(int64_t)blockIdx.x * kFields + 1];
    for (int q = 0; q < w; q++) {
        pc += wc[q];
        pz += wz[q];
    }
    int64_t run = pc + ic - c, zrun = pz + iz - z;
#pragma unroll
    for (int u = 0; u < kPer; u++) {
        const int64_t q = q0 + u;
        if (q < G) {
            off[q] = run;
            if constexpr (kFull) {
                nz[q] = (int32_t)zrun;
                if (order && v[u] > 0) order[zrun] = (int32_t)q;
            }
        }
        run += v[u];
        zrun += v[u] > 0;
    }
}

// Chunk partials needed for G entries (int64 words).
inline int64_t part_words(int64_t G) { return ((G + kChunk - 1) / kChunk) * kFields + kFields; }

}  // namespace scan
