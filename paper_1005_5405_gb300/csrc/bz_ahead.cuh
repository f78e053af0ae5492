// bz_ahead.cuh -- the shared sample plans of many steps, built ahead in one
// launch per kernel class.
//
// A step's plan (its Monte Carlo sample set, Sec. 4.2 / Algorithm 2, the
// active-node numbering, the destination-sorted term records and their
// bank-aware order) depends on the step number only, never on the state.
// So the plans of K consecutive steps are built together: every kernel of
// the plan chain takes a plan slot in its grid's y (or z, or x) index, and
// the step n is kept in slot n mod K.  Each step then copies its slot into
// the arrays the active-node kernel and its fallback read (k_ahead_take).
// The per-step chain of small, latency-bound launches leaves the critical
// path of the step, and the term order can afford whole runs (no chunks).
#pragma once
#include "bz_lazy.cuh"

namespace bzk {

struct AheadPlans {
    int K;                          // slots
    int nt, nvt, mcap, osh;
    int4 *idx;                      // K x nt: node indices of the samples
    PlanA<float, int> *pa;          // K x nt: their first two nodes and weights
    ushort4 *qc;                    // K x nt: compact indices
    int *flag, *cidx, *act;         // K x nvt
    uint32_t *mask;                 // K x nvt/32
    int *wpre;                      // K x nvt/32
    int *meta;                      // K x kLzMetaSize
    int *count, *cursor, *rowend;   // K x nvt
    int *dest0;                     // K x kLzRoleT
    uint2 *rec;                     // K x recn term records
    int64_t recn;
    unsigned long long *cnt;        // K x 2: samples with a node outside the box, near a face
};

__device__ __forceinline__ int ahead_slot(const AheadPlans &A, int64_t step0, int y)
{
    return (int)((step0 + y) % A.K);
}

// Samples of steps step0 + blockIdx.y (one thread per sample), their marks
// on the active nodes and the per-slot counts of out-of-box and near-face
// samples.  g: the handle's geometry in logical node order (swz = 0).  The
// FP32 sampler of the per-cell sets draws them (uniform velocity grids; a
// sample near a velocity-cell face is drawn again in FP64), so the node
// indices are those of the FP64 computation and W carries FP32 rounding.
__global__ void k_ahead_plan(Geo g, AheadPlans A, int64_t step0)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t step = step0 + blockIdx.y;
    const int s = ahead_slot(A, step0, blockIdx.y);
    const bool act = l < A.nt;
    SampleOut o = {};
    if (act) {
        o = draw_sample_cell<float>(g, step, 0xFFFFFFFFu, (uint32_t)l);
        const int64_t off = (int64_t)s * A.nt + l;
        A.idx[off] = make_int4(o.idx[0], o.idx[1], o.idx[2], o.idx[3]);
        A.pa[off] = make_plan_a<float, int>(o.idx[0], o.idx[1], o.W);
        int *fl = A.flag + (int64_t)s * A.nvt;
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (o.idx[r] >= 0) fl[o.idx[r]] = 1;
    }
    const unsigned mo = __ballot_sync(0xFFFFFFFFu, act && o.outside);
    const unsigned mn = __ballot_sync(0xFFFFFFFFu, act && o.near);
    if ((threadIdx.x & 31) == 0) {
        if (mo) atomicAdd(A.cnt + 2 * s, (unsigned long long)__popc(mo));
        if (mn) atomicAdd(A.cnt + 2 * s + 1, (unsigned long long)__popc(mn));
    }
}

// Compact numbering of the marked nodes: one CTA of 1024 threads per step.
__global__ void __launch_bounds__(1024) k_ahead_scan(AheadPlans A, int64_t step0)
{
    const int s = ahead_slot(A, step0, blockIdx.x);
    const int64_t v = (int64_t)s * A.nvt, w = (int64_t)s * (A.nvt / 32);
    lz_scan_block(A.nvt, A.mcap, A.flag + v, A.cidx + v, A.act + v, A.mask + w, A.wpre + w,
                  A.meta + s * kLzMetaSize, nullptr);
}

__global__ void k_ahead_remap(AheadPlans A, int64_t step0)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= A.nt) return;
    const int s = ahead_slot(A, step0, blockIdx.y);
    const int64_t t = (int64_t)s * A.nt, v = (int64_t)s * A.nvt;
    lz_remap_one(l, A.idx + t, A.cidx + v, A.qc + t, A.count + v);
}

// Sorted order of the collision terms: one CTA of 1024 threads per step.
__global__ void __launch_bounds__(1024) k_ahead_lscan(AheadPlans A, int64_t step0)
{
    const int s = ahead_slot(A, step0, blockIdx.x);
    const int64_t v = (int64_t)s * A.nvt;
    lz_lscan_block(kLzRoleT, A.osh, A.count + v, A.cursor + v, A.rowend + v, A.meta + s * kLzMetaSize,
                   A.rec + s * A.recn, A.dest0 + s * kLzRoleT);
}

__global__ void k_ahead_lfill(AheadPlans A, int64_t step0)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= A.nt) return;
    const int s = ahead_slot(A, step0, blockIdx.y);
    const int64_t t = (int64_t)s * A.nt, v = (int64_t)s * A.nvt;
    lz_lfill_one(l, kLzRoleT, A.osh, A.qc + t, A.pa + t, A.cursor + v, A.rowend + v,
                 A.meta + s * kLzMetaSize, A.rec + s * A.recn, A.dest0 + s * kLzRoleT);
}

// The plan of step `step` into the arrays the step reads, and its counters
// into the handle's statistics (as the per-step chain records them: [1]
// out-of-box samples, [2] near-face samples, [5] overflowing steps, [6]
// active nodes).  Thread i0 of `stride` threads; the thread with i0 == 0
// records the counters.
__device__ __forceinline__ void ahead_take(const AheadPlans &A, int64_t step, int4 *__restrict__ idx,
                                           PlanA<float, int> *__restrict__ pa, int *__restrict__ meta,
                                           uint32_t *__restrict__ mask, int *__restrict__ wpre,
                                           int *__restrict__ act, uint2 *__restrict__ rec,
                                           int *__restrict__ dest0, unsigned long long *__restrict__ stats,
                                           int64_t i0, int64_t stride)
{
    const int s = (int)(step % A.K);
    const int *sm = A.meta + s * kLzMetaSize;
    const int M = min(sm[0], A.nvt), C = sm[3];
    const int64_t t0 = (int64_t)s * A.nt, v0 = (int64_t)s * A.nvt, w0 = (int64_t)s * (A.nvt / 32);
    for (int64_t i = i0; i < A.nt; i += stride) {
        idx[i] = A.idx[t0 + i];
        pa[i] = A.pa[t0 + i];
    }
    for (int64_t i = i0; i < A.nvt / 32; i += stride) {
        mask[i] = A.mask[w0 + i];
        wpre[i] = A.wpre[w0 + i];
    }
    for (int64_t i = i0; i < M; i += stride) act[i] = A.act[v0 + i];
    const int64_t nrec = min((int64_t)C * kLzRoleT, A.recn);
    const uint2 *sr = A.rec + s * A.recn;
    for (int64_t i = i0; i < nrec; i += stride) rec[i] = sr[i];
    for (int64_t i = i0; i < kLzRoleT; i += stride) dest0[i] = A.dest0[(int64_t)s * kLzRoleT + i];
    if (i0 < kLzMetaSize) meta[i0] = sm[i0];
    if (i0 == 0 && stats) {
        stats[1] += A.cnt[2 * s];
        stats[2] += A.cnt[2 * s + 1];
        if (sm[1]) stats[5] += 1ull;
        stats[6] = (unsigned long long)sm[0];
    }
}

// The plan of the current step (*stepp) of one handle.  Grid-stride over
// every array.
__global__ void k_ahead_take(AheadPlans A, const int64_t *__restrict__ stepp, int4 *__restrict__ idx,
                             PlanA<float, int> *__restrict__ pa, int *__restrict__ meta,
                             uint32_t *__restrict__ mask, int *__restrict__ wpre, int *__restrict__ act,
                             uint2 *__restrict__ rec, int *__restrict__ dest0,
                             unsigned long long *__restrict__ stats)
{
    ahead_take(A, *stepp, idx, pa, meta, mask, wpre, act, rec, dest0, stats,
               (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

}  // namespace bzk
