// bz_batch.cuh -- many cavity instances advanced by one launch per kernel class.
//
// Each instance is a complete problem of its own (grid, velocity box, Kn,
// lid, samples, Philox instance word); all are FP32 with a multiple-of-4
// velocity axis so that they run on the FP32 per-cell code of bz_cell4.cuh.
// The work of a step is flattened over the instances: faces (walls), samples
// (sampling and the scatter list) and cells (the per-cell step).  A flat index
// is mapped to its instance through prefix arrays.  The state of instance i at
// step n lives in h[n & 1] and every kernel reads n from the instance's device
// step counter, so one captured step replays correctly any number of times.
#pragma once

#include "bz_ahead.cuh"

namespace bzk {

struct BInst {
    Geo g;                       // geometry and tables of the instance
    Map4 map[2];                 // quad mapping for 512- and 1024-thread CTAs
    float *h[2];                 // state buffers, h[step & 1] is current
    float *ghost;
    double *nw;
    ushort4 *pidx;
    PlanA<float, uint16_t> *pa;
    int *sc_count, *sc_cursor, *sc_meta;
    uint32_t *sc_ent;
    double *mom;
    int64_t *step;
};

// Largest i with pre[i] <= k (pre[0] = 0, pre[n] = total).
__device__ __forceinline__ int inst_of(const int *__restrict__ pre, int n, int k)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Walls of every face of every instance: one CTA per face.
__global__ void kb_walls(const BInst *__restrict__ inst, const int *__restrict__ face_pre, int n)
{
    __shared__ double red[kMaxWarps * kRedSlots];
    __shared__ double tot[4];
    __shared__ double s_nw;
    __shared__ float sA[kMaxN], sv[kMaxN];
    const int i = inst_of(face_pre, n, blockIdx.x);
    const BInst &b = inst[i];
    const int64_t step = *b.step;
    walls_face<float>(b.g, step, b.h[step & 1], b.ghost, b.nw, nullptr,
                      blockIdx.x - face_pre[i], sA, sv, red, tot, &s_nw);
}

// Sample sets of every instance (one thread per sample) and the per-node
// counts of the scatter list.
__global__ void kb_plan(const BInst *__restrict__ inst, const int *__restrict__ samp_pre, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= samp_pre[n]) return;
    const int i = inst_of(samp_pre, n, k);
    const BInst &b = inst[i];
    const Geo &g = b.g;
    const int l = k - samp_pre[i];
    SampleOut o = draw_sample(g, *b.step, 0xFFFFFFFFu, (uint32_t)l);
    const int N = g.nv, nq = N / 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {          // the quad-rotated shared-memory order
        const int j = o.idx[q];
        if (j < 0) continue;
        const int jx = j / (N * N), jz = j % N, row = j - jz;
        int r = jz / 4 + jx % nq;
        if (r >= nq) r -= nq;
        o.idx[q] = row + 4 * r + (jz & 3);
    }
    const ushort4 u = Idx4<uint16_t>::make(o.idx);
    b.pidx[l] = u;
    b.pa[l] = make_plan_a<float, uint16_t>(o.idx[0], o.idx[1], o.W);
    if (u.x != 0xFFFF) atomicAdd(b.sc_count + u.x, 1);
    if (u.y != 0xFFFF) atomicAdd(b.sc_count + u.y, 1);
    if (u.z != 0xFFFF) atomicAdd(b.sc_count + u.z, 1);
    if (u.w != 0xFFFF) atomicAdd(b.sc_count + u.w, 1);
}

// Exclusive scan of the counts: one CTA of 1024 threads per instance; T is
// the block size of the per-cell kernel (the scatter list layout uses it).
__global__ void __launch_bounds__(1024) kb_scatter_scan(const BInst *__restrict__ inst, int T)
{
    __shared__ int part[1024];
    const BInst &b = inst[blockIdx.x];
    const int nvt = b.g.nvt, t = threadIdx.x, per = (nvt + 1023) / 1024;
    const int lo = t * per, e = min(nvt, lo + per);
    int s = 0;
    for (int j = lo; j < e; ++j) s += b.sc_count[j];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;
    for (int j = lo; j < e; ++j) {
        b.sc_cursor[j] = run;
        run += b.sc_count[j];
        b.sc_count[j] = 0;                 // ready for the next step
    }
    if (t == 1023) {
        b.sc_meta[0] = part[1023];
        b.sc_meta[1] = (part[1023] + T - 1) / T;
    }
}

__global__ void kb_scatter_fill(const BInst *__restrict__ inst, const int *__restrict__ samp_pre,
                                int n, int T)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= samp_pre[n]) return;
    const int i = inst_of(samp_pre, n, k);
    const BInst &b = inst[i];
    const int l = k - samp_pre[i];
    const int C = b.sc_meta[1];
    const ushort4 q = b.pidx[l];
    const unsigned short d[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (d[r] == 0xFFFF) continue;
        const int pos = atomicAdd(b.sc_cursor + d[r], 1);
        const int tt = pos / C, ii = pos - tt * C;
        b.sc_ent[(int64_t)ii * T + tt] = ((uint32_t)d[r] << 16) | (r < 2 ? 0x8000u : 0u) | (uint32_t)l;
    }
}

// The per-cell step of every cell of every instance, persistent CTAs walking
// the flat cell list.  A CTA rebuilds its shared tables when it moves on to
// another instance.  Without the kb_advance launch that normally follows, a
// repeated launch recomputes the same step (the autotuner relies on this).
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
kb_cell4(const BInst *__restrict__ inst, const int *__restrict__ cell_pre, int n)
{
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ Geo sg;
    __shared__ int s_inst;
    const int total = cell_pre[n], vi = MAXT == 512 ? 0 : 1;
    int cur = -1, fallback = 0;
    Cell4Smem S{};
    for (int k = blockIdx.x; k < total; k += gridDim.x) {
        if (threadIdx.x == 0) s_inst = inst_of(cell_pre, n, k);
        __syncthreads();
        const int i = s_inst;
        if (i != cur) {
            if (threadIdx.x == 0) sg = inst[i].g;
            __syncthreads();
            S = carve4(smem_raw, sg.nv, sg.nvt);
            cell4_setup(sg, S);
            cur = i;
        }
        const BInst &b = inst[i];
        const int64_t step = *b.step;
        cell4_cell<true>(sg, b.map[vi], cell_of(sg, k - cell_pre[i]), b.h[step & 1], b.ghost, b.pa,
                         b.sc_ent, b.sc_meta, b.h[(step + 1) & 1], b.mom, S, fallback, nullptr, 0);
        __syncthreads();
    }
}

__global__ void kb_advance(const BInst *__restrict__ inst, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) *inst[i].step += 1;
}

// ---------------------------------------------------------------------
// Persistent active-node schedule: every instance keeps its own active-node
// step (bz_lazy.cuh: sample plan, compact arrays, deferred correction), and
// one launch per kernel class runs that step for all instances.  The per-step
// plan kernels are flattened over the samples (or take one CTA per
// instance); the per-cell kernel k_lz runs as persistent CTAs that claim
// segments (an instance and a range of its cell groups) from a counter, one
// pipeline per segment.  An instance whose step has more active nodes than
// its compact arrays hold takes the 4-node-vector kernel instead (a gated
// chain that does nothing otherwise).
// ---------------------------------------------------------------------
struct LzInst {
    Geo g;                       // the instance's problem (the 4-node kernel's plan order)
    LzArgs a[2];                 // arguments of k_lz for a state of step parity 0 and 1
    int64_t *step;               // device step counter
    float *h[2], *mu[2];         // state buffers and their pending corrections, by step parity
    float *ghost;
    double *nw;
    int4 *idx;                   // the step's sample set (node indices, logical order)
    PlanA<float, int> *pa;
    ushort4 *qc;                 // compact indices of the samples' nodes
    int *flag, *cidx, *count, *cursor, *rowend;
    // the 4-node-vector fallback
    Map4 map;
    ushort4 *pidx16;
    PlanA<float, uint16_t> *pa16;
    int *sc_count, *sc_cursor, *sc_meta;
    uint32_t *sc_ent;
    AheadPlans ahead;            // the instance's plans built ahead (K = 0: none)
};

// The plans of every instance's current step from its slots built ahead (grid
// row y: instance y), as k_ahead_take copies them for a single handle.
__global__ void kbl_take(const LzInst *__restrict__ inst)
{
    const LzInst &b = inst[blockIdx.y];
    const LzArgs &a = b.a[0];
    ahead_take(b.ahead, *b.step, b.idx, b.pa, const_cast<int *>(a.meta), const_cast<uint32_t *>(a.mask),
               const_cast<int *>(a.wpre), const_cast<int *>(a.act), const_cast<uint2 *>(a.rec),
               const_cast<int *>(a.dest0), a.stats, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
               (int64_t)gridDim.x * blockDim.x);
}

// Walls of every face of every instance (the input's pending corrections
// applied): one CTA per face.
__global__ void kbl_walls(const LzInst *__restrict__ inst, const int *__restrict__ face_pre, int n)
{
    __shared__ double red[kMaxWarps * kRedSlots];
    __shared__ double tot[4];
    __shared__ double s_nw;
    __shared__ float sA[kMaxN], sv[kMaxN];
    const int i = inst_of(face_pre, n, blockIdx.x);
    const LzInst &b = inst[i];
    const int64_t step = *b.step;
    const int p = (int)(step & 1);
    walls_face<float>(b.g, step, b.h[p], b.ghost, b.nw, nullptr, blockIdx.x - face_pre[i], sA, sv, red, tot,
                      &s_nw, b.mu[p]);
}

// The sample sets of every instance (one thread per sample) and the marks of
// the nodes they map to.
__global__ void kbl_plan(const LzInst *__restrict__ inst, const int *__restrict__ samp_pre, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= samp_pre[n]) return;
    const int i = inst_of(samp_pre, n, k);
    const LzInst &b = inst[i];
    const int l = k - samp_pre[i];
    // FP32 sampler, FP64 redraw near a velocity-cell face: the FP64 nodes.
    const SampleOut o = draw_sample_cell<float>(b.g, *b.step, 0xFFFFFFFFu, (uint32_t)l);
    b.idx[l] = make_int4(o.idx[0], o.idx[1], o.idx[2], o.idx[3]);
    b.pa[l] = make_plan_a<float, int>(o.idx[0], o.idx[1], o.W);
#pragma unroll
    for (int r = 0; r < 4; ++r)
        if (o.idx[r] >= 0) b.flag[o.idx[r]] = 1;
}

// Compact numbering of the marked nodes: one CTA of 1024 threads per instance.
__global__ void __launch_bounds__(1024) kbl_scan(const LzInst *__restrict__ inst)
{
    const LzInst &b = inst[blockIdx.x];
    const LzArgs &a = b.a[0];
    lz_scan_block(b.g.nvt, a.mcap, b.flag, b.cidx, const_cast<int *>(a.act), const_cast<uint32_t *>(a.mask),
                  const_cast<int *>(a.wpre), const_cast<int *>(a.meta), a.stats);
}

__global__ void kbl_remap(const LzInst *__restrict__ inst, const int *__restrict__ samp_pre, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= samp_pre[n]) return;
    const int i = inst_of(samp_pre, n, k);
    const LzInst &b = inst[i];
    lz_remap_one(k - samp_pre[i], b.idx, b.cidx, b.qc, b.count);
}

// Sorted order of the collision terms: one CTA of 1024 threads per instance.
__global__ void __launch_bounds__(1024) kbl_lscan(const LzInst *__restrict__ inst)
{
    const LzInst &b = inst[blockIdx.x];
    const LzArgs &a = b.a[0];
    lz_lscan_block(kLzRoleT, 4, b.count, b.cursor, b.rowend, const_cast<int *>(a.meta),
                   const_cast<uint2 *>(a.rec), const_cast<int *>(a.dest0));
}

__global__ void kbl_lfill(const LzInst *__restrict__ inst, const int *__restrict__ samp_pre, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= samp_pre[n]) return;
    const int i = inst_of(samp_pre, n, k);
    const LzInst &b = inst[i];
    const LzArgs &a = b.a[0];
    lz_lfill_one(k - samp_pre[i], kLzRoleT, 4, b.qc, b.pa, b.cursor, b.rowend, a.meta,
                 const_cast<uint2 *>(a.rec), const_cast<int *>(a.dest0));
}

// The per-cell step of every instance: persistent CTAs claim segments
// (x: instance, y: first group, z: groups, w: stride between them) from *next
// until none are left.  The segments of an instance are claimed one after
// the other, so they run at the same time and interleave over its groups
// (neighbouring cells are streamed together and their slabs shared in L2).
// Groups of four cells; one launch per velocity grid (NV: its axis length as
// a compile-time constant, 0 read at run time), sized for that grid.
template <int NV>
__global__ void __launch_bounds__(kLzThreads, 1) kbl_lz(const LzInst *__restrict__ inst,
                                                       const int4 *__restrict__ segs, int nseg,
                                                       int *__restrict__ next)
{
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ int s_seg;
    __shared__ Geo s_g;                     // the segment's problem and arguments
    __shared__ LzArgs s_a;
    for (;;) {
        __syncthreads();                    // the last segment's shared memory is free
        if (threadIdx.x == 0) s_seg = atomicAdd(next, 1);
        __syncthreads();
        const int sg = s_seg;
        if (sg >= nseg) break;
        const int4 q = segs[sg];
        const LzInst &b = inst[q.x];
        if (threadIdx.x == 0) {
            s_g = b.g;
            s_a = b.a[*b.step & 1];
        }
        __syncthreads();
        lz_run<4, NV, false>(s_g, s_a, smem_raw, q.y, q.w, q.z);
    }
}

// Fallback of the instances whose step overflowed (meta[1] set); every
// launch returns at once for the others.
__global__ void kbl_fb_plan(const LzInst *__restrict__ inst, const int *__restrict__ samp_pre, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= samp_pre[n]) return;
    const int i = inst_of(samp_pre, n, k);
    const LzInst &b = inst[i];
    if (!b.a[0].meta[1]) return;
    lz_fb_plan_one(k - samp_pre[i], b.g.nv, b.idx, b.pa, b.pidx16, b.pa16, b.sc_count);
}

__global__ void __launch_bounds__(1024) kbl_fb_scan(const LzInst *__restrict__ inst, int T)
{
    __shared__ int part[1024];
    const LzInst &b = inst[blockIdx.x];
    if (!b.a[0].meta[1]) return;
    scatter_scan_body(b.g.nvt, T, b.sc_count, b.sc_cursor, b.sc_meta, part);
    __syncthreads();
    for (int j = threadIdx.x; j < b.g.nvt; j += blockDim.x) b.sc_count[j] = 0;   // ready for the next step
}

__global__ void kbl_fb_fill(const LzInst *__restrict__ inst, const int *__restrict__ samp_pre, int n, int T)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= samp_pre[n]) return;
    const int i = inst_of(samp_pre, n, k);
    const LzInst &b = inst[i];
    if (!b.a[0].meta[1]) return;
    const int l = k - samp_pre[i], C = b.sc_meta[1];
    const ushort4 q = b.pidx16[l];
    const unsigned short d[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (d[r] == 0xFFFF) continue;
        const int pos = atomicAdd(b.sc_cursor + d[r], 1);
        const int tt = pos / C, ii = pos - tt * C;
        b.sc_ent[(int64_t)ii * T + tt] = ((uint32_t)d[r] << 16) | (r < 2 ? 0x8000u : 0u) | (uint32_t)l;
    }
}

// The input of an overflowed instance corrected in place, its pending
// corrections (and those of the output, which the 4-node kernel writes
// corrected) cleared: one CTA per cell at a time over the flat cell list.
__global__ void kbl_fb_materialize(const LzInst *__restrict__ inst, const int *__restrict__ cell_pre, int n)
{
    __shared__ float sv[kMaxN];
    __shared__ float smu[8];
    for (int i = 0; i < n; ++i) {
      const LzInst &b = inst[i];
      if (!b.a[0].meta[1]) continue;
      for (int c = blockIdx.x; c < cell_pre[i + 1] - cell_pre[i]; c += gridDim.x) {
        const Geo &g = b.g;
        const int p = (int)(*b.step & 1);
        const int N = g.nv, nq = N / 4, Q = N * N / 4;
        __syncthreads();
        for (int t = threadIdx.x; t < N; t += blockDim.x) sv[t] = (float)g.axv[t];
        if (threadIdx.x < 8) smu[threadIdx.x] = b.mu[p][(int64_t)c * 8 + threadIdx.x];
        __syncthreads();
        float4 *hc = reinterpret_cast<float4 *>(b.h[p]) + (int64_t)c * (g.nvt / 4);
        for (int o = threadIdx.x; o < g.nvt / 4; o += blockDim.x) {
            const int jx = o / Q, q = o % Q, jy = q / nq, jz = 4 * (q % nq);
            const float vx = sv[jx], vy = sv[jy];
            const float base = smu[0] + smu[1] * vx + smu[2] * vy + smu[4] * (vx * vx + vy * vy);
            float4 h = hc[o];
            float *hp = &h.x;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float vz = sv[jz + r];
                hp[r] = lz_corr(hp[r], base + smu[3] * vz + smu[4] * vz * vz, g.epsf);
            }
            hc[o] = h;
        }
        if (threadIdx.x < 8) {
            b.mu[p][(int64_t)c * 8 + threadIdx.x] = 0.f;
            b.mu[p ^ 1][(int64_t)c * 8 + threadIdx.x] = 0.f;
        }
      }
    }
}

// The 4-node-vector step of the cells of overflowed instances (persistent
// CTAs of 512 threads over the flat cell list).
__global__ void __launch_bounds__(512, 1) kbl_fb_cell4(const LzInst *__restrict__ inst,
                                                      const int *__restrict__ cell_pre, int n)
{
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ Geo sg;
    int fallback = 0;
    for (int i = 0; i < n; ++i) {
        const LzInst &b = inst[i];
        if (!b.a[0].meta[1]) continue;
        __syncthreads();
        if (threadIdx.x == 0) sg = b.g;
        __syncthreads();
        const Cell4Smem S = carve4(smem_raw, sg.nv, sg.nvt);
        cell4_setup(sg, S);
        const int64_t step = *b.step;
        for (int c = blockIdx.x; c < cell_pre[i + 1] - cell_pre[i]; c += gridDim.x) {
            cell4_cell<true>(sg, b.map, cell_of(sg, c), b.h[step & 1], b.ghost, b.pa16, b.sc_ent, b.sc_meta,
                             b.h[(step + 1) & 1], b.a[0].mom, S, fallback, nullptr, 0);
            __syncthreads();
        }
    }
}

__global__ void kbl_advance(const LzInst *__restrict__ inst, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) *inst[i].step += 1;
}

}  // namespace bzk
