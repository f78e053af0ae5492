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

#include "bz_cell4.cuh"

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

}  // namespace bzk
