// bz_lazy.cuh -- FP32 step on the active velocity nodes, correction deferred.
//
// Same mathematics as k_cell4 (Eqs. streaming2D, monteCarloInt,
// collision_step, rinorm_a, correzione, densita..sforzi), organised around two
// facts:
//
// * The Monte Carlo terms of a step touch only the nodes that one of its
//   shared samples maps to (v, v1, v*, v1*): for Maxwellian draws a small
//   fraction of the grid (about 7% of 32^3 at 2x10^4 samples).  Every other
//   node keeps h_c = h~.  The per-step plan lists those "active" nodes once
//   (compact index m), and the per-cell gather and scatter work on arrays of
//   M entries instead of the whole velocity slab.
// * The correction h^{n+1} = h_c + (1 + eps h_c)(mu . psi) needs mu, which
//   needs the moments of every node.  Instead of holding the whole slab until
//   mu is known, the step stores h_c and the cell's mu; whoever reads the
//   state next (the next step's streaming, the walls, a state copy) applies
//   the correction on the fly.  The state is therefore the pair (h_c, mu);
//   mu = 0 is an ordinary state.
//
// Without the slab a CTA needs two small compact arrays and a chunk of the
// per-sample products, so two CTAs share an SM and each works on G cells at
// once (the G values of a node are adjacent, so one vector access serves all
// G cells and each sample is read from L2 once per G cells).
//
// The conserved-moment sums of N_c and the output moments come from 26
// monomial sums (degree <= 4) of N = w h~ over all nodes, taken while
// streaming, plus the same sums of the collision increment over the active
// nodes.  If a step has more active nodes than the kernel's arrays hold
// (mcap), the kernel returns at once and the k_cell4 path computes the step.
#pragma once

#include "bz_cell4.cuh"

namespace bzk {

constexpr int kLzMaxChunks = 16;
constexpr int kLzMono = 26;        // monomial sums per cell
constexpr int kLzX = 30;           // with v^2, v_x v^2, v_y v^2, v_z v^2

// meta layout: [0] M, [1] overflow, [2 + k] S_k (k <= nchunk, start of chunk k
// in the sorted order), [3 + nchunk + k] C_k (words per thread), [4 +
// 2 nchunk + k] base_k (first word of chunk k in the list).
__host__ __device__ constexpr int lz_meta_s(int k) { return 2 + k; }
__host__ __device__ constexpr int lz_meta_c(int nchunk, int k) { return 3 + nchunk + k; }
__host__ __device__ constexpr int lz_meta_b(int nchunk, int k) { return 4 + 2 * nchunk + k; }
__host__ __device__ constexpr int lz_meta_size(int nchunk) { return 5 + 3 * nchunk; }

// ---------------------------------------------------------------------
// Per-step plan (once per step; every cell shares it)
// ---------------------------------------------------------------------

// Marks every node a sample of the step maps to.
__global__ void k_lz_mark(int nt, const int4 *__restrict__ idx, int *__restrict__ flag)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nt) return;
    const int4 q = idx[l];
    if (q.x >= 0) flag[q.x] = 1;
    if (q.y >= 0) flag[q.y] = 1;
    if (q.z >= 0) flag[q.z] = 1;
    if (q.w >= 0) flag[q.w] = 1;
}

// Compact numbering of the marked nodes (ascending node order), one CTA of
// 1024 threads: cidx[j] = m, act[m] = j, the bit mask of marked nodes and, per
// 32-node word, the compact index of its first marked node.  Clears the flags.
// stats (nullable): [5] counts steps whose active set exceeded mcap.
__global__ void __launch_bounds__(1024) k_lz_scan(int nvt, int mcap, int *__restrict__ flag,
                                                 int *__restrict__ cidx, int *__restrict__ act,
                                                 uint32_t *__restrict__ mask, int *__restrict__ wpre,
                                                 int *__restrict__ meta,
                                                 unsigned long long *__restrict__ stats = nullptr)
{
    __shared__ int part[1024];
    const int t = threadIdx.x, nw = nvt / 32, per = (nw + 1023) / 1024;
    const int w0 = min(nw, t * per), w1 = min(nw, w0 + per);
    int cnt = 0;
    for (int w = w0; w < w1; ++w) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) bits |= (flag[w * 32 + b] ? 1u : 0u) << b;
        mask[w] = bits;
        cnt += __popc(bits);
    }
    part[t] = cnt;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - cnt;
    for (int w = w0; w < w1; ++w) {
        const uint32_t bits = mask[w];
        wpre[w] = run;
        for (int b = 0; b < 32; ++b) {
            const int j = w * 32 + b;
            if (bits >> b & 1u) {
                cidx[j] = run;
                act[run] = j;
                ++run;
            }
            flag[j] = 0;
        }
    }
    if (t == 1023) {
        meta[0] = part[1023];
        meta[1] = part[1023] > mcap ? 1 : 0;
        if (stats) {
            if (part[1023] > mcap) atomicAdd(stats + 5, 1ull);
            stats[6] = (unsigned long long)part[1023];
        }
    }
}

// Compact sample records (a, b, W) and (a, b, a*, b*), and the per-(chunk,
// destination) term counts of the scatter list.
__global__ void k_lz_remap(int nt, int L, const int4 *__restrict__ idx,
                           const PlanA<float, int> *__restrict__ pa, const int *__restrict__ cidx,
                           const int *__restrict__ meta, PlanA<float, uint16_t> *__restrict__ pc,
                           ushort4 *__restrict__ qc, int *__restrict__ count)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nt) return;
    const int4 q = idx[l];
    const int d[4] = {q.x >= 0 ? cidx[q.x] : -1, q.y >= 0 ? cidx[q.y] : -1,
                      q.z >= 0 ? cidx[q.z] : -1, q.w >= 0 ? cidx[q.w] : -1};
    pc[l] = make_plan_a<float, uint16_t>(d[0], d[1], (double)pa[l].W);
    qc[l] = Idx4<uint16_t>::make(d);
    const int M = meta[0], k = l / L;
#pragma unroll
    for (int r = 0; r < 4; ++r)
        if (d[r] >= 0) atomicAdd(count + k * M + d[r], 1);
}

// Exclusive scan of the counts over (chunk, destination) and the per-chunk
// layout of the list for T threads; clears the counts.
__global__ void __launch_bounds__(1024) k_lz_lscan(int nchunk, int T, int *__restrict__ count,
                                                  int *__restrict__ cursor, int *__restrict__ meta)
{
    __shared__ int part[1024];
    const int t = threadIdx.x, n = nchunk * meta[0], per = (n + 1023) / 1024;
    const int b = min(n, t * per), e = min(n, b + per);
    int s = 0;
    for (int i = b; i < e; ++i) s += count[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;
    for (int i = b; i < e; ++i) {
        cursor[i] = run;
        run += count[i];
        count[i] = 0;
    }
    __syncthreads();
    if (t == 0) {
        const int M = meta[0];
        int base = 0;
        for (int k = 0; k <= nchunk; ++k) {
            const int key = k * M;
            const int S = k == nchunk ? part[1023] : (key < n ? cursor[key] : part[1023]);
            meta[lz_meta_s(k)] = S;
        }
        for (int k = 0; k < nchunk; ++k) {
            const int E = meta[lz_meta_s(k + 1)] - meta[lz_meta_s(k)];
            const int C = (E + T - 1) / T;
            meta[lz_meta_c(nchunk, k)] = C;
            meta[lz_meta_b(nchunk, k)] = base;
            base += C * T;
        }
    }
}

// Scatter list: every (destination, sample, sign) term of chunk k as
// m << 16 | loss << 15 | l' (l' the sample's index within its chunk), sorted
// by m; thread tt's run of C_k words of the sorted order is stored at stride
// T from base_k, so that the threads' i-th words are adjacent.
__global__ void k_lz_lfill(int nt, int L, int nchunk, int T, const ushort4 *__restrict__ qc,
                           int *__restrict__ cursor, const int *__restrict__ meta,
                           uint32_t *__restrict__ ent)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nt) return;
    const int M = meta[0], k = l / L, lp = l - k * L;
    const int S = meta[lz_meta_s(k)], C = meta[lz_meta_c(nchunk, k)];
    const int base = meta[lz_meta_b(nchunk, k)];
    const ushort4 q = qc[l];
    const unsigned short d[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (d[r] == 0xFFFF) continue;
        const int pos = atomicAdd(cursor + k * M + d[r], 1) - S;
        const int tt = pos / C, i = pos - tt * C;
        ent[base + (int64_t)i * T + tt] = ((uint32_t)d[r] << 16) | (r < 2 ? 0x8000u : 0u) | (uint32_t)lp;
    }
}

// ---------------------------------------------------------------------
// Fallback when a step has more active nodes than mcap: the k_cell4 plan is
// derived from the logical one, the input is corrected in place and mu_out
// is cleared (k_cell4 writes corrected states).  All return at once otherwise.
// ---------------------------------------------------------------------
__global__ void k_lz_fb_plan(int nt, int N, const int *__restrict__ meta,
                             const int4 *__restrict__ idx, const PlanA<float, int> *__restrict__ pa,
                             ushort4 *__restrict__ pidx16, PlanA<float, uint16_t> *__restrict__ pa16,
                             int *__restrict__ count)
{
    if (!meta[1]) return;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nt) return;
    const int4 q = idx[l];
    int o[4] = {q.x, q.y, q.z, q.w};
    const int nq = N / 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int j = o[k];
        if (j < 0) continue;
        const int jx = j / (N * N), jz = j % N, row = j - jz;
        int r = jz / 4 + jx % nq;
        if (r >= nq) r -= nq;
        o[k] = row + 4 * r + (jz & 3);
    }
    const ushort4 u = Idx4<uint16_t>::make(o);
    pidx16[l] = u;
    pa16[l] = make_plan_a<float, uint16_t>(o[0], o[1], (double)pa[l].W);
    if (u.x != 0xFFFF) atomicAdd(count + u.x, 1);
    if (u.y != 0xFFFF) atomicAdd(count + u.y, 1);
    if (u.z != 0xFFFF) atomicAdd(count + u.z, 1);
    if (u.w != 0xFFFF) atomicAdd(count + u.w, 1);
}

// Clears n floats when gate[1] is set (the pending corrections of a state
// that the fallback corrected in place).
__global__ void k_lz_clear(const int *__restrict__ gate, float *__restrict__ x, int64_t n)
{
    if (!gate[1]) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = 0.f;
}

// The correction of a stored node value: h = h_c + (1 + eps h_c) kappa.
__device__ __forceinline__ float lz_corr(float hc, float kappa, float eps)
{
    return fmaf(eps * hc, kappa, hc + kappa);
}

// h <- h_c + (1 + eps h_c)(mu_c . psi_j) for every node (in place allowed);
// mu_zero (nullable) is then cleared.  When skip_unless (nullable) points to
// 0, does nothing.  One CTA per cell at a time; float4 over jz.
__global__ void k_lz_materialize(Geo g, const int *__restrict__ skip_unless,
                                 const float *__restrict__ hin, const float *__restrict__ mu,
                                 float *__restrict__ hout, float *__restrict__ mu_zero)
{
    if (skip_unless && !skip_unless[1]) return;
    __shared__ float sv[kMaxN];
    __shared__ float smu[8];
    const int N = g.nv, nq = N / 4, Q = N * N / 4;
    for (int i = threadIdx.x; i < N; i += blockDim.x) sv[i] = (float)g.axv[i];
    const float eps = (float)g.eps;
    const int64_t plane = g.nvt / 4;
    for (int c = blockIdx.x; c < g.nr; c += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < 8) smu[threadIdx.x] = mu[(int64_t)c * 8 + threadIdx.x];
        __syncthreads();
        const float4 *src = reinterpret_cast<const float4 *>(hin) + (int64_t)c * plane;
        float4 *dst = reinterpret_cast<float4 *>(hout) + (int64_t)c * plane;
        for (int o = threadIdx.x; o < (int)plane; o += blockDim.x) {
            const int jx = o / Q, q = o % Q, jy = q / nq, jz = 4 * (q % nq);
            const float vx = sv[jx], vy = sv[jy];
            const float base = smu[0] + smu[1] * vx + smu[2] * vy + smu[4] * (vx * vx + vy * vy);
            float4 h = src[o];
            float *hp = &h.x;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float vz = sv[jz + i];
                hp[i] = lz_corr(hp[i], base + smu[3] * vz + smu[4] * vz * vz, eps);
            }
            dst[o] = h;
        }
    }
    if (mu_zero) {
        const int64_t n = (int64_t)g.nr * 8;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x)
            mu_zero[i] = 0.f;
    }
}

// ---------------------------------------------------------------------
// The per-cell kernel
// ---------------------------------------------------------------------

template <int G> struct LzVec;
template <> struct LzVec<1> { using T = float; };
template <> struct LzVec<2> { using T = float2; };

__device__ __forceinline__ float lz_get(float a, int) { return a; }
__device__ __forceinline__ float lz_get(float2 a, int g) { return g ? a.y : a.x; }
__device__ __forceinline__ float lz_axpy(float s, float a, float b) { return fmaf(s, a, b); }
__device__ __forceinline__ float2 lz_axpy(float s, float2 a, float2 b)
{
    return make_float2(fmaf(s, a.x, b.x), fmaf(s, a.y, b.y));
}
__device__ __forceinline__ float lz_gw(float W, float a, float b, float e)
{
    return W * (a + b + e * a * b);
}
__device__ __forceinline__ float2 lz_gw(float W, float2 a, float2 b, float e)
{
    return make_float2(W * (a.x + b.x + e * a.x * b.x), W * (a.y + b.y + e * a.y * b.y));
}
template <typename V> __device__ __forceinline__ V lz_zero();
template <> __device__ __forceinline__ float lz_zero<float>() { return 0.f; }
template <> __device__ __forceinline__ float2 lz_zero<float2>() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ float lz_shfl_up(float v, int o) { return __shfl_up_sync(0xFFFFFFFFu, v, o); }
__device__ __forceinline__ float2 lz_shfl_up(float2 v, int o)
{
    return make_float2(__shfl_up_sync(0xFFFFFFFFu, v.x, o), __shfl_up_sync(0xFFFFFFFFu, v.y, o));
}

// ---------------------------------------------------------------------
// Per-thread asynchronous copies global -> shared (cp.async), completed by
// the issuing thread's cp.async.wait_group: each thread prefetches the source
// values of its own nodes several streaming stages ahead, with no register
// cost and no synchronisation with other threads.
// ---------------------------------------------------------------------
constexpr int kLzStages = 3;       // stages in flight per thread

__device__ __forceinline__ uint32_t lz_saddr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void lz_cp8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(lz_saddr(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void lz_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void lz_cp_wait_stage()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(kLzStages - 1) : "memory");
}
__device__ __forceinline__ void lz_cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Everything the kernel needs besides the geometry (by value).
struct LzArgs {
    Map4 m;                 // node-pair mapping: Q pairs per jx-plane, K planes per
                            // stage (thread t works on plane t / Q of each stage),
                            // J = N / K stages per cell
    const float *hin, *mu_in, *ghost;
    float *hout, *mu_out;
    double *mom;
    const PlanA<float, uint16_t> *pc;
    const uint32_t *ent;
    const int *meta;
    const uint32_t *mask;
    const int *wpre, *act;
    int mcap, L, nchunk;
    float e0[kLzX];         // sum_j w_j X_k(v_j) of the 30 monomials
    long long *clk;         // nullable: phase trace of CTA 0 (kClkCells groups x kClkPhases)
};

constexpr int kLzMaxWarps = 16;    // the kernel runs at most 512 threads

// Shared memory.  A fixed-layout head (compile-time offsets, so the kernel
// keeps no pointers to it in registers): reduction scratch and per-cell sums,
// per-axis tables, the correction tables of the five cells a cell's
// streaming reads, the stage barriers.  Then, at run-time offsets: the
// active-node bit mask and word prefixes, the compact arrays (h~ and the
// collision increment, G values per node), and one region used first as the
// per-thread staging slots of the streaming prefetch (kLzStages stages x
// {own, x source, y source} x threads, 8 bytes each) and then as the chunk of
// per-sample products.
struct LzHead {
    float red[kLzMaxWarps * 32];
    float tot[64];
    float F[4 * 32], D[4 * 32];       // fill sums and increment sums per cell
    float v[kMaxN], A[kMaxN], IA[kMaxN], cax[kMaxN], cuy[kMaxN];
    float4 gram[kMaxN];               // v, v^2, v^3, v^4
    float2 vz2[kMaxN / 2], Az2[kMaxN / 2];   // v and A of the node pairs along jz
    float ca[5 * kMaxN];              // mu0 + mu_x v + mu_4 v^2 of the five cells
    float mus[5 * 8];                 // mu of the five cells
};

__host__ __device__ inline size_t lz_region_bytes(int T, int G, int L)
{
    const size_t ring = (size_t)kLzStages * 3 * T * sizeof(float2),
                 chunk = sizeof(float) * (size_t)G * L;
    return ring > chunk ? ring : chunk;
}

// Bytes before the region, and the run-time offsets.
struct LzOff {
    uint32_t mask, wpre, act, A, B, region;
};
__host__ __device__ inline LzOff lz_offsets(int nvt, int mcap, int G)
{
    LzOff o;
    size_t off = (sizeof(LzHead) + 15) & ~(size_t)15;
    o.mask = (uint32_t)off; off += sizeof(uint32_t) * (nvt / 32);
    o.wpre = (uint32_t)off; off += sizeof(uint16_t) * (nvt / 32);
    o.act = (uint32_t)off; off += sizeof(uint16_t) * (size_t)mcap;
    off = (off + 15) & ~(size_t)15;
    o.A = (uint32_t)off; off += sizeof(float) * (size_t)G * mcap;
    o.B = (uint32_t)off; off += sizeof(float) * (size_t)G * mcap;
    off = (off + 127) & ~(size_t)127;
    o.region = (uint32_t)off;
    return o;
}
__host__ __device__ inline size_t lz_fixed_bytes(int nv, int nvt, int mcap, int G)
{
    (void)nv;
    return lz_offsets(nvt, mcap, G).region;
}

// Monomial index of psi_a * phi_b in the 30-entry sum vector X (psi = 1,
// v_x, v_y, v_z, v^2; phi = 1, v_x, v_y, v_z, v_x^2, v_y^2, v_z^2, v_x v_y,
// v_x v_z, v_y v_z).  X order: 0 1; 1-3 v_x, v_y, v_z; 4-6 v_x^2, v_y^2,
// v_z^2; 7-9 v_x v_y, v_x v_z, v_y v_z; 10-12 v_x^3, v_y^3, v_z^3; 13 v_x^2 v_y;
// 14 v_x^2 v_z; 15 v_x v_y^2; 16 v_y^2 v_z; 17 v_x v_z^2; 18 v_y v_z^2;
// 19 v_x v_y v_z; 20-22 v_x^2 v^2, v_y^2 v^2, v_z^2 v^2; 23-25 v_x v_y v^2,
// v_x v_z v^2, v_y v_z v^2; 26 v^2; 27-29 v_x v^2, v_y v^2, v_z v^2.
__device__ __constant__ const unsigned char kLzPsiPhi[5][10] = {
    {0, 1, 2, 3, 4, 5, 6, 7, 8, 9},
    {1, 4, 7, 8, 10, 15, 17, 13, 14, 19},
    {2, 7, 5, 9, 13, 11, 18, 15, 19, 16},
    {3, 8, 9, 6, 14, 16, 12, 19, 17, 18},
    {26, 27, 28, 29, 20, 21, 22, 23, 24, 25}};

// The 26 monomial sums of sum_nodes n(v) from per-thread power sums over jx
// (s[p] = sum n v_x^p) at fixed v_y = y, v_z = z.
__device__ __forceinline__ void lz_mono_from_powers(const float (&s)[5], float y, float z,
                                                    float (&M)[kLzMono])
{
    const float y2 = y * y, z2 = z * z, q = y2 + z2, yz = y * z;
    M[0] += s[0];
    M[1] += s[1];
    M[2] += y * s[0];
    M[3] += z * s[0];
    M[4] += s[2];
    M[5] += y2 * s[0];
    M[6] += z2 * s[0];
    M[7] += y * s[1];
    M[8] += z * s[1];
    M[9] += yz * s[0];
    M[10] += s[3];
    M[11] += y2 * y * s[0];
    M[12] += z2 * z * s[0];
    M[13] += y * s[2];
    M[14] += z * s[2];
    M[15] += y2 * s[1];
    M[16] += y2 * z * s[0];
    M[17] += z2 * s[1];
    M[18] += y * z2 * s[0];
    M[19] += yz * s[1];
    const float t2 = s[2] + q * s[0];
    M[20] += s[4] + q * s[2];
    M[21] += y2 * t2;
    M[22] += z2 * t2;
    M[23] += y * (s[3] + q * s[1]);
    M[24] += z * (s[3] + q * s[1]);
    M[25] += yz * t2;
}

// The same sums for one node value d at velocity (x, y, z).
__device__ __forceinline__ void lz_mono_node(float d, float x, float y, float z,
                                             float (&M)[kLzMono])
{
    const float s[5] = {d, d * x, d * x * x, d * x * x * x, d * x * x * x * x};
    lz_mono_from_powers(s, y, z, M);
}

// X (30) from the 26 sums.
__device__ __forceinline__ void lz_extend(const float *T, float *X)
{
    for (int k = 0; k < kLzMono; ++k) X[k] = T[k];
    X[26] = T[4] + T[5] + T[6];
    X[27] = T[10] + T[15] + T[17];
    X[28] = T[13] + T[11] + T[18];
    X[29] = T[14] + T[16] + T[12];
}

// Correction and output moments of one cell from the sums F (of N = w h~)
// and D (of the collision increment): mu to mu_out, moments to mom.
__device__ __noinline__ void lz_finish(const Geo &g, const LzArgs &a, int c, const float *F,
                                       const float *D, int *fallback)
{
    float T[kLzMono], X[kLzX], XF[kLzX];
    for (int k = 0; k < kLzMono; ++k) T[k] = F[k] + D[k];
    lz_extend(T, X);
    lz_extend(F, XF);
    // Eqs. rinorm_a, correzione: G mu = -(post - pre) with the sums of N_c.
    float P[19];
    for (int k = 0; k < 10; ++k) P[k] = X[k];
    P[10] = X[27];
    P[11] = X[28];
    P[12] = X[29];
    P[13] = X[20] + X[21] + X[22];
    P[14] = XF[0];
    P[15] = XF[1];
    P[16] = XF[2];
    P[17] = XF[3];
    P[18] = XF[26];
    float mu[5];
    if (!correction_spd(g, P, mu)) {
        double Pd[19], m8[5];
        for (int k = 0; k < 19; ++k) Pd[k] = (double)P[k];
        correction_solve<float>(g, Pd, m8, fallback);
        for (int k = 0; k < 5; ++k) mu[k] = (float)m8[k];
    }
    float *mo = a.mu_out + (int64_t)c * 8;
    for (int k = 0; k < 5; ++k) mo[k] = mu[k];
    // Moments of h^{n+1}: sum w h phi = sum N_c phi + sum_a mu_a (E0 + eps sum N_c psi_a phi).
    const float eps = (float)g.eps;
    float m10[10];
    for (int b = 0; b < 10; ++b) {
        float s = X[b];
        for (int k = 0; k < 5; ++k) {
            const int x = kLzPsiPhi[k][b];
            s += mu[k] * (a.e0[x] + eps * X[x]);
        }
        m10[b] = s;
    }
    if (a.mom) finalize_moments_f(m10, eps, a.mom + (int64_t)c * 11);
}

// Planes per streaming stage for node pairs and 512 threads: the largest
// divisor K of N with K * N^2 / 2 <= 512.
__host__ __device__ constexpr int lz_planes(int N)
{
    int K = 1;
    for (int k = 1; k <= N; ++k)
        if (N % k == 0 && k * (N * N / 2) <= 512) K = k;
    return K;
}

// NV: the velocity axis length as a compile-time constant (0: read g.nv at
// run time).  Thread t owns node pair q = t mod Q of jx-plane (t div Q) of
// every streaming stage.
template <int G, int NV>
__global__ void __launch_bounds__(512, 2) k_lz(Geo g, LzArgs a)
{
    using V = typename LzVec<G>::T;
    extern __shared__ __align__(16) char smem_raw[];
    if (a.meta[1]) return;                        // too many active nodes: k_cell4 runs
    const int N = NV ? NV : g.nv;
    const int N2 = N * N, nvt = N2 * N, T = blockDim.x, t = threadIdx.x;
    const int Q = N2 / 2, nq = N / 2, P = NV ? lz_planes(NV) : a.m.K, J = N / P;
    const int half = N / 2;
    const int64_t plane = nvt / 2;                // float2 per cell
    LzHead &S = *reinterpret_cast<LzHead *>(smem_raw);
    const LzOff so = lz_offsets(nvt, a.mcap, G);
    uint32_t *smask = reinterpret_cast<uint32_t *>(smem_raw + so.mask);
    uint16_t *swpre = reinterpret_cast<uint16_t *>(smem_raw + so.wpre);
    uint16_t *sact = reinterpret_cast<uint16_t *>(smem_raw + so.act);
    float *region = reinterpret_cast<float *>(smem_raw + so.region);
    V *Ac = reinterpret_cast<V *>(smem_raw + so.A);
    V *Bc = reinterpret_cast<V *>(smem_raw + so.B);
    V *gw = reinterpret_cast<V *>(region);
    float2 *slots = reinterpret_cast<float2 *>(region);   // [stage][source][thread]
    const float eps = (float)g.eps;
    const int M = a.meta[0];
    // ---- tables (once per launch) ----------------------------------------
    for (int i = t; i < N; i += T) {
        const double v = g.axv[i], A = g.axA[i];
        S.v[i] = (float)v;
        S.A[i] = (float)A;
        S.IA[i] = (float)(1.0 / A);
        S.cax[i] = (float)fabs(v * g.dt / g.dx);
        S.cuy[i] = (float)fabs(v * g.dt / g.dy);
        S.gram[i] = make_float4((float)v, (float)(v * v), (float)(v * v * v), (float)(v * v * v * v));
    }
    for (int w = t; w < nvt / 32; w += T) {
        smask[w] = a.mask[w];
        swpre[w] = (uint16_t)a.wpre[w];
    }
    for (int m = t; m < M; m += T) sact[m] = (uint16_t)a.act[m];
    __syncthreads();
    for (int i = t; i < N / 2; i += T) {
        S.vz2[i] = make_float2(S.v[2 * i], S.v[2 * i + 1]);
        S.Az2[i] = make_float2(S.A[2 * i], S.A[2 * i + 1]);
    }
    __syncthreads();

    const int q = t % Q, pl = t / Q;
    const bool active = pl < P;
    const int jy = q / nq, qz = q % nq;
    const bool yup = jy >= half;                  // v_y > 0: the y source is below
    const int ys = yup ? 3 : 4;
    const float2 *hin2 = reinterpret_cast<const float2 *>(a.hin);
    float2 *hout2 = reinterpret_cast<float2 *>(a.hout);
    int fallback = 0;
    const int ngroups = (g.nr + G - 1) / G;
    int ngrp = 0;
    auto stamp = [&](int ph) {
        if (a.clk && blockIdx.x == 0 && t == 0 && ngrp < kClkCells)
            a.clk[ngrp * kClkPhases + ph] = clock64();
    };

    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++ngrp) {
        stamp(0);
        int cg[G], cx[G], cy[G];
        int ncell = 0;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int kc = grp * G + k;
            cg[k] = kc < g.nr ? cell_of(g, kc) : -1;
            cx[k] = cg[k] >= 0 ? cg[k] % g.nx : 0;
            cy[k] = cg[k] >= 0 ? cg[k] / g.nx : 0;
            ncell += cg[k] >= 0 ? 1 : 0;
        }
        // Prefetch position: cell pk of the group, stage pst of that cell.
        // Each call copies this thread's own, x-source and y-source pairs of
        // that stage into its slots (sources beyond a wall are not copied)
        // and commits one group of copies.
        int pk = 0, pst = 0, pslot = 0;
        auto prefetch = [&]() {
            if (active && pk < ncell) {
                const int c = G == 1 || pk == 0 ? cg[0] : cg[G - 1];
                const int ix = G == 1 || pk == 0 ? cx[0] : cx[G - 1];
                const int iy = G == 1 || pk == 0 ? cy[0] : cy[G - 1];
                const int jx = pst * P + pl;
                const float2 *own = hin2 + (int64_t)c * plane + jx * Q + q;
                float2 *sl = slots + pslot * 3 * T + t;
                lz_cp8(sl, own);
                const bool xr = jx < half;
                if (xr ? ix < g.nx - 1 : ix > 0) lz_cp8(sl + T, own + (xr ? plane : -plane));
                if (yup ? iy > 0 : iy < g.ny - 1)
                    lz_cp8(sl + 2 * T, own + (yup ? -(int64_t)g.nx : (int64_t)g.nx) * plane);
            }
            lz_cp_commit();
            if (++pst == J) {
                pst = 0;
                ++pk;
            }
            if (++pslot == kLzStages) pslot = 0;
        };
        // The region was the previous group's per-sample chunk.
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kLzStages; ++kk) prefetch();
        for (int i = t; i < M; i += T) Bc[i] = lz_zero<V>();
        if (ncell < G)
            for (int i = t; i < M; i += T) Ac[i] = lz_zero<V>();

        // ---- streaming with the deferred correction applied to its sources
        int cslot = 0;                            // slots of the stage being consumed
#pragma unroll 1
        for (int k = 0; k < ncell; ++k) {
            const int c = k == 0 ? cg[0] : cg[G - 1];
            const int ix = k == 0 ? cx[0] : cx[G - 1], iy = k == 0 ? cy[0] : cy[G - 1];
            // mu of the five cells the streaming reads: own, right, left, below, above.
            __syncthreads();
            if (t < 40) {
                const int s5 = t / 8, r = t % 8;
                int cs = c;
                bool ok = true;
                if (s5 == 1) { ok = ix < g.nx - 1; cs = c + 1; }
                if (s5 == 2) { ok = ix > 0; cs = c - 1; }
                if (s5 == 3) { ok = iy > 0; cs = c - g.nx; }
                if (s5 == 4) { ok = iy < g.ny - 1; cs = c + g.nx; }
                S.mus[t] = ok && r < 5 ? a.mu_in[(int64_t)cs * 8 + r] : 0.f;
            }
            __syncthreads();
            for (int i = t; i < 5 * N; i += T) {
                const int s5 = i / N, jx = i - s5 * N;
                const float vx = S.v[jx];
                S.ca[i] = S.mus[s5 * 8] + S.mus[s5 * 8 + 1] * vx + S.mus[s5 * 8 + 4] * vx * vx;
            }
            __syncthreads();
            const bool yin = yup ? iy > 0 : iy < g.ny - 1;
            const float *yg = a.ghost + (yup ? 2 * g.ny + ix : 2 * g.ny + g.nx + ix) * N;
            // The (v_y, v_z) part of each source cell's pending correction at
            // this thread's two nodes: mu_y v_y + mu_z v_z + mu_4 (v_y^2 + v_z^2)
            // for the own cell (o), the y source (y), the right (r) and left (l) cells.
            float bdo[2], bdy[2], bdr[2], bdl[2];
            {
                const float vy = S.v[jy];
                const float2 z2 = S.vz2[qz];
                const float vz[2] = {z2.x, z2.y};
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const float qi = vy * vy + vz[i] * vz[i];
                    bdo[i] = S.mus[2] * vy + S.mus[3] * vz[i] + S.mus[4] * qi;
                    bdy[i] = S.mus[ys * 8 + 2] * vy + S.mus[ys * 8 + 3] * vz[i] + S.mus[ys * 8 + 4] * qi;
                    bdr[i] = S.mus[8 + 2] * vy + S.mus[8 + 3] * vz[i] + S.mus[8 + 4] * qi;
                    bdl[i] = S.mus[16 + 2] * vy + S.mus[16 + 3] * vz[i] + S.mus[16 + 4] * qi;
                }
            }
            // Per-thread power sums over jx of N = w h~ / (A_y A_z) for the pair.
            float s[2][5];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int pp = 0; pp < 5; ++pp) s[i][pp] = 0.f;
#pragma unroll 1
            for (int st = 0; st < J; ++st) {
                // This thread's copies of the stage have landed.
                lz_cp_wait_stage();
                const float2 *sl = slots + cslot * 3 * T + t;
                if (active) {
                    const int jx = st * P + pl;
                    const bool xr = jx < half;                 // v_x < 0: source right
                    const bool xin = xr ? ix < g.nx - 1 : ix > 0;
                    const int xs = xr ? 1 : 2;
                    const float2 h0 = sl[0];
                    const float xgv = xin ? 0.f : a.ghost[(xr ? g.ny + iy : iy) * N + jy];
                    const float2 hx = xin ? sl[T] : make_float2(xgv, xgv);
                    const float ygv = yin ? 0.f : yg[jx];
                    const float2 hy = yin ? sl[2 * T] : make_float2(ygv, ygv);
                    const float ax = S.cax[jx], ay = S.cuy[jy];
                    const float4 gv = S.gram[jx];
                    const float Ax = S.A[jx];
                    // Pending correction of each source: ca(jx) + its (v_y, v_z) part.
                    const float cao = S.ca[jx], cax = S.ca[xs * N + jx], cay = S.ca[ys * N + jx];
                    const float h0a[2] = {h0.x, h0.y}, hxa[2] = {hx.x, hx.y}, hya[2] = {hy.x, hy.y};
                    float ht[2];
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const float bdx = xr ? bdr[i] : bdl[i];
                        const float u0 = lz_corr(h0a[i], cao + bdo[i], eps);
                        const float ux = xin ? lz_corr(hxa[i], cax + bdx, eps) : hxa[i];
                        const float uy = yin ? lz_corr(hya[i], cay + bdy[i], eps) : hya[i];
                        ht[i] = u0 - ax * (u0 - ux) - ay * (u0 - uy);
                        const float n = ht[i] * Ax;       // times A_y A_z after the loop
                        s[i][0] += n;
                        s[i][1] = fmaf(n, gv.x, s[i][1]);
                        s[i][2] = fmaf(n, gv.y, s[i][2]);
                        s[i][3] = fmaf(n, gv.z, s[i][3]);
                        s[i][4] = fmaf(n, gv.w, s[i][4]);
                    }
                    hout2[(int64_t)c * plane + jx * Q + q] = make_float2(ht[0], ht[1]);
                    // Active nodes of the pair go to the compact array.
                    const int j0 = jx * N2 + jy * N + 2 * qz;
                    const uint32_t mw = smask[j0 >> 5];
                    const int sh = j0 & 31;
                    const uint32_t bits = (mw >> sh) & 3u;
                    if (bits) {
                        int mi = swpre[j0 >> 5] + __popc(mw & ((1u << sh) - 1u));
                        float *Af = reinterpret_cast<float *>(Ac);
                        if (bits & 1u) Af[(mi++) * G + k] = ht[0];
                        if (bits & 2u) Af[mi * G + k] = ht[1];
                    }
                }
                // The slots just read take the stage kLzStages ahead.
                prefetch();
                if (++cslot == kLzStages) cslot = 0;
            }
            float Msum[kLzMono];
#pragma unroll
            for (int r = 0; r < kLzMono; ++r) Msum[r] = 0.f;
            if (active) {
                const float2 a2 = S.Az2[qz], z2 = S.vz2[qz];
                const float Ay = S.A[jy], vy = S.v[jy];
                const float Ayz[2] = {Ay * a2.x, Ay * a2.y}, vz[2] = {z2.x, z2.y};
#pragma unroll
                for (int i = 0; i < 2; ++i) {
#pragma unroll
                    for (int pp = 0; pp < 5; ++pp) s[i][pp] *= Ayz[i];
                    lz_mono_from_powers(s[i], vy, vz[i], Msum);
                }
            }
            block_reduce4<kLzMono>(Msum, S.red, S.tot);
            if (t < kLzMono) S.F[k * 32 + t] = S.tot[t];
            stamp(1 + k);
        }
        lz_cp_wait_all();
        __syncthreads();

        // ---- Monte Carlo terms (Eq. monteCarloInt), chunk by chunk ---------
        for (int ck = 0; ck < a.nchunk; ++ck) {
            const int lb = ck * a.L, le = min(g.nt, lb + a.L);
            {
                // Eight sample records in flight per thread.
                int l = lb + t;
                for (; l + 7 * T < le; l += 8 * T) {
                    PlanA<float, uint16_t> r[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) r[u] = a.pc[l + u * T];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int ia = r[u].a(), ib = r[u].b();
                        const V va = ia >= 0 ? Ac[ia] : lz_zero<V>();
                        const V vb = ib >= 0 ? Ac[ib] : lz_zero<V>();
                        gw[l + u * T - lb] = lz_gw(r[u].W, va, vb, eps);
                    }
                }
                for (; l < le; l += T) {
                    const PlanA<float, uint16_t> r = a.pc[l];
                    const int ia = r.a(), ib = r.b();
                    const V va = ia >= 0 ? Ac[ia] : lz_zero<V>();
                    const V vb = ib >= 0 ? Ac[ib] : lz_zero<V>();
                    gw[l - lb] = lz_gw(r.W, va, vb, eps);
                }
            }
            __syncthreads();
            if (ck == 0) stamp(3);
            {
                // Each thread walks its run of the destination-sorted list,
                // sums the terms of one destination in registers and adds the
                // sum once: plainly for a destination inside its run, with
                // atomics for the first and last ones (neighbouring runs may
                // share them).  The G values of a node are adjacent, so one
                // 8-byte access serves the group.
                const int S0 = a.meta[lz_meta_s(ck)], E = a.meta[lz_meta_s(ck + 1)] - S0;
                const int C = a.meta[lz_meta_c(a.nchunk, ck)];
                const uint32_t *ent = a.ent + a.meta[lz_meta_b(a.nchunk, ck)];
                const int n = max(0, min(C, E - t * C));
                float *Bf = reinterpret_cast<float *>(Bc);
                int cur = -1;
                bool first = true;
                V acc = lz_zero<V>();
                auto flush = [&](bool shared) {
                    if (cur < 0) return;
                    if (shared) {
#pragma unroll
                        for (int k = 0; k < G; ++k) atomicAdd(Bf + cur * G + k, lz_get(acc, k));
                    } else {
                        Bc[cur] = lz_axpy(1.f, acc, Bc[cur]);
                    }
                };
                auto term = [&](uint32_t w, V r) {
                    const int dest = (int)(w >> 16);
                    if (dest != cur) {
                        flush(first);
                        first = cur < 0;
                        cur = dest;
                        acc = lz_zero<V>();
                    }
                    acc = lz_axpy((w & 0x8000u) ? -1.f : 1.f, r, acc);
                };
                // Batches of 8 words; two batches ahead are in flight while
                // one is applied (the list streams from L2).
                int i = 0;
                uint32_t wa[8], wb[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    wa[u] = u < n ? ent[u * T + t] : 0u;
                    wb[u] = 8 + u < n ? ent[(8 + u) * T + t] : 0u;
                }
                for (; i + 7 < n; i += 8) {
                    uint32_t w[8];
                    V r[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        w[u] = wa[u];
                        wa[u] = wb[u];
                    }
                    if (i + 23 < n) {
#pragma unroll
                        for (int u = 0; u < 8; ++u) wb[u] = ent[(i + 16 + u) * T + t];
                    } else {
#pragma unroll
                        for (int u = 0; u < 8; ++u) wb[u] = i + 16 + u < n ? ent[(i + 16 + u) * T + t] : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) r[u] = gw[w[u] & 0x7FFFu];
#pragma unroll
                    for (int u = 0; u < 8; ++u) term(w[u], r[u]);
                }
                for (; i < n; ++i) {
                    const uint32_t w = ent[i * T + t];
                    term(w, gw[w & 0x7FFFu]);
                }
                flush(true);
            }
            __syncthreads();
            if (ck == 0) stamp(4);
        }
        stamp(5);

        // ---- sums of the collision increment; correction and moments ------
#pragma unroll 1
        for (int k = 0; k < ncell; ++k) {
            float Dsum[kLzMono];
#pragma unroll
            for (int r = 0; r < kLzMono; ++r) Dsum[r] = 0.f;
            const float *Bf = reinterpret_cast<const float *>(Bc);
            for (int mm = t; mm < M; mm += T) {
                const int j = sact[mm];
                const int jx = j / N2, jyy = (j / N) % N, jz = j % N;
                lz_mono_node(Bf[mm * G + k], S.v[jx], S.v[jyy], S.v[jz], Dsum);
            }
            block_reduce4<kLzMono>(Dsum, S.red, S.tot);
            if (t < kLzMono) S.D[k * 32 + t] = S.tot[t];
        }
        __syncthreads();
        // One warp per cell of the group.
        if ((t & 31) == 0 && (t >> 5) < ncell) {
            const int k = t >> 5;
            lz_finish(g, a, k == 0 ? cg[0] : cg[G - 1], S.F + k * 32, S.D + k * 32, &fallback);
        }
        stamp(6);

        // ---- h_c = h~ + dN / w on the active nodes --------------------------
        {
            const float *Af = reinterpret_cast<const float *>(Ac);
            const float *Bf = reinterpret_cast<const float *>(Bc);
            for (int i = t; i < M * G; i += T) {
                const int mm = i / G, k = i - mm * G;
                if (k >= ncell) continue;
                const int j = sact[mm];
                const int jx = j / N2, jyy = (j / N) % N, jz = j % N;
                const float iw = S.IA[jx] * S.IA[jyy] * S.IA[jz];
                a.hout[(int64_t)(k == 0 ? cg[0] : cg[G - 1]) * nvt + j] = fmaf(Bf[i], iw, Af[i]);
            }
        }
        __syncthreads();
        stamp(7);
    }
    (void)fallback;
}

}  // namespace bzk
