// bz_cell4.cuh -- per-cell relaxation kernel, FP32 fast path.
//
// Same mathematics as k_cell (Eqs. streaming2D, monteCarloInt,
// collision_step, rinorm_a, correzione, densita..sforzi) for FP32 states whose
// velocity axis has a multiple of 4 nodes.  Thread t owns a "quad" of four
// consecutive jz nodes of one (jy) row and a contiguous range of J jx-planes:
//   q = t mod Q (Q = N^2/4 quads per plane), k = t div Q, jx in [kJ, kJ + J).
// All slab traffic (global and shared) is 16-byte vectors and the per-jx
// tables are read as broadcast float4s shared by the quad's four nodes.  The
// scatter of Eq. monteCarloInt walks a destination-sorted list of the step's
// terms (built once per step by k_scatter_*), so a thread adds the sum of a
// node's terms with one shared-memory atomic instead of one per term.
#pragma once

#include "bz_kernels.cuh"

namespace bzk {

constexpr int kClkCells = 8;    // cells traced per launch (CTA 0)
constexpr int kClkPhases = 9;   // stamps per cell

struct Map4 {
    int Q;   // quads per jx-plane (N^2 / 4)
    int K;   // jx chunks
    int J;   // jx planes per chunk (N / K)
};

// Shared-memory layout of k_cell4.
struct Cell4Smem {
    float *red;      // kMaxWarps * 32
    double *tot;     // 32 (totf aliases its first 128 bytes)
    double *mu;      // 8
    float4 *conv;    // N: {A, v, v^2, 0}
    float4 *gram;    // N: {v, v^2, v^3, v^4}
    float4 *fin;     // N: {1/A, cx, A, A v}   (cx = mu_x v + mu_4 v^2, per cell)
    float *Av2;      // N: A v^2
    float *cu;       // N: v dt/dx
    float *v;        // N
    float *A;        // N
    float *IA;       // N
    int *rot;        // N: jx mod (N/4), the quad rotation of plane jx
    float4 *vzq;     // N/4: v of the four jz nodes of quad column qz
    float4 *Azq;     // N/4: A of those nodes
    float4 *IAzq;    // N/4: 1/A of those nodes
    float4 *slab4;   // N^3 / 4
    float *gw;       // Nt: g_l W_l of the gather phase
};

__host__ __device__ inline size_t cell4_smem_bytes(int nv, int nvt, int nt)
{
    size_t off = sizeof(float) * kMaxWarps * 32 + sizeof(double) * (32 + 8);
    off += sizeof(float4) * 3 * nv + sizeof(float) * 5 * nv + sizeof(int) * nv;
    off = (off + 15) & ~(size_t)15;
    off += sizeof(float4) * 3 * (nv / 4);
    off += sizeof(float) * nvt;
    off += sizeof(float) * nt;
    return off;
}

__device__ __forceinline__ Cell4Smem carve4(char *base, int N, int nvt)
{
    Cell4Smem s;
    size_t off = 0;
    s.red = (float *)(base + off); off += sizeof(float) * kMaxWarps * 32;
    s.tot = (double *)(base + off); off += sizeof(double) * 32;
    s.mu = (double *)(base + off); off += sizeof(double) * 8;
    s.conv = (float4 *)(base + off); off += sizeof(float4) * N;
    s.gram = (float4 *)(base + off); off += sizeof(float4) * N;
    s.fin = (float4 *)(base + off); off += sizeof(float4) * N;
    s.Av2 = (float *)(base + off); off += sizeof(float) * N;
    s.cu = (float *)(base + off); off += sizeof(float) * N;
    s.v = (float *)(base + off); off += sizeof(float) * N;
    s.A = (float *)(base + off); off += sizeof(float) * N;
    s.IA = (float *)(base + off); off += sizeof(float) * N;
    s.rot = (int *)(base + off); off += sizeof(int) * N;
    off = (off + 15) & ~(size_t)15;
    s.vzq = (float4 *)(base + off); off += sizeof(float4) * (N / 4);
    s.Azq = (float4 *)(base + off); off += sizeof(float4) * (N / 4);
    s.IAzq = (float4 *)(base + off); off += sizeof(float4) * (N / 4);
    s.slab4 = (float4 *)(base + off);
    off += sizeof(float) * nvt;
    s.gw = (float *)(base + off);
    return s;
}

// Destination-sorted scatter list of a step (shared by every cell): every
// valid (node, sample, sign) term of Eq. monteCarloInt as one 32-bit word
// node << 16 | loss << 15 | l, sorted by node by a counting sort, and stored
// so that thread t of the cell kernel reads its contiguous run of C words at
// stride T (coalesced).  meta[0] = number of words E, meta[1] = C.
static __global__ void k_scatter_count(int nt, const ushort4 *__restrict__ pidx, int *__restrict__ count)
{
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nt) return;
    ushort4 q = pidx[l];
    if (q.x != 0xFFFF) atomicAdd(count + q.x, 1);
    if (q.y != 0xFFFF) atomicAdd(count + q.y, 1);
    if (q.z != 0xFFFF) atomicAdd(count + q.z, 1);
    if (q.w != 0xFFFF) atomicAdd(count + q.w, 1);
}

// Exclusive scan of the per-node counts (one CTA of 1024 threads).
// gate (nullable): when it is given and gate[1] is 0, the kernel does nothing.
// Exclusive scan of the per-node counts (one CTA of 1024 threads, part: 1024
// ints of shared memory): cursor = first position of each node's words,
// meta = {E, C = ceil(E / T)}.
__device__ __forceinline__ void scatter_scan_body(int nvt, int T, const int *__restrict__ count,
                                                  int *__restrict__ cursor, int *__restrict__ meta,
                                                  int *part)
{
    const int t = threadIdx.x, per = (nvt + 1023) / 1024;
    const int b = t * per, e = min(nvt, b + per);
    int s = 0;
    for (int j = b; j < e; ++j) s += count[j];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {       // Hillis-Steele inclusive scan
        int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;
    for (int j = b; j < e; ++j) {
        cursor[j] = run;
        run += count[j];
    }
    if (t == 1023) {
        meta[0] = part[1023];
        meta[1] = (part[1023] + T - 1) / T;
    }
}

static __global__ void __launch_bounds__(1024) k_scatter_scan(int nvt, int T, const int *__restrict__ count,
                                                      int *__restrict__ cursor, int *__restrict__ meta,
                                                      const int *__restrict__ gate = nullptr)
{
    if (gate && !gate[1]) return;
    __shared__ int part[1024];
    scatter_scan_body(nvt, T, count, cursor, meta, part);
}

static __global__ void k_scatter_fill(int nt, int T, const ushort4 *__restrict__ pidx,
                               int *__restrict__ cursor, const int *__restrict__ meta,
                               uint32_t *__restrict__ ent, const int *__restrict__ gate = nullptr)
{
    if (gate && !gate[1]) return;
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nt) return;
    const int C = meta[1];
    const ushort4 q = pidx[l];
    const unsigned short d[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (d[k] == 0xFFFF) continue;
        const int pos = atomicAdd(cursor + d[k], 1);
        const int tt = pos / C, i = pos - tt * C;
        ent[(int64_t)i * T + tt] = ((uint32_t)d[k] << 16) | (k < 2 ? 0x8000u : 0u) | (uint32_t)l;
    }
}

// G mu = -D (Eqs. rinorm_a, correzione): the correction restores the
// conserved moments of h~, so its right-hand side is minus the conserved
// moments of the collision increment, D_a = sum_j psi_a (N_c,j - N_j), taken
// directly from the increment sums (never as the difference of the large
// post- and pre-collision sums).  P[0..13] are the moment sums of N_c over
// 1, vx, vy, vz, vx2, vy2, vz2, vxvy, vxvz, vyvz, vx v2, vy v2, vz v2, v4
// (they give G = G0 + eps sum_j N_c psi psi^T) and P[14..18] the increment
// sums D over 1, vx, vy, vz, v2.  Solved in registers by Gaussian
// elimination without pivoting (stable for the symmetric positive definite
// Gram matrix), then one step of iterative refinement whose residual
// -D - G mu is evaluated exactly with error-free products and sums and
// rounded once, so mu is as accurate as the FP32 entries of G and D allow.
// False if a pivot is not positive.  lane >= 0: all 32 lanes of a warp call
// it with the same P and their lane index, and lane a < 5 evaluates row a of
// the residual (the rest is the same on every lane).
__device__ __forceinline__ bool correction_spd(const Geo &g, const float *P, float *mu, int lane = -1)
{
    if (g.solve_fb) return false;
    const float e = g.epsf;
    const float p4 = P[4] + P[5] + P[6];
    const float m[5][5] = {
        {P[0], P[1], P[2], P[3], p4},
        {P[1], P[4], P[7], P[8], P[10]},
        {P[2], P[7], P[5], P[9], P[11]},
        {P[3], P[8], P[9], P[6], P[12]},
        {p4, P[10], P[11], P[12], P[13]}};
    float A[5][5], U[5][5], L[5][5], ip[5], b[5], x[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) {
#pragma unroll
        for (int c = 0; c < 5; ++c) A[a][c] = U[a][c] = g.G0f[a * 5 + c] + e * m[a][c];
        b[a] = -P[14 + a];
    }
#pragma unroll
    for (int kk = 0; kk < 5; ++kk) {
        const float piv = U[kk][kk];
        if (!(piv > 0.f)) return false;
        ip[kk] = 1.f / piv;
#pragma unroll
        for (int i = kk + 1; i < 5; ++i) {
            L[i][kk] = U[i][kk] * ip[kk];
#pragma unroll
            for (int j = kk + 1; j < 5; ++j) U[i][j] -= L[i][kk] * U[kk][j];
        }
    }
    // x = U^-1 L^-1 r, for the right-hand side and then the residual.
    auto lu_solve = [&](float (&r)[5], float (&y)[5]) {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            float s = r[i];
#pragma unroll
            for (int k = 0; k < i; ++k) s -= L[i][k] * r[k];
            r[i] = s;
        }
#pragma unroll
        for (int i = 4; i >= 0; --i) {
            float s = r[i];
#pragma unroll
            for (int j = i + 1; j < 5; ++j) s -= U[i][j] * y[j];
            y[i] = s * ip[i];
        }
    };
    float r[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) r[a] = b[a];
    lu_solve(r, x);
    // Row a of b - A x, exactly, rounded once.
    auto residual = [&](const float (&Ar)[5], float ba) {
        float hi = ba, lo = 0.f;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            float p, pe, s, se;
            two_prod(Ar[c], x[c], p, pe);
            two_sum(hi, -p, s, se);
            hi = s;
            lo = __fadd_rn(lo, __fsub_rn(se, pe));
        }
        return __fadd_rn(hi, lo);
    };
    if (lane < 0) {
#pragma unroll
        for (int a = 0; a < 5; ++a) r[a] = residual(A[a], b[a]);
    } else {
        float Ar[5], ba = 0.f;
#pragma unroll
        for (int c = 0; c < 5; ++c) Ar[c] = 0.f;
#pragma unroll
        for (int a = 0; a < 5; ++a)
            if (lane == a) {
#pragma unroll
                for (int c = 0; c < 5; ++c) Ar[c] = A[a][c];
                ba = b[a];
            }
        const float ra = residual(Ar, ba);
#pragma unroll
        for (int a = 0; a < 5; ++a) r[a] = __shfl_sync(0xFFFFFFFFu, ra, a);
    }
    float dx[5];
    lu_solve(r, dx);
#pragma unroll
    for (int a = 0; a < 5; ++a) mu[a] = x[a] + dx[a];
    return true;
}

// Sum K (<= 32) per-thread values over the block.  Inside a warp the values
// are transposed while being added (31 shuffles for any K <= 32, lane i ends
// with the warp total of value i); one thread per value then adds the warp
// totals.  Totals are stored in tot[0..K).
template <int K>
__device__ __forceinline__ void block_reduce4(float (&v)[K], float *red, float *tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    float x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = i < K ? v[i] : 0.f;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool up = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            float send = up ? x[i] : x[i + w];
            float keep = up ? x[i + w] : x[i];
            x[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, w);
        }
    }
    if (lane < K) red[warp * 32 + lane] = x[0];
    __syncthreads();
    if (threadIdx.x < K) {
        // Compensated sum of the warp totals.
        float s = 0.f, c = 0.f;
        for (int w = 0; w < nwarps; ++w) {
            float e;
            two_sum(s, red[w * 32 + threadIdx.x], s, e);
            c = __fadd_rn(c, e);
        }
        tot[threadIdx.x] = __fadd_rn(s, c);
    }
    __syncthreads();
}

__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }

// One upwind update of a quad (Eq. streaming2D, both signs handled by |Cu|).
__device__ __forceinline__ float4 upwind4(float4 h0, float4 hx, float4 hy, float ax, float ay)
{
    float4 o;
    o.x = h0.x - ax * (h0.x - hx.x) - ay * (h0.x - hy.x);
    o.y = h0.y - ax * (h0.y - hx.y) - ay * (h0.y - hy.y);
    o.z = h0.z - ax * (h0.z - hx.z) - ay * (h0.z - hy.z);
    o.w = h0.w - ax * (h0.w - hx.w) - ay * (h0.w - hy.w);
    return o;
}

// Free streaming alone (Eq. streaming2D) for FP32 states with a multiple-of-4
// velocity axis: each thread moves 16-byte quads of four jz nodes, one CTA
// per cell at a time in the strip order, interior cells without branches.
// SX: stretched cells (the cell's own widths scale its Courant numbers).
template <bool SX>
__global__ void __launch_bounds__(1024) k_stream4(Geo g, const float *__restrict__ hin,
                                                  const float *__restrict__ ghost,
                                                  float *__restrict__ hout)
{
    // blockDim.x is a multiple of Q: thread t keeps quad q = t mod Q of every
    // plane and walks the planes jx = t div Q, t div Q + blockDim.x / Q, ...
    __shared__ float scu[kMaxN];
    const int N = g.nv, nq = N / 4, Q = N * N / 4, half = N / 2;
    for (int i = threadIdx.x; i < N; i += blockDim.x) scu[i] = (float)(g.axv[i] * g.dt / g.dx);
    __syncthreads();
    const int64_t plane = g.nvt / 4;
    const float ry = (float)(g.dx / g.dy);
    const int q = threadIdx.x % Q, jxs = threadIdx.x / Q, jstep = blockDim.x / Q;
    const int jy = q / nq;
    float ay = fabsf(scu[jy] * ry), fx = 1.f;
    for (int kc = blockIdx.x; kc < g.nr; kc += gridDim.x) {
        const int c = cell_of(g, kc);
        const int ix = c % g.nx, iy = c / g.nx;
        if (SX) {
            // Courant factors of this cell: its own widths.
            fx = (float)g.sx[ix];
            ay = fabsf(scu[jy]) * (float)g.sy[iy];
        }
        const float4 *own = reinterpret_cast<const float4 *>(hin) + (int64_t)c * plane;
        float4 *dst = reinterpret_cast<float4 *>(hout) + (int64_t)c * plane;
        if (ix > 0 && ix < g.nx - 1 && iy > 0 && iy < g.ny - 1) {
            const float4 *ys = jy < half ? own + (int64_t)g.nx * plane : own - (int64_t)g.nx * plane;
            const float4 *xr = own + plane, *xl = own - plane;
#pragma unroll 4
            for (int jx = jxs; jx < N; jx += jstep) {
                const int o = jx * Q + q;
                const float4 hx = jx < half ? xr[o] : xl[o];
                dst[o] = upwind4(own[o], hx, ys[o], SX ? fabsf(scu[jx]) * fx : fabsf(scu[jx]), ay);
            }
        } else {
            for (int jx = jxs; jx < N; jx += jstep) {
                const int o = jx * Q + q;
                float4 hx, hy;
                if (jx < half) hx = ix < g.nx - 1 ? own[o + plane] : f4(ghost[(g.ny + iy) * N + jy]);
                else hx = ix > 0 ? own[o - plane] : f4(ghost[iy * N + jy]);
                if (jy < half)
                    hy = iy < g.ny - 1 ? own[o + (int64_t)g.nx * plane]
                                       : f4(ghost[(2 * g.ny + g.nx + ix) * N + jx]);
                else
                    hy = iy > 0 ? own[o - (int64_t)g.nx * plane] : f4(ghost[(2 * g.ny + ix) * N + jx]);
                dst[o] = upwind4(own[o], hx, hy, SX ? fabsf(scu[jx]) * fx : fabsf(scu[jx]), ay);
            }
        }
    }
}

// Eqs. densita..sforzi from float sums (see finalize_moments).
static __device__ __noinline__ void finalize_moments_f(const float *m, float e, double *o)
{
    const float rho = m[0], n = 1.f + e * rho;
    const float u[3] = {m[1] / n, m[2] / n, m[3] / n};
    o[0] = rho;
    o[1] = u[0];
    o[2] = u[1];
    o[3] = u[2];
    o[4] = ((2.f / 3.f) * (m[4] + m[5] + m[6]) - rho) / n -
           (2.f * e / 3.f) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k) o[5 + k] = 2.f * m[4 + k] - 2.f * e * n * u[pa[k]] * u[pb[k]];
}

// Per-instance shared tables of the FP32 cell kernel (N entries each).
__device__ __forceinline__ void cell4_setup(const Geo &g, const Cell4Smem &S)
{
    const int N = g.nv, T = blockDim.x, t = threadIdx.x;
    for (int i = t; i < N; i += T) {
        const double v = g.axv[i], A = g.axA[i];
        S.conv[i] = make_float4((float)A, (float)v, (float)(v * v), 0.f);
        S.gram[i] = make_float4((float)v, (float)(v * v), (float)(v * v * v), (float)(v * v * v * v));
        S.fin[i] = make_float4((float)(1.0 / A), 0.f, (float)A, (float)(A * v));
        S.Av2[i] = (float)(A * v * v);
        S.cu[i] = (float)(v * g.dt / g.dx);
        S.v[i] = (float)v;
        S.A[i] = (float)A;
        S.IA[i] = (float)(1.0 / A);
        S.rot[i] = i % (N / 4);
    }
    __syncthreads();
    for (int i = t; i < N / 4; i += T) {
        S.vzq[i] = make_float4(S.v[4 * i], S.v[4 * i + 1], S.v[4 * i + 2], S.v[4 * i + 3]);
        S.Azq[i] = make_float4(S.A[4 * i], S.A[4 * i + 1], S.A[4 * i + 2], S.A[4 * i + 3]);
        S.IAzq[i] = make_float4(S.IA[4 * i], S.IA[4 * i + 1], S.IA[4 * i + 2], S.IA[4 * i + 3]);
    }
    __syncthreads();
}

// One cell c of instance g: streaming into the slab (FUSED) or a copy of
// h~, the Monte Carlo gather and scatter, the correction and the write-back.
// Called by every thread of the CTA with the tables of g in place.
// What the adjoint mode of cell4_cell adds: two more slabs (N_c, then
// lam_c / w; dJ/dh~), 20 saved correction sums, a per-jx table, lam of the
// cell in and dJ/dh~ out (global, logical order), the sample set.
struct Adj4 {
    float4 *B, *C;
    float *P, *cxi;
    const float *lam;
    float *lt;
    const ushort4 *pidx;
    // The loss terms of the step (destination a or b of a sample), sorted by
    // destination in runs of lmeta[1] records per thread (k_adj_fill2);
    // lmeta[0] is their number.
    const uint4 *lrec;
    const int *lmeta;
};

// The adjoint's two lists of the step's terms.  The forward list: every
// (node, sample, sign) term, as for k_cell4 (k_scatter_fill).  The loss
// list of the transposed update: per sample with nodes (a, b, a*, b*) in the
// shared-memory order (0xFFFF outside the grid) and weight W, one record for
// each valid destination d in {a, b}:
//   {a* | b* << 16, a | b << 16, W, d | (d is b) << 16}.
// Counts, cursors and headers of the forward list come first, those of the
// loss list nvt entries (two ints) after them.
static __global__ void k_adj_count2(int nt, int nvt, const ushort4 *__restrict__ pidx,
                                    int *__restrict__ count)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nt) return;
    const ushort4 q = pidx[l];
    if (q.x != 0xFFFF) {
        atomicAdd(count + q.x, 1);
        atomicAdd(count + nvt + q.x, 1);
    }
    if (q.y != 0xFFFF) {
        atomicAdd(count + q.y, 1);
        atomicAdd(count + nvt + q.y, 1);
    }
    if (q.z != 0xFFFF) atomicAdd(count + q.z, 1);
    if (q.w != 0xFFFF) atomicAdd(count + q.w, 1);
}
static __global__ void __launch_bounds__(1024) k_adj_scan2(int nvt, int T, const int *__restrict__ count,
                                                           int *__restrict__ cursor, int *__restrict__ meta)
{
    __shared__ int part[1024];
    const int k = blockIdx.x;
    scatter_scan_body(nvt, T, count + k * nvt, cursor + k * nvt, meta + 2 * k, part);
}
static __global__ void k_adj_fill2(int nt, int nvt, int T, const ushort4 *__restrict__ pidx,
                                   const PlanA<float, uint16_t> *__restrict__ pa,
                                   int *__restrict__ cursor, const int *__restrict__ meta,
                                   uint32_t *__restrict__ ent, uint4 *__restrict__ rec)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nt) return;
    const ushort4 q = pidx[l];
    const unsigned short d[4] = {q.x, q.y, q.z, q.w};
    const int C = meta[1], CL = meta[3];
    const uint32_t gain = (uint32_t)q.z | ((uint32_t)q.w << 16), loss = (uint32_t)q.x | ((uint32_t)q.y << 16);
    const uint32_t W = __float_as_uint(pa[l].W);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (d[k] == 0xFFFF) continue;
        const int pos = atomicAdd(cursor + d[k], 1), tt = pos / C, i = pos - tt * C;
        ent[(int64_t)i * T + tt] = ((uint32_t)d[k] << 16) | (k < 2 ? 0x8000u : 0u) | (uint32_t)l;
        if (k < 2) {
            const int pl = atomicAdd(cursor + nvt + d[k], 1), tl = pl / CL, il = pl - tl * CL;
            rec[(int64_t)il * T + tl] = make_uint4(gain, loss, W, (uint32_t)d[k] | ((uint32_t)k << 16));
        }
    }
}

// x = G^{-1} rhs for the Gram matrix G = G0 + eps sum_j N_c,j psi_j psi_j^T
// of the correction (P[0..13] its moment sums, as in correction_spd), by
// elimination without pivoting (in registers; stable for the symmetric
// positive definite G); Cholesky, then pivoted elimination, if a pivot is not
// positive (fallback counted).
static __device__ __noinline__ void gram_solve(const Geo &g, const float *P, const float *rhs, float *x,
                                        int *fallback)
{
    const float e = g.epsf;
    const float p4 = P[4] + P[5] + P[6];
    const float m[5][5] = {
        {P[0], P[1], P[2], P[3], p4},
        {P[1], P[4], P[7], P[8], P[10]},
        {P[2], P[7], P[5], P[9], P[11]},
        {P[3], P[8], P[9], P[6], P[12]},
        {p4, P[10], P[11], P[12], P[13]}};
    float G[5][5], U[5][5], b[5], y[5];
    bool ok = !g.solve_fb;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
#pragma unroll
        for (int c = 0; c < 5; ++c) G[a][c] = U[a][c] = g.G0f[a * 5 + c] + e * m[a][c];
        b[a] = y[a] = rhs[a];
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        ok = ok && U[k][k] > 0.f;
        const float ip = 1.f / U[k][k];
#pragma unroll
        for (int i = k + 1; i < 5; ++i) {
            const float f = U[i][k] * ip;
#pragma unroll
            for (int j = k + 1; j < 5; ++j) U[i][j] -= f * U[k][j];
            y[i] -= f * y[k];
        }
    }
    if (ok) {
#pragma unroll
        for (int i = 4; i >= 0; --i) {
            float s = y[i];
#pragma unroll
            for (int j = i + 1; j < 5; ++j) s -= U[i][j] * x[j];
            x[i] = s / U[i][i];
        }
        return;
    }
    chol_or_ge<float>(G, b, x, fallback, g.solve_fb != 0);
}

// Adjoint part of one cell (after the forward recompute of cell4_cell in
// adjoint mode: S.slab4 holds h~, X.B holds N_c, muf[0..4] mu, X.P the sums
// of G).  With lam = dJ/dh^{n+1} of the cell:
//   nu = sum_j lam_j (1 + eps h_c,j) psi_j,  xi = G^{-1} nu,
//   lam_c,j = (lam_j - w_j psi_j.xi)(1 + eps psi_j.mu)      (dJ/dN_c times w)
//   dJ/dh~_j = lam_c,j + w_j psi_j.xi                        (N = w h~ and pre)
//   gamma_l = W_l (q_a* + q_b* - q_a - q_b),  q = lam_c / w  (dJ/d(g_l W_l))
//   dJ/dh~_a += gamma_l (1 + eps h~_b),  dJ/dh~_b += gamma_l (1 + eps h~_a).
__device__ __forceinline__ void adj4_tail(const Geo &g, const Map4 &m, int c, const Cell4Smem &S,
                                          const Adj4 &X, const PlanA<float, uint16_t> *__restrict__ pa,
                                          float *muf, int &fallback)
{
    const int N = g.nv, nvt = g.nvt, T = blockDim.x, t = threadIdx.x;
    const float eps = g.epsf;
    float *totf = reinterpret_cast<float *>(S.tot);
    const int Q = m.Q, nq = N / 4, q = t % Q, kchunk = t / Q;
    const bool active = kchunk < m.K;
    const int jy = q / nq, qz = q % nq, rowq = jy * nq;
    const int jx0 = active ? kchunk * m.J : 0, jx1 = active ? jx0 + m.J : 0;
    auto phys = [&](int jx) {
        int r = qz + S.rot[jx];
        r -= r >= nq ? nq : 0;
        return jx * Q + rowq + r;
    };
    const float vy = S.v[jy];

    // ---- nu, with lam of the cell staged into C ----------------------------
    float nu[5];
    {
        float a0 = 0.f, a1 = 0.f, a3 = 0.f, a4 = 0.f;
        if (active) {
            const float4 *lam4 = reinterpret_cast<const float4 *>(X.lam + (int64_t)c * nvt);
            const float4 z4 = S.vzq[qz], i4 = S.IAzq[qz];
            const float iay = S.IA[jy];
            const float vz[4] = {z4.x, z4.y, z4.z, z4.w};
            const float IAyz[4] = {iay * i4.x, iay * i4.y, iay * i4.z, iay * i4.w};
            float qq[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) qq[i] = vy * vy + vz[i] * vz[i];
#pragma unroll 2
            for (int jx = jx0; jx < jx1; ++jx) {
                const int o = phys(jx);
                const float4 n = X.B[o], l = lam4[jx * Q + q];
                X.C[o] = l;
                const float4 gv = S.gram[jx];      // v, v^2, v^3, v^4
                const float ia = S.IA[jx];
                const float nn[4] = {n.x, n.y, n.z, n.w}, ll[4] = {l.x, l.y, l.z, l.w};
                float ts = 0.f, tz = 0.f, tq = 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float hc = nn[i] * (ia * IAyz[i]);
                    const float tv = ll[i] * (1.f + eps * hc);
                    ts += tv;
                    tz += tv * vz[i];
                    tq += tv * qq[i];
                }
                a0 += ts;
                a1 += ts * gv.x;
                a3 += tz;
                a4 += ts * gv.y + tq;
            }
        }
        nu[0] = a0;
        nu[1] = a1;
        nu[2] = vy * a0;
        nu[3] = a3;
        nu[4] = a4;
    }
    block_reduce4<5>(nu, S.red, totf);
    float *xif = muf + 8;
    if (t == 0) gram_solve(g, X.P, totf, xif, &fallback);
    __syncthreads();
    for (int i = t; i < N; i += T) X.cxi[i] = xif[1] * S.v[i] + xif[4] * S.v[i] * S.v[i];
    __syncthreads();

    // ---- lam_c / w into B, lam_c + w psi.xi into C ---------------------------
    if (active) {
        const float4 z4 = S.vzq[qz], a4v = S.Azq[qz], i4 = S.IAzq[qz];
        const float ay = S.A[jy], iay = S.IA[jy];
        const float vz[4] = {z4.x, z4.y, z4.z, z4.w};
        const float Ayz[4] = {ay * a4v.x, ay * a4v.y, ay * a4v.z, ay * a4v.w};
        const float IAyz[4] = {iay * i4.x, iay * i4.y, iay * i4.z, iay * i4.w};
        float ctm[4], cti[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float qi = vy * vy + vz[i] * vz[i];
            ctm[i] = muf[0] + muf[2] * vy + muf[3] * vz[i] + muf[4] * qi;
            cti[i] = xif[0] + xif[2] * vy + xif[3] * vz[i] + xif[4] * qi;
        }
#pragma unroll 2
        for (int jx = jx0; jx < jx1; ++jx) {
            const int o = phys(jx);
            const float4 l = X.C[o];
            const float4 fv = S.fin[jx];          // 1/A, cx, A, A v
            const float cxi = X.cxi[jx];
            const float ll[4] = {l.x, l.y, l.z, l.w};
            float bq[4], cq[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float w = fv.z * Ayz[i], px = cti[i] + cxi, pm = ctm[i] + fv.y;
                const float lc = (ll[i] - w * px) * (1.f + eps * pm);
                bq[i] = lc * (fv.x * IAyz[i]);
                cq[i] = lc + w * px;
            }
            X.B[o] = make_float4(bq[0], bq[1], bq[2], bq[3]);
            X.C[o] = make_float4(cq[0], cq[1], cq[2], cq[3]);
        }
    }
    __syncthreads();

    // ---- transposed Monte Carlo update --------------------------------------
    // Each thread walks its run of the destination-sorted loss terms: the
    // term of sample l at its node d in {a, b} adds gamma_l (1 + eps h~_p),
    // p the other pre-collision node, to dJ/dh~_d.  A destination's sum is
    // added plainly once the run leaves it, atomically for the run's first
    // and last destinations (neighbouring runs may share them).
    {
        const float *Bf = reinterpret_cast<const float *>(X.B);
        const float *Af = reinterpret_cast<const float *>(S.slab4);
        float *Cf = reinterpret_cast<float *>(X.C);
        const int E = X.lmeta[0], C = X.lmeta[1];
        const int n = max(0, min(C, E - t * C));
        int cur = -1;
        bool first = true;
        float acc = 0.f;
        auto qv = [&](uint32_t i) { return i != 0xFFFFu ? Bf[i] : 0.f; };
        auto term = [&](uint4 r) {
            const float gam = __uint_as_float(r.z) * ((qv(r.x & 0xFFFFu) + qv(r.x >> 16)) -
                                                      (qv(r.y & 0xFFFFu) + qv(r.y >> 16)));
            const uint32_t p = (r.w >> 16) ? (r.y & 0xFFFFu) : (r.y >> 16);
            const float hp = p != 0xFFFFu ? Af[p] : 0.f;
            const int d = (int)(r.w & 0xFFFFu);
            if (d != cur) {
                if (cur >= 0) {
                    if (first) atomicAdd(Cf + cur, acc);
                    else Cf[cur] += acc;
                    first = false;
                }
                cur = d;
                acc = 0.f;
            }
            acc = fmaf(gam, fmaf(eps, hp, 1.f), acc);
        };
        const uint4 *rp = X.lrec + t;
        int i = 0;
        for (; i + 3 < n; i += 4) {
            uint4 r[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) r[u] = rp[(int64_t)(i + u) * T];
#pragma unroll
            for (int u = 0; u < 4; ++u) term(r[u]);
        }
        for (; i < n; ++i) term(rp[(int64_t)i * T]);
        if (cur >= 0) atomicAdd(Cf + cur, acc);
    }
    __syncthreads();

    // ---- dJ/dh~ of the cell out (logical order) ------------------------------
    if (active) {
        float4 *dst = reinterpret_cast<float4 *>(X.lt + (int64_t)c * nvt);
#pragma unroll 2
        for (int jx = jx0; jx < jx1; ++jx) dst[jx * Q + q] = X.C[phys(jx)];
    }
    __syncthreads();
}

template <bool FUSED, bool ADJ = false>
__device__ __forceinline__ void cell4_cell(const Geo &g, const Map4 &m, int c,
                                           const float *__restrict__ hin,
                                           const float *__restrict__ ghost,
                                           const PlanA<float, uint16_t> *__restrict__ pa,
                                           const uint32_t *__restrict__ ent,
                                           const int *__restrict__ meta, float *__restrict__ hout,
                                           double *__restrict__ mom, const Cell4Smem &S,
                                           int &fallback, long long *__restrict__ clk, int ncell,
                                           const Adj4 *X = nullptr)
{
    // The forward step works in place on one slab; the adjoint keeps h~ in
    // the slab and builds N, N_c in a second one.
    float4 *nsl = ADJ ? X->B : S.slab4;
    const int N = g.nv, nvt = g.nvt, T = blockDim.x, t = threadIdx.x;
    auto stamp = [&](int ph) {
        if (clk && blockIdx.x == 0 && t == 0 && ncell < kClkCells)
            clk[ncell * kClkPhases + ph] = clock64();
    };
    const float eps = g.epsf;
    float *totf = reinterpret_cast<float *>(S.tot);
    // Quad of this thread.
    const int Q = m.Q, nq = N / 4;
    const int q = t % Q, kchunk = t / Q;
    const bool active = kchunk < m.K;
    const int jy = q / nq, jz0 = 4 * (q % nq);
    const int jx0 = active ? kchunk * m.J : 0, jx1 = active ? jx0 + m.J : 0;
    (void)jz0;
    // Per-node constants of the quad (v_z, A_y A_z, 1/(A_y A_z), v_y^2 + v_z^2)
    // are re-read from shared tables inside each pass rather than kept live
    // across the whole cell: registers are the binding limit at 1024 threads.
#define QUAD_CONSTS                                                                  \
    const float vy = S.v[jy];                                                        \
    float vz[4], Ayz[4], IAyz[4], qq[4];                                             \
    {                                                                                \
        const float4 z4 = S.vzq[qz], a4 = S.Azq[qz], i4 = S.IAzq[qz];                \
        const float ay_ = S.A[jy], iay_ = S.IA[jy];                                  \
        vz[0] = z4.x; vz[1] = z4.y; vz[2] = z4.z; vz[3] = z4.w;                      \
        Ayz[0] = ay_ * a4.x; Ayz[1] = ay_ * a4.y; Ayz[2] = ay_ * a4.z; Ayz[3] = ay_ * a4.w; \
        IAyz[0] = iay_ * i4.x; IAyz[1] = iay_ * i4.y; IAyz[2] = iay_ * i4.z; IAyz[3] = iay_ * i4.w; \
        for (int i_ = 0; i_ < 4; ++i_) qq[i_] = vy * vy + vz[i_] * vz[i_];          \
    }                                                                                \
    (void)IAyz; (void)Ayz; (void)qq; (void)vz
    const float ry = g.ryf;
    const int half = N / 2;
    const int Q4 = Q;   // float4 stride of one jx-plane
    // Shared-memory position of this thread's quad in plane jx: quads of a row
    // are rotated by jx so that the jz-concentrated sample gathers spread over
    // all banks (the plan's node indices use the same order).
    const int qz = q % nq, rowq = jy * nq;
    auto phys = [&](int jx) {
        int r = qz + S.rot[jx];
        r -= r >= nq ? nq : 0;
        return jx * Q4 + rowq + r;
    };
    const int ix = c % g.nx, iy = c / g.nx;
    const float4 *own4 = reinterpret_cast<const float4 *>(hin + (int64_t)c * nvt);
    stamp(0);

    // ---- slab <- h~ ------------------------------------------------------
    if (active) {
        if (FUSED) {
            // Courant factors of this cell (its own widths on stretched grids).
            const float fx = g.sx ? (float)g.sx[ix] : 1.f, fy = g.sy ? (float)g.sy[iy] : ry;
            const float cuy = S.cu[jy] * fy, ay = fabsf(cuy);
            const int64_t plane = (int64_t)nvt / 4;
            if (ix > 0 && ix < g.nx - 1 && iy > 0 && iy < g.ny - 1) {
                // Interior cell: all upwind sources are neighbour slabs.
                const float4 *ys = cuy > 0.f ? own4 - (int64_t)g.nx * plane
                                             : own4 + (int64_t)g.nx * plane;
                const float4 *xr = own4 + plane, *xl = own4 - plane;
                const int e = min(jx1, half), b = max(jx0, half);
                if (!g.sx) {
#pragma unroll 4
                    for (int jx = jx0; jx < e; ++jx) {
                        const int o = jx * Q4 + q;
                        const float4 h0 = own4[o], hx = xr[o], hy = ys[o];
                        S.slab4[phys(jx)] = upwind4(h0, hx, hy, fabsf(S.cu[jx]), ay);
                    }
#pragma unroll 4
                    for (int jx = b; jx < jx1; ++jx) {
                        const int o = jx * Q4 + q;
                        const float4 h0 = own4[o], hx = xl[o], hy = ys[o];
                        S.slab4[phys(jx)] = upwind4(h0, hx, hy, fabsf(S.cu[jx]), ay);
                    }
                } else {
                    for (int jx = jx0; jx < e; ++jx) {
                        const int o = jx * Q4 + q;
                        const float4 h0 = own4[o], hx = xr[o], hy = ys[o];
                        S.slab4[phys(jx)] = upwind4(h0, hx, hy, fabsf(S.cu[jx]) * fx, ay);
                    }
                    for (int jx = b; jx < jx1; ++jx) {
                        const int o = jx * Q4 + q;
                        const float4 h0 = own4[o], hx = xl[o], hy = ys[o];
                        S.slab4[phys(jx)] = upwind4(h0, hx, hy, fabsf(S.cu[jx]) * fx, ay);
                    }
                }
            } else {
                const float4 *ys = nullptr;
                const float *yg = nullptr;
                if (cuy > 0.f) {
                    if (iy > 0) ys = own4 - (int64_t)g.nx * plane;
                    else yg = ghost + (2 * g.ny + ix) * N;
                } else {
                    if (iy < g.ny - 1) ys = own4 + (int64_t)g.nx * plane;
                    else yg = ghost + (2 * g.ny + g.nx + ix) * N;
                }
                for (int jx = jx0; jx < jx1; ++jx) {
                    const int o = jx * Q4 + q;
                    const float4 h0 = own4[o];
                    float4 hx;
                    if (jx < half)   // v_x < 0: right neighbour or right-wall ghost
                        hx = ix < g.nx - 1 ? own4[plane + o] : f4(ghost[(g.ny + iy) * N + jy]);
                    else             // v_x > 0: left neighbour or left-wall ghost
                        hx = ix > 0 ? own4[o - plane] : f4(ghost[iy * N + jy]);
                    const float4 hy = ys ? ys[o] : f4(yg[jx]);
                    S.slab4[phys(jx)] = upwind4(h0, hx, hy, fabsf(S.cu[jx]) * fx, ay);
                }
            }
        } else {
#pragma unroll 4
            for (int jx = jx0; jx < jx1; ++jx) S.slab4[phys(jx)] = own4[jx * Q4 + q];
        }
    }
    __syncthreads();

    stamp(1);
    // ---- phase A: g_l W_l on h~ (Jacobi) into shared memory ---------------
    {
        const float *slab = reinterpret_cast<const float *>(S.slab4);
        int l = t;
        for (; l + 15 * T < g.nt; l += 16 * T) {
            PlanA<float, uint16_t> rec[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) rec[u] = pa[l + u * T];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int a = rec[u].a(), b = rec[u].b();
                const float ha = a >= 0 ? slab[a] : 0.f;
                const float hb = b >= 0 ? slab[b] : 0.f;
                S.gw[l + u * T] = (ha + hb + eps * ha * hb) * rec[u].W;
            }
        }
        for (; l < g.nt; l += T) {
            const PlanA<float, uint16_t> r = pa[l];
            const int a = r.a(), b = r.b();
            const float ha = a >= 0 ? slab[a] : 0.f;
            const float hb = b >= 0 ? slab[b] : 0.f;
            S.gw[l] = (ha + hb + eps * ha * hb) * r.W;
        }
    }
    __syncthreads();

    stamp(2);
    // ---- N = w h~ in place, with the invariants of h~ ----------------------
    float p0 = 0.f, p1 = 0.f, p3 = 0.f, p4 = 0.f;
    if (active) {
        QUAD_CONSTS;
#pragma unroll 4
        for (int jx = jx0; jx < jx1; ++jx) {
            const int o = phys(jx);
            float4 h = S.slab4[o];
            const float4 cv = S.conv[jx];        // {A, v, v^2, -}
            float n0 = h.x * (cv.x * Ayz[0]), n1 = h.y * (cv.x * Ayz[1]);
            float n2 = h.z * (cv.x * Ayz[2]), n3 = h.w * (cv.x * Ayz[3]);
            nsl[o] = make_float4(n0, n1, n2, n3);
            const float sn = (n0 + n1) + (n2 + n3);
            p0 += sn;
            p1 += sn * cv.y;
            p3 += n0 * vz[0] + n1 * vz[1] + n2 * vz[2] + n3 * vz[3];
            p4 += n0 * (cv.z + qq[0]) + n1 * (cv.z + qq[1]) + n2 * (cv.z + qq[2]) +
                  n3 * (cv.z + qq[3]);
        }
    }
    __syncthreads();

    stamp(3);
    // ---- phase B: gains and losses (Eq. monteCarloInt) --------------------
    // Each thread walks its run of the destination-sorted list, sums the
    // terms of one node in a register and adds the sum with one atomic.
    {
        float *slabw = reinterpret_cast<float *>(nsl);
        const int E = meta[0], C = meta[1];
        const int base = t * C, n = max(0, min(C, E - base));
        // Only the first and the last node of a run can be shared with the
        // neighbouring runs; they are added atomically, the others plainly.
        int cur = -1;
        bool first = true;
        float acc = 0.f;
        auto flush = [&](bool shared) {
            if (cur >= 0 && acc != 0.f) {
                if (shared) atomicAdd(slabw + cur, acc);
                else slabw[cur] += acc;
            }
        };
        auto term = [&](uint32_t w, float r) {
            const int dest = (int)(w >> 16);
            if (dest != cur) {
                flush(first);
                first = cur < 0;
                cur = dest;
                acc = 0.f;
            }
            acc += (w & 0x8000u) ? -r : r;
        };
        int i = 0;
        for (; i + 7 < n; i += 8) {
            uint32_t w[8];
            float r[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) w[u] = ent[(int64_t)(i + u) * T + t];
#pragma unroll
            for (int u = 0; u < 8; ++u) r[u] = S.gw[w[u] & 0x7FFFu];   // before any flush
#pragma unroll
            for (int u = 0; u < 8; ++u) term(w[u], r[u]);
        }
        for (; i < n; ++i) {
            const uint32_t w = ent[(int64_t)i * T + t];
            term(w, S.gw[w & 0x7FFFu]);
        }
        flush(true);
    }
    __syncthreads();

    stamp(4);
    // ---- moments of N_c for the correction (post pass) --------------------
    float acc[19];
    {
        QUAD_CONSTS;
        float s[4][5];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 5; ++k) s[i][k] = 0.f;
        if (active) {
#pragma unroll 2
            for (int jx = jx0; jx < jx1; ++jx) {
                float4 n = nsl[phys(jx)];
                const float4 gv = S.gram[jx];   // v, v^2, v^3, v^4
                const float nn[4] = {n.x, n.y, n.z, n.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    s[i][0] += nn[i];
                    s[i][1] += nn[i] * gv.x;
                    s[i][2] += nn[i] * gv.y;
                    s[i][3] += nn[i] * gv.z;
                    s[i][4] += nn[i] * gv.w;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 19; ++k) acc[k] = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float z = vz[i], qi = qq[i];
            const float s0 = s[i][0], s1 = s[i][1], s2 = s[i][2], s3 = s[i][3], s4 = s[i][4];
            acc[0] += s0;
            acc[1] += s1;
            acc[2] += vy * s0;
            acc[3] += z * s0;
            acc[4] += s2;
            acc[5] += vy * vy * s0;
            acc[6] += z * z * s0;
            acc[7] += vy * s1;
            acc[8] += z * s1;
            acc[9] += vy * z * s0;
            acc[10] += s3 + qi * s1;
            acc[11] += vy * (s2 + qi * s0);
            acc[12] += z * (s2 + qi * s0);
            acc[13] += s4 + 2.f * qi * s2 + qi * qi * s0;
        }
        // The thread's share of the increment sums D (post minus pre over
        // its own nodes, so only thread-sized partial sums cancel).
        acc[14] = acc[0] - p0;
        acc[15] = acc[1] - p1;
        acc[16] = acc[2] - vy * p0;
        acc[17] = acc[3] - p3;
        acc[18] = (acc[4] + acc[5] + acc[6]) - p4;
    }
    block_reduce4<19>(acc, S.red, totf);
    stamp(5);

    // ---- correction solve (warp 0, which shares the residual of the
    // refinement) and per-cell tables --------------------------------------
    float *muf = reinterpret_cast<float *>(S.mu);
    if (t < 32) {
        float mu5[5];
        const bool ok = correction_spd(g, totf, mu5, t);
        if (t == 0) {
            if (ok) {
                for (int a = 0; a < 5; ++a) muf[a] = mu5[a];
            } else {
                double m8[5], Pd[19];
                for (int a = 0; a < 19; ++a) Pd[a] = (double)totf[a];
                int f2 = 0;
                correction_solve<float>(g, Pd, m8, &f2);
                ++fallback;
                for (int a = 0; a < 5; ++a) muf[a] = (float)m8[a];
            }
            if constexpr (ADJ)
                for (int a = 0; a < 14; ++a) X->P[a] = totf[a];
        }
    }
    __syncthreads();
    const float mu0 = muf[0], mux = muf[1], muy = muf[2], muz = muf[3], mu4 = muf[4];
    for (int i = t; i < N; i += T) S.fin[i].y = mux * S.v[i] + mu4 * S.v[i] * S.v[i];
    __syncthreads();
    stamp(6);

    if constexpr (ADJ) {
        adj4_tail(g, m, c, S, *X, pa, muf, fallback);
        return;
    }

    // ---- corrected write-back and output moments ---------------------------
    float mo[10];
    {
        QUAD_CONSTS;
        float tt[4][3];
#pragma unroll
        for (int i = 0; i < 4; ++i) tt[i][0] = tt[i][1] = tt[i][2] = 0.f;
        float ct[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) ct[i] = mu0 + muy * vy + muz * vz[i] + mu4 * qq[i];
        if (active) {
            float4 *dst4 = reinterpret_cast<float4 *>(hout + (int64_t)c * nvt);
#pragma unroll 2
            for (int jx = jx0; jx < jx1; ++jx) {
                const int o = jx * Q4 + q;
                float4 n = S.slab4[phys(jx)];
                const float4 fv = S.fin[jx];        // 1/A, cx, A, A v
                const float av2 = S.Av2[jx];
                const float nn[4] = {n.x, n.y, n.z, n.w};
                float hn[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float hc = nn[i] * (fv.x * IAyz[i]);
                    const float corr = ct[i] + fv.y;
                    hn[i] = hc + (1.f + eps * hc) * corr;
                    tt[i][0] += hn[i] * fv.z;
                    tt[i][1] += hn[i] * fv.w;
                    tt[i][2] += hn[i] * av2;
                }
                dst4[o] = make_float4(hn[0], hn[1], hn[2], hn[3]);
            }
        }
#pragma unroll
        for (int k = 0; k < 10; ++k) mo[k] = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float a = Ayz[i], z = vz[i];
            const float t0 = a * tt[i][0], t1 = a * tt[i][1], t2 = a * tt[i][2];
            mo[0] += t0;
            mo[1] += t1;
            mo[2] += vy * t0;
            mo[3] += z * t0;
            mo[4] += t2;
            mo[5] += vy * vy * t0;
            mo[6] += z * z * t0;
            mo[7] += vy * t1;
            mo[8] += z * t1;
            mo[9] += vy * z * t0;
        }
    }
    stamp(7);
    block_reduce4<10>(mo, S.red, totf);
    if (t == 0 && mom) finalize_moments_f(totf, eps, mom + (int64_t)c * 11);
    __syncthreads();
    stamp(8);
}

template <bool FUSED, int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
k_cell4(Geo g, Map4 m, const float *__restrict__ hin, const float *__restrict__ ghost,
        const PlanA<float, uint16_t> *__restrict__ pa, const uint32_t *__restrict__ ent,
        const int *__restrict__ meta, float *__restrict__ hout, double *__restrict__ mom,
        unsigned long long *__restrict__ stats, long long *__restrict__ clk,
        const int *__restrict__ gate = nullptr)
{
    if (gate && !gate[1]) return;
    extern __shared__ __align__(16) char smem_raw[];
    const Cell4Smem S = carve4(smem_raw, g.nv, g.nvt);
    cell4_setup(g, S);
    int fallback = 0, ncell = 0;
    for (int kc = blockIdx.x; kc < g.nr; kc += gridDim.x, ++ncell)
        cell4_cell<FUSED>(g, m, cell_of(g, kc), hin, ghost, pa, ent, meta, hout, mom, S,
                          fallback, clk, ncell);
    if (fallback && stats) atomicAdd(stats + 3, (unsigned long long)fallback);
}


// dJ/dh^n from dJ/dh~ (FP32, velocity axis a multiple of 4): the transposed
// upwind stencil (h^n_c feeds h~ of its downwind neighbours: right for v_x >
// 0, above for v_y > 0) in 16-byte quads of four jz nodes, plus on boundary
// cells the outgoing-flux terms lF[f] |v_n| w of their faces and on the lid
// row the lid-shear term wD 2 w v_x v_y / nx.  blockDim a multiple of Q.
static __global__ void __launch_bounds__(1024) k_adj_stream4(Geo g, const float *__restrict__ lt,
                                                             const double *__restrict__ lF,
                                                             float *__restrict__ lam_out, double wD)
{
    __shared__ float sv[kMaxN], sax[kMaxN], say[kMaxN], sA[kMaxN];
    const int N = g.nv, nq = N / 4, Q = N * N / 4, half = N / 2;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double v = g.axv[i];
        sv[i] = (float)v;
        sax[i] = (float)(fabs(v) * g.dt / g.dx);
        say[i] = (float)(fabs(v) * g.dt / g.dy);
        sA[i] = (float)g.axA[i];
    }
    __syncthreads();
    const int64_t plane = g.nvt / 4;
    const int q = threadIdx.x % Q, jxs = threadIdx.x / Q, jstep = blockDim.x / Q;
    const int jy = q / nq, jz0 = 4 * (q % nq);
    const float vy = sv[jy], ay = say[jy];
    const float dcoef = (float)(wD * 2.0 / g.nx);
    for (int kc = blockIdx.x; kc < g.nr; kc += gridDim.x) {
        const int c = cell_of(g, kc);
        const int ix = c % g.nx, iy = c / g.nx;
        const float4 *own = reinterpret_cast<const float4 *>(lt) + (int64_t)c * plane;
        float4 *dst = reinterpret_cast<float4 *>(lam_out) + (int64_t)c * plane;
        // Downwind y neighbour of this thread's row (v_y > 0: above).
        const float4 *ys = own + (jy >= half ? (int64_t)g.nx : -(int64_t)g.nx) * plane;
        if (ix > 0 && ix < g.nx - 1 && iy > 0 && iy < g.ny - 1) {
            // Interior cell: both downwind neighbours are cells.
            const float4 *xr = own + plane, *xl = own - plane;
#pragma unroll 4
            for (int jx = jxs; jx < N; jx += jstep) {
                const int o = jx * Q + q;
                const float ax = sax[jx];
                const float4 l0 = own[o], lx = jx >= half ? xr[o] : xl[o], ly = ys[o];
                const float c0 = 1.f - ax - ay;
                dst[o] = make_float4(c0 * l0.x + ax * lx.x + ay * ly.x, c0 * l0.y + ax * lx.y + ay * ly.y,
                                     c0 * l0.z + ax * lx.z + ay * ly.z, c0 * l0.w + ax * lx.w + ay * ly.w);
            }
            continue;
        }
        const bool yd = jy >= half ? iy < g.ny - 1 : iy > 0;
        for (int jx = jxs; jx < N; jx += jstep) {
            const int o = jx * Q + q;
            const float ax = sax[jx];
            const bool xd = jx >= half ? ix < g.nx - 1 : ix > 0;   // v_x > 0: right
            const float4 l0 = own[o];
            const float4 lx = xd ? own[o + (jx >= half ? plane : -plane)] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 ly = yd ? ys[o] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 r;
            const float c0 = 1.f - ax - ay;
            r.x = c0 * l0.x + ax * lx.x + ay * ly.x;
            r.y = c0 * l0.y + ax * lx.y + ay * ly.y;
            r.z = c0 * l0.z + ax * lx.z + ay * ly.z;
            r.w = c0 * l0.w + ax * lx.w + ay * ly.w;
            const float vx = sv[jx];
            float ex = 0.f;
            if (ix == 0 && vx < 0.f) ex -= (float)lF[iy] * vx;
            if (ix == g.nx - 1 && vx > 0.f) ex += (float)lF[g.ny + iy] * vx;
            if (iy == 0 && vy < 0.f) ex -= (float)lF[2 * g.ny + ix] * vy;
            float dl = 0.f;
            if (iy == g.ny - 1 && vy > 0.f) {
                ex += (float)lF[2 * g.ny + g.nx + ix] * vy;
                dl = dcoef * vx * vy;
            }
            const float wxy = sA[jx] * sA[jy];
            float *rr = &r.x;
#pragma unroll
            for (int i = 0; i < 4; ++i) rr[i] += (ex + dl) * wxy * sA[jz0 + i];
            dst[o] = r;
        }
    }
}

// The per-sample products of the forward gather live in the last adjoint
// slab when they fit (that slab is first used after them).
__host__ __device__ inline bool adj4_gw_in_slab(int nvt, int nt) { return nt <= nvt; }

// Shared-memory bytes of k_adj_cell4: those of k_cell4 plus two slabs, the
// saved correction sums and one per-jx table.
__host__ __device__ inline size_t adj4_smem_bytes(int nv, int nvt, int nt)
{
    size_t off = (cell4_smem_bytes(nv, nvt, adj4_gw_in_slab(nvt, nt) ? 0 : nt) + 15) & ~(size_t)15;
    return off + 2 * sizeof(float) * nvt + sizeof(float) * (16 + nv);
}

// Forward recompute and adjoint of the per-cell relaxation of one step for
// every cell (FP32 fast path): lt = dJ/dh~ from lam = dJ/dh^{n+1}.
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1024 / MAXT)
k_adj_cell4(Geo g, Map4 m, const float *__restrict__ hin, const float *__restrict__ ghost,
            const ushort4 *__restrict__ pidx, const PlanA<float, uint16_t> *__restrict__ pa,
            const uint32_t *__restrict__ ent, const int *__restrict__ meta,
            const uint4 *__restrict__ lrec, const int *__restrict__ lmeta,
            const float *__restrict__ lam, float *__restrict__ lt,
            unsigned long long *__restrict__ stats)
{
    extern __shared__ __align__(16) char smem_raw[];
    Cell4Smem S = carve4(smem_raw, g.nv, g.nvt);
    Adj4 X;
    {
        const bool gin = adj4_gw_in_slab(g.nvt, g.nt);
        size_t off = (cell4_smem_bytes(g.nv, g.nvt, gin ? 0 : g.nt) + 15) & ~(size_t)15;
        X.B = reinterpret_cast<float4 *>(smem_raw + off);
        X.C = X.B + g.nvt / 4;
        X.P = reinterpret_cast<float *>(X.C + g.nvt / 4);
        X.cxi = X.P + 16;
        X.lam = lam;
        X.lt = lt;
        X.pidx = pidx;
        X.lrec = lrec;
        X.lmeta = lmeta;
        if (gin) S.gw = reinterpret_cast<float *>(X.C);
    }
    cell4_setup(g, S);
    int fallback = 0;
    for (int kc = blockIdx.x; kc < g.nr; kc += gridDim.x)
        cell4_cell<true, true>(g, m, cell_of(g, kc), hin, ghost, pa, ent, meta, nullptr, nullptr,
                               S, fallback, nullptr, 0, &X);
    if (fallback && stats) atomicAdd(stats + 3, (unsigned long long)fallback);
}

}  // namespace bzk
