// bz_kernels.cuh -- sm_103a kernels of the semi-regular Boltzmann step.
//
// Method: Frezzotti, Ghiroldi & Gibelli, "Solving the Boltzmann equation on
// GPUs" (Secs. 2-4).  One time step is
//   k_walls   wall densities n_w and emitted ghost values (Eq. bcMax)
//   k_plan    the shared Monte Carlo sample set (Sec. 4.2, Algorithm 2)
//   k_fused   per spatial cell: upwind streaming into a shared-memory slab
//             (Eq. streaming2D), Jacobi Monte Carlo collision update
//             (Eqs. monteCarloInt, collision_step), conservation correction
//             (Eqs. rinorm_a, correzione) and the moments (Eqs. densita..sforzi)
// with k_stream + k_collide as the unfused equivalent.
//
// Layout: h[cell][j], j = (jx*N + jy)*N + jz.  A CTA owns one cell at a time;
// thread t owns the velocity "pairs" p = jy*N + jz with p = t (mod T) and
// walks jx, so a warp touches 32 consecutive nodes (coalesced global access,
// conflict-free shared access) and every per-node weight factorises as
// A[jx] * A[jy] * A[jz] with A(v) = dv pi^{-1/2} e^{-v^2}.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bzk {

constexpr int kMaxThreads = 1024;
constexpr int kMaxWarps = kMaxThreads / 32;
constexpr int kMaxN = 64;          // velocity nodes per axis
constexpr int kRedSlots = 20;      // values per block reduction

// Problem description shared by every kernel (by value).
struct Geo {
    int nx, ny, nv, nvt, nr, nfaces;
    int nt;                     // Monte Carlo samples per step
    double vmax, dv, dt, dx, dy, eps, cw;   // cw = pi K dt / Nt
    float epsf, ryf;            // eps and dx / dy rounded to float (no FP64 per cell)
    uint32_t seed, instance;
    double lid_u0, lid_amp, lid_period;
    const double *lid_profile;  // device, nx, or nullptr
    const double *axv;          // device, nv: node velocity per axis
    const double *axA;          // device, nv: dv pi^{-1/2} exp(-v^2)
    // Wall flux constants (Eq. bcMax with discrete sums):
    double cout;                // sum_{v_n<0} |v_n| w_j (same for all walls)
    double hn;                  // sum_{v_n>0} v_n A(v_n)
    double zsum;                // sum_z A(v_z)
    double G0[25];              // sum_j w_j psi_a psi_b, psi = (1, v, v^2)
    float G0f[25];              // the same, rounded to float
    int swz;                    // plan node indices in the quad-rotated shared-memory order
    int strip;                  // cells are visited in column strips of this width
    int solve_fb;               // 1: every correction solve takes its pivoted fallback (tests)
    // Stretched grids (nullptr when uniform).  axe: nv + 1 velocity cell
    // edges; axd: nv widths; sx, sy: per column / row, dx / dx_i and
    // dx / dy_j (the Courant numbers are cu(v) times these); wlid: per lid
    // face, dx_i / L (the weights of the lid-shear mean).
    const double *axe, *axd;
    const double *sx, *sy;
    const double *wlid;
    float vmaxf, idvf, cwf;     // vmax, 1 / dv and cw rounded to float (FP32 sampling)
    int redraw_cap;             // per-cell FP32 sampling: FP64 redraw queue entries (-1: all)
};

// Visiting order of the cells by the persistent per-cell kernels: column
// strips of width g.strip, row by row inside a strip, so that the cells in
// flight at any time form a compact block and the upwind neighbour slabs
// (left/right and below/above) are read from L2 rather than HBM.
__device__ __forceinline__ int cell_of(const Geo &g, int k)
{
    const int S = g.strip, full = g.nx / S, inFull = full * S * g.ny;
    if (k < inFull) {
        const int s = k / (S * g.ny), r = k - s * S * g.ny;
        return (r / S) * g.nx + s * S + r % S;
    }
    const int R = g.nx - full * S, kk = k - inFull;
    return (kk / R) * g.nx + full * S + kk % R;
}

// ---------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11)
// ---------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t lo0 = m0 * c.x, hi0 = __umulhi(m0, c.x);
        uint32_t lo1 = m1 * c.z, hi1 = __umulhi(m1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

static __global__ void k_philox(uint2 key, const uint4 *__restrict__ ctr, uint4 *__restrict__ out,
                         int64_t n)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], key);
}

// ---------------------------------------------------------------------
// Sampling (Eq. coll8Dim; Sec. 4.2).  All arithmetic that decides a node
// index is IEEE double with explicit rounding intrinsics (no contraction).
// ---------------------------------------------------------------------
__device__ __forceinline__ double u01(uint32_t x)
{
    return __dmul_rn(__dadd_rn((double)x, 0.5), 2.3283064365386962890625e-10);
}

__device__ __forceinline__ int node_axis(double v, double vmax, double dv, int n, int *near)
{
    double t = __ddiv_rn(__dadd_rn(v, vmax), dv);
    double fl = floor(t);
    double fr = __dsub_rn(t, fl);
    if (fr < 1e-9 || fr > 1.0 - 1e-9) *near = 1;
    if (!(t >= 0.0) || fl >= (double)n) return -1;
    return (int)fl;
}

__device__ __forceinline__ int node_of(const double v[3], double vmax, double dv, int n,
                                       int *near)
{
    int a = node_axis(v[0], vmax, dv, n, near);
    int b = node_axis(v[1], vmax, dv, n, near);
    int c = node_axis(v[2], vmax, dv, n, near);
    if (a < 0 || b < 0 || c < 0) return -1;
    return (a * n + b) * n + c;
}

// Stretched velocity cells: the cell k with e[k] <= v < e[k+1] (a value on
// an edge belongs to the upper cell), by bisection over the n + 1 edges.
__device__ __forceinline__ int node_axis_edges(double v, const double *__restrict__ e, int n,
                                               int *near)
{
    if (!(v >= e[0]) || v >= e[n]) return -1;
    int lo = 0, hi = n - 1;                  // e[lo] <= v < e[hi + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (v >= e[mid]) lo = mid;
        else hi = mid - 1;
    }
    const double w = __dsub_rn(e[lo + 1], e[lo]);
    if (__dsub_rn(v, e[lo]) < 1e-9 * w || __dsub_rn(e[lo + 1], v) < 1e-9 * w) *near = 1;
    return lo;
}

__device__ __forceinline__ int node_of(const double v[3], const Geo &g, int *near)
{
    if (!g.axe) return node_of(v, g.vmax, g.dv, g.nv, near);
    const int n = g.nv;
    int a = node_axis_edges(v[0], g.axe, n, near);
    int b = node_axis_edges(v[1], g.axe, n, near);
    int c = node_axis_edges(v[2], g.axe, n, near);
    if (a < 0 || b < 0 || c < 0) return -1;
    return (a * n + b) * n + c;
}

struct SampleOut {
    int idx[4];
    double W;
    int near, outside;
};

__device__ __forceinline__ SampleOut draw_sample(const Geo &g, int64_t step, uint32_t cellword,
                                                 uint32_t l)
{
    uint2 key = make_uint2(g.seed, g.instance);
    uint4 a = philox4x32_10(make_uint4(l, (uint32_t)step, cellword, 0u), key);
    uint4 b = philox4x32_10(make_uint4(l, (uint32_t)step, cellword, 1u), key);
    const double twopi = 6.283185307179586;
    // Box-Muller pairs: normals of variance 1/2 match Phi0 = pi^{-3/2} e^{-v^2}.
    double r0 = __dsqrt_rn(-log(u01(a.x))), t0 = __dmul_rn(twopi, u01(a.y));
    double r1 = __dsqrt_rn(-log(u01(a.z))), t1 = __dmul_rn(twopi, u01(a.w));
    double r2 = __dsqrt_rn(-log(u01(b.x))), t2 = __dmul_rn(twopi, u01(b.y));
    double v[3], v1[3], k[3];
    v[0] = __dmul_rn(r0, cos(t0));
    v[1] = __dmul_rn(r0, sin(t0));
    v[2] = __dmul_rn(r1, cos(t1));
    v1[0] = __dmul_rn(r1, sin(t1));
    v1[1] = __dmul_rn(r2, cos(t2));
    v1[2] = __dmul_rn(r2, sin(t2));
    // Unit vector on the sphere through (k_z, phi).
    double kz = __dsub_rn(1.0, __dmul_rn(2.0, u01(b.z)));
    double ph = __dmul_rn(twopi, u01(b.w));
    double st = __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(kz, kz)));
    k[0] = __dmul_rn(st, cos(ph));
    k[1] = __dmul_rn(st, sin(ph));
    k[2] = kz;
    // v* = v + (v_r.k) k, v1* = v1 - (v_r.k) k with v_r = v1 - v (Algorithm 2).
    double vr0 = __dsub_rn(v1[0], v[0]), vr1 = __dsub_rn(v1[1], v[1]),
           vr2 = __dsub_rn(v1[2], v[2]);
    double s = __dadd_rn(__dadd_rn(__dmul_rn(vr0, k[0]), __dmul_rn(vr1, k[1])),
                         __dmul_rn(vr2, k[2]));
    double vs[3], v1s[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double sk = __dmul_rn(s, k[c]);
        vs[c] = __dadd_rn(v[c], sk);
        v1s[c] = __dsub_rn(v1[c], sk);
    }
    SampleOut o;
    int near = 0;
    o.idx[0] = node_of(v, g, &near);
    o.idx[1] = node_of(v1, g, &near);
    o.idx[2] = node_of(vs, g, &near);
    o.idx[3] = node_of(v1s, g, &near);
    o.near = near;
    o.outside = (o.idx[0] < 0) | (o.idx[1] < 0) | (o.idx[2] < 0) | (o.idx[3] < 0);
    o.W = __dmul_rn(g.cw, fabs(s));
    return o;
}

// The same sample in FP32, for FP32 states on uniform velocity grids.  The
// coordinates that pick nodes are computed in FP32 with a bounded error: the
// uniforms and k_z are rounded once from their integers, -ln u near u = 1
// comes from the exact complement 1 - u, sin(theta) = 2 sqrt(u (1 - u)), and
// the angles 2 pi u are split into a float part for sincospif and an exact
// remainder added to first order.  With CUDA's 1-ulp bounds for logf, log1pf
// and sincospif this keeps every coordinate of v and v1 within 1.3e-6 of its
// exact value and every coordinate of v* and v1* within 2.4e-5 (|v| < 4.8 by
// the Box-Muller radius at the smallest uniform).  A coordinate closer to a
// cell face than about four times its bound (kFastMarginA / kFastMarginB, in
// velocity units, plus the rounding of the cell coordinate itself) sets
// *redo: the caller draws that sample again with draw_sample.  Every other
// sample selects exactly the nodes of the FP64 computation.  W = cw |s|
// carries the FP32 error of s (at most 1.6e-5 absolute).
constexpr float kFastMarginA = 6e-6f;    // v, v1
constexpr float kFastMarginB = 1e-4f;    // v*, v1*

// u = (x + 1/2) 2^-32 with a single rounding to float.
__device__ __forceinline__ float u01f(uint32_t x)
{
    return __fmaf_rn((float)(x & 255u) + 0.5f, 0x1p-32f, (float)(x >> 8) * 0x1p-24f);
}
// -ln u for u = (x + 1/2) 2^-32 (near u = 1 from 1 - u = (~x + 1/2) 2^-32).
__device__ __forceinline__ float neglog_u01f(uint32_t x)
{
    if (x < 0x80000000u) return -logf(u01f(x));
    return -log1pf(-u01f(~x));
}
// (sin, cos) of 2 pi u for u = (x + 1/2) 2^-32: with x read as a signed
// integer the angle is pi t, t = (x + 1/2) 2^-31 in [-1, 1), split exactly
// into th = (x >> 8) 2^-23 and the remainder tl < 1.2e-7, whose rotation is
// added to first order (the dropped term is below 1e-13).
__device__ __forceinline__ void sincos_2pi_u01f(uint32_t x, float *sv, float *cv)
{
    const int32_t xs = (int32_t)x;
    const float th = (float)(xs >> 8) * 0x1p-23f;
    const float d = ((float)(xs & 255) + 0.5f) * (0x1p-31f * 3.14159265358979f);
    float s, c;
    sincospif(th, &s, &c);
    *sv = __fmaf_rn(c, d, s);
    *cv = __fmaf_rn(-s, d, c);
}
// Cell of one coordinate on a uniform axis (-1 outside the box); *near when
// the coordinate lies within m cell widths of a face.
__device__ __forceinline__ int node_axis_fast(float v, float vmax, float idv, int n, float m, bool *near)
{
    const float t = __fmul_rn(__fadd_rn(v, vmax), idv);
    const float fl = floorf(t), fr = t - fl;
    if (fr < m || fr > 1.f - m) *near = true;
    if (!(t >= 0.f) || fl >= (float)n) return -1;
    return (int)fl;
}

__device__ __forceinline__ SampleOut draw_sample_fast(const Geo &g, int64_t step, uint32_t cellword,
                                                      uint32_t l, bool *redo)
{
    const uint2 key = make_uint2(g.seed, g.instance);
    const uint4 a = philox4x32_10(make_uint4(l, (uint32_t)step, cellword, 0u), key);
    const uint4 b = philox4x32_10(make_uint4(l, (uint32_t)step, cellword, 1u), key);
    const float r0 = sqrtf(neglog_u01f(a.x)), r1 = sqrtf(neglog_u01f(a.z)), r2 = sqrtf(neglog_u01f(b.x));
    float s0, c0, s1, c1, s2, c2, sp, cp;
    sincos_2pi_u01f(a.y, &s0, &c0);
    sincos_2pi_u01f(a.w, &s1, &c1);
    sincos_2pi_u01f(b.y, &s2, &c2);
    sincos_2pi_u01f(b.w, &sp, &cp);
    const float v[3] = {r0 * c0, r0 * s0, r1 * c1};
    const float v1[3] = {r1 * s1, r2 * c2, r2 * s2};
    // k_z = 1 - 2u = (y + 1/2) 2^-31 with y = 2^31 - 1 - x (exact in int32);
    // sin(theta) = sqrt(1 - k_z^2) = 2 sqrt(u (1 - u)).
    const int32_t ys = (int32_t)(0x7FFFFFFFu - b.z);
    const float kz = __fmaf_rn((float)(ys & 255) + 0.5f, 0x1p-31f, (float)(ys >> 8) * 0x1p-23f);
    const float st = 2.f * sqrtf(u01f(b.z) * u01f(~b.z));
    const float k[3] = {st * cp, st * sp, kz};
    const float s = (v1[0] - v[0]) * k[0] + (v1[1] - v[1]) * k[1] + (v1[2] - v[2]) * k[2];
    const float vmax = g.vmaxf, idv = g.idvf, mt = 2.4e-7f * (float)g.nv;
    const float ma = kFastMarginA * idv + mt, mb = kFastMarginB * idv + mt;
    const int n = g.nv;
    bool near = false;
    auto node = [&](float x, float y, float z, float m) {
        const int i = node_axis_fast(x, vmax, idv, n, m, &near),
                  j = node_axis_fast(y, vmax, idv, n, m, &near),
                  q = node_axis_fast(z, vmax, idv, n, m, &near);
        return (i < 0 || j < 0 || q < 0) ? -1 : (i * n + j) * n + q;
    };
    SampleOut o;
    o.idx[0] = node(v[0], v[1], v[2], ma);
    o.idx[1] = node(v1[0], v1[1], v1[2], ma);
    o.idx[2] = node(v[0] + s * k[0], v[1] + s * k[1], v[2] + s * k[2], mb);
    o.idx[3] = node(v1[0] - s * k[0], v1[1] - s * k[1], v1[2] - s * k[2], mb);
    *redo = near;
    o.near = 0;
    o.outside = (o.idx[0] < 0) | (o.idx[1] < 0) | (o.idx[2] < 0) | (o.idx[3] < 0);
    o.W = (double)(g.cwf * fabsf(s));
    return o;
}

// The sampler the per-cell kernels use for states of type R: FP32 with an
// FP64 redraw near a face (uniform grids, FP32 states), else FP64.
template <typename R>
__device__ __forceinline__ SampleOut draw_sample_cell(const Geo &g, int64_t step, uint32_t cell,
                                                      uint32_t l)
{
    if (sizeof(R) == 4 && !g.axe) {
        bool redo;
        const SampleOut o = draw_sample_fast(g, step, cell, l, &redo);
        if (!redo) return o;
    }
    return draw_sample(g, step, cell, l);
}

// The sample set of one cell as the per-cell kernels draw it, for
// inspection: idx[l] in logical node order, W[l].
template <typename R>
__global__ void k_plan_cell(Geo g, int64_t step, uint32_t cell, int4 *__restrict__ idx, double *__restrict__ W)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= g.nt) return;
    const SampleOut o = draw_sample_cell<R>(g, step, cell, (uint32_t)l);
    idx[l] = make_int4(o.idx[0], o.idx[1], o.idx[2], o.idx[3]);
    W[l] = o.W;
}

// Node indices of a sample (v, v1, v*, v1*).  Grids with fewer than 65535
// nodes use 16-bit indices (0xFFFF = outside the box) to halve the bytes every
// CTA streams from L2 per cell; larger grids use 32-bit indices (-1 outside).
template <typename I> struct Idx4;
template <> struct Idx4<int> {
    using type = int4;
    static __device__ __forceinline__ type make(const int *q) { return make_int4(q[0], q[1], q[2], q[3]); }
};
template <> struct Idx4<uint16_t> {
    using type = ushort4;
    static __device__ __forceinline__ type make(const int *q)
    {
        return make_ushort4((unsigned short)q[0], (unsigned short)q[1], (unsigned short)q[2],
                            (unsigned short)q[3]);
    }
};
__device__ __forceinline__ int idx_of(int v) { return v; }
__device__ __forceinline__ int idx_of(unsigned short v) { return v == 0xFFFFu ? -1 : (int)v; }

// What the gather phase of a cell needs per sample: the nodes of v and v1 and
// the weight W (8 bytes for FP32 state with 16-bit indices).
template <typename R, typename I> struct PlanA;
template <> struct __align__(8) PlanA<float, uint16_t> {
    uint32_t ab;
    float W;
    __device__ __forceinline__ int a() const { return idx_of((unsigned short)(ab & 0xFFFFu)); }
    __device__ __forceinline__ int b() const { return idx_of((unsigned short)(ab >> 16)); }
};
template <> struct __align__(16) PlanA<double, uint16_t> {
    uint32_t ab, pad;
    double W;
    __device__ __forceinline__ int a() const { return idx_of((unsigned short)(ab & 0xFFFFu)); }
    __device__ __forceinline__ int b() const { return idx_of((unsigned short)(ab >> 16)); }
};
template <> struct __align__(16) PlanA<float, int> {
    int ia, ib;
    float W;
    int pad;
    __device__ __forceinline__ int a() const { return ia; }
    __device__ __forceinline__ int b() const { return ib; }
};
template <> struct __align__(16) PlanA<double, int> {
    int ia, ib;
    double W;
    __device__ __forceinline__ int a() const { return ia; }
    __device__ __forceinline__ int b() const { return ib; }
};

template <typename R, typename I>
__device__ __forceinline__ PlanA<R, I> make_plan_a(int a, int b, double W)
{
    PlanA<R, I> o;
    if constexpr (sizeof(I) == 2) {
        o.ab = (uint32_t)(a & 0xFFFF) | ((uint32_t)(b & 0xFFFF) << 16);
    } else {
        o.ia = a;
        o.ib = b;
    }
    o.W = (R)W;
    return o;
}

// One thread per sample; the set is shared by every cell of the step.
// The step number is read from device memory so that launches captured in a
// CUDA graph stay correct when the graph is replayed (k_advance moves it on).
template <typename R, typename I>
__global__ void k_plan(Geo g, const int64_t *__restrict__ stepp,
                       typename Idx4<I>::type *__restrict__ idx, PlanA<R, I> *__restrict__ pa,
                       double *__restrict__ Wd, unsigned long long *__restrict__ stats)
{
    const int64_t step = *stepp;
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    SampleOut o = {};
    bool act = l < g.nt;
    if (act) {
        o = draw_sample(g, step, 0xFFFFFFFFu, (uint32_t)l);
        if (g.swz) {
            // Shared-memory order of the FP32 vector kernel: within each
            // (jx, jy) row the quads of four jz nodes are rotated by jx.
            const int N = g.nv, nq = N / 4;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j = o.idx[k];
                if (j < 0) continue;
                const int jx = j / (N * N), jz = j % N, row = j - jz;
                int r = jz / 4 + jx % nq;
                if (r >= nq) r -= nq;
                o.idx[k] = row + 4 * r + (jz & 3);
            }
        }
        idx[l] = Idx4<I>::make(o.idx);
        if (pa) pa[l] = make_plan_a<R, I>(o.idx[0], o.idx[1], o.W);
        if (Wd) Wd[l] = o.W;
    }
    if (stats) {
        unsigned mo = __ballot_sync(0xFFFFFFFFu, act && o.outside);
        unsigned mn = __ballot_sync(0xFFFFFFFFu, act && o.near);
        if ((threadIdx.x & 31) == 0) {
            if (mo) atomicAdd(stats + 1, (unsigned long long)__popc(mo));
            if (mn) atomicAdd(stats + 2, (unsigned long long)__popc(mn));
        }
    }
}

// ---------------------------------------------------------------------
// Block reductions (per-thread partials -> per-warp -> double totals)
// ---------------------------------------------------------------------
// Error-free transformations in FP32: a + b = s + e exactly (Knuth's
// TwoSum) and a b = p + e exactly (the product's rounding error from one
// fused multiply-add).  Explicit rounding intrinsics keep the compiler from
// contracting or reassociating them.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

template <int K, typename A>
__device__ __forceinline__ void block_reduce(A (&v)[K], double *red /* kMaxWarps*kRedSlots */,
                                             double *tot /* K */)
{
    // Per-warp shuffle sums, then one thread per value adds the warp partials
    // in the accumulator precision (no FP64 on the FP32 path: GB300's FP64
    // rate is a small fraction of FP32) and stores the total as double.
    A *ra = reinterpret_cast<A *>(red);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        A x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
        if (lane == 0) ra[warp * kRedSlots + k] = x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        A s = A(0);
        if constexpr (sizeof(A) == 4) {
            // FP32: compensated sum of the warp partials.
            float c = 0.f;
            for (int w = 0; w < nwarps; ++w) {
                float e;
                two_sum(s, ra[w * kRedSlots + threadIdx.x], s, e);
                c = __fadd_rn(c, e);
            }
            s = __fadd_rn(s, c);
        } else {
            for (int w = 0; w < nwarps; ++w) s += ra[w * kRedSlots + threadIdx.x];
        }
        tot[threadIdx.x] = (double)s;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------
// Diffuse walls (Eq. bcMax): one CTA per boundary face.
// Faces: [0,ny) left, [ny,2ny) right, [2ny,2ny+nx) bottom, then the lid.
// ---------------------------------------------------------------------
__device__ __forceinline__ double lid_speed(const Geo &g, int ix, int64_t step)
{
    double base = g.lid_profile ? g.lid_profile[ix] : g.lid_u0;
    if (g.lid_period > 0.0) {
        double t = (double)step * g.dt;
        base += g.lid_amp * sin(6.283185307179586 * t / g.lid_period);
    }
    return base;
}

struct Face {
    int cell, nax;   // boundary cell, normal axis (0 = x, 1 = y)
    double nsign;    // inward normal = nsign * e_nax
    double U;        // wall speed along the tangential axis (x for the lid)
};

__device__ __forceinline__ Face face_of(const Geo &g, int f, int64_t step)
{
    Face F;
    F.U = 0.0;
    if (f < g.ny) {
        F.cell = f * g.nx; F.nax = 0; F.nsign = 1.0;
    } else if (f < 2 * g.ny) {
        F.cell = (f - g.ny) * g.nx + g.nx - 1; F.nax = 0; F.nsign = -1.0;
    } else if (f < 2 * g.ny + g.nx) {
        F.cell = f - 2 * g.ny; F.nax = 1; F.nsign = 1.0;
    } else {
        int ix = f - 2 * g.ny - g.nx;
        F.cell = (g.ny - 1) * g.nx + ix; F.nax = 1; F.nsign = -1.0;
        F.U = lid_speed(g, ix, step);
    }
    return F;
}

// The wall kernels: one CTA of kWallThreads threads per face (with about 60
// registers a thread, eight CTAs fit an SM, so a 256x256 cavity's 1024
// faces run in one wave), each thread with kWallLoads loads in flight.
constexpr int kWallThreads = 128;
constexpr int kWallLoads = 16;

// ghost[f*nv + jt]: emitted h for inflow nodes of face f, indexed by the
// tangential velocity index (jy for side walls, jx for bottom and lid).
// shear[ix]: x-momentum flux through lid face ix (lid faces only).
// One boundary face f: outgoing flux, wall density and ghost values, and on
// the lid the shear.  Called by every thread of a CTA; sA, sv (kMaxN each),
// red, tot (>= 2) and snw are shared scratch.
// mu (nullable): per-cell deferred corrections (8 floats per cell) of a state
// stored as h_c, whose value is h_c + (1 + eps h_c)(mu_c . psi_j).
template <typename R>
__device__ __forceinline__ void walls_face(const Geo &g, int64_t step, const R *__restrict__ h,
                                           R *__restrict__ ghost, double *__restrict__ nw_out,
                                           double *__restrict__ shear, int f, R *sA, R *sv,
                                           double *red, double *tot, double *snw,
                                           const float *__restrict__ mu = nullptr)
{
    const Face F = face_of(g, f, step);
    const int N = g.nv, N2 = N * N;
    const bool lid = f >= 2 * g.ny + g.nx;
    const R ns = (R)F.nsign;
    R m5[5] = {R(0), R(0), R(0), R(0), R(0)};
    if (mu)
        for (int k = 0; k < 5; ++k) m5[k] = (R)mu[(int64_t)F.cell * 8 + k];
    // Per normal-axis node: the outgoing weight -v_n A(v_n) (0 for incoming
    // nodes), the normal part of the pending correction, m_n v_n + m_4 v_n^2,
    // and on the lid A(v_n) v_n for the shear.
    __shared__ R s_cw[kMaxN], s_kn[kMaxN], s_cl[kMaxN];
    const R mn = F.nax == 0 ? m5[1] : m5[2], mt = F.nax == 0 ? m5[2] : m5[1];
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const R A = (R)g.axA[i], v = (R)g.axv[i];
        sA[i] = A;
        sv[i] = v;
        s_cw[i] = v * ns < R(0) ? -(v * ns) * A : R(0);
        s_kn[i] = mn * v + m5[4] * v * v;
        s_cl[i] = A * v;
    }
    __syncthreads();
    const R *hc = h + (int64_t)F.cell * g.nvt;
    // Outgoing flux sum_{v_n<0} |v_n| w_j h_j and, on the lid, the cell part
    // of the shear, sum_{v_y>0} w_j v_x v_y h_j (per-thread sums in the state
    // precision, combined in double).  Threads take the pairs of the other
    // two axes (z fastest, so their loads are adjacent) and loop over the
    // outgoing half of the normal axis only (v_n < 0: nodes below N/2 for an
    // inward normal along +e_n, above for -e_n, the axes being symmetric).
    // With w_j = A_n A_a A_z the sums over the normal axis are taken first.
    R acc[2] = {R(0), R(0)};
    const R eps = (R)g.eps;
    const int lo = F.nsign > 0.0 ? 0 : N - N / 2, hi = F.nsign > 0.0 ? N / 2 : N;
    for (int q = threadIdx.x; q < N2; q += blockDim.x) {
        const int qa = q / N, jz = q - qa * N;   // (jy, jz) on side walls, (jx, jz) on bottom and lid
        const R vz = sv[jz], va = sv[qa], Aq = sA[qa] * sA[jz];
        const int64_t base = F.nax == 0 ? (int64_t)q : (int64_t)qa * N2 + jz;
        const int64_t stride = F.nax == 0 ? N2 : N;
        // The tangential part of the pending correction of these nodes.
        const R kq = m5[0] + mt * va + m5[3] * vz + m5[4] * (va * va + vz * vz);
        R s0 = R(0), s1 = R(0);
        // kWallLoads planes at a time (the whole outgoing half up to 32
        // nodes per axis): their loads are in flight together.
        for (int jn0 = lo; jn0 < hi; jn0 += kWallLoads) {
            R hs[kWallLoads];
#pragma unroll
            for (int k = 0; k < kWallLoads; ++k) {
                const int jn = jn0 + k;
                hs[k] = jn < hi ? hc[base + jn * stride] : R(0);
            }
#pragma unroll
            for (int k = 0; k < kWallLoads; ++k) {
                const int jn = jn0 + k;
                if (jn >= hi) break;
                R hv = hs[k];
                if (mu) {
                    const R kap = kq + s_kn[jn];
                    hv = hv + (R(1) + eps * hv) * kap;
                }
                s0 += s_cw[jn] * hv;
                if (lid) s1 += s_cl[jn] * hv;
            }
        }
        acc[0] += Aq * s0;
        if (lid) acc[1] += Aq * va * s1;
    }
    block_reduce<2, R>(acc, red, tot);
    if (F.U == 0.0 && !lid) {
        // A wall at rest: Phi_w = Phi0, so D_in = h_n z_sum^2 = c_out (the
        // tangential sum of A is z_sum), n_w = 1 + eps F / c_out, and every
        // emitted value is (n_w - 1) / eps = F / c_out.
        const double gh = tot[0] / g.cout;
        if (threadIdx.x == 0 && nw_out) nw_out[f] = 1.0 + g.eps * gh;
        for (int jt = threadIdx.x; jt < N; jt += blockDim.x) ghost[f * N + jt] = (R)gh;
        __syncthreads();
        return;
    }
    if (threadIdx.x < 32) {
        // D_in = sum_{v_n>0} v_n dV Phi_w(v_j), separable in the three axes
        // (the tangential factor summed by one warp).
        double tsum = 0.0;
        for (int jt = threadIdx.x; jt < N; jt += 32) {
            const double d = g.axv[jt] - F.U;
            tsum += (g.axd ? g.axd[jt] : g.dv) * 0.5641895835477563 * exp(-d * d);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) tsum += __shfl_xor_sync(0xFFFFFFFFu, tsum, o);
        if (threadIdx.x == 0) {
            const double din = g.hn * tsum * g.zsum;
            const double nw = (g.cout + g.eps * tot[0]) / din;
            *snw = nw;
            if (nw_out) nw_out[f] = nw;
        }
    }
    __syncthreads();
    // ln n_w only in the threads that emit ghosts or sum the lid shear.
    const double nw = *snw, U = F.U;
    const double lnw = (int)threadIdx.x < N || threadIdx.x < 32 ? log(nw) : 0.0;
    for (int jt = threadIdx.x; jt < N; jt += blockDim.x) {
        double vt = g.axv[jt];
        // n_w Phi_w / Phi0 - 1 = expm1(ln n_w + 2 v_t U - U^2)
        double gh = expm1(lnw + 2.0 * vt * U - U * U) / g.eps;
        ghost[f * N + jt] = (R)gh;
    }
    if (lid && shear && threadIdx.x < 32) {
        // Emitted part: sum over v_y < 0 of w v_x v_y h_w(jx), separable
        // (each factor summed by one warp).
        double sx = 0.0, sy = 0.0;
        for (int jx = threadIdx.x; jx < N; jx += 32) {
            const double gh = expm1(lnw + 2.0 * g.axv[jx] * U - U * U) / g.eps;
            sx += g.axA[jx] * g.axv[jx] * gh;
            if (g.axv[jx] < 0.0) sy += g.axA[jx] * g.axv[jx];
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            sx += __shfl_xor_sync(0xFFFFFFFFu, sx, o);
            sy += __shfl_xor_sync(0xFFFFFFFFu, sy, o);
        }
        if (threadIdx.x == 0) shear[f - 2 * g.ny - g.nx] = 2.0 * (tot[1] + sx * sy * g.zsum);
    }
    __syncthreads();
}

// ghost[f*nv + jt]: emitted h for inflow nodes of face f, indexed by the
// tangential velocity index (jy for side walls, jx for bottom and lid).
// shear[ix]: x-momentum flux through lid face ix (lid faces only).
template <typename R>
__global__ void k_walls(Geo g, const int64_t *__restrict__ stepp, const R *__restrict__ h,
                        R *__restrict__ ghost, double *__restrict__ nw_out,
                        double *__restrict__ shear, const float *__restrict__ mu = nullptr)
{
    __shared__ double red[kMaxWarps * kRedSlots];
    __shared__ double tot[4];
    __shared__ double s_nw;
    __shared__ R sA[kMaxN], sv[kMaxN];
    walls_face<R>(g, *stepp, h, ghost, nw_out, shear, blockIdx.x, sA, sv, red, tot, &s_nw, mu);
}

// Advances the device step counter by one (the last launch of a step).
static __global__ void k_advance(int64_t *__restrict__ stepp) { *stepp += 1; }

// out[0..nx) = the face shears, out[nx] = D, their mean over the lid
// weighted by the face widths (wlid[i] = dx_i / L; nullptr: uniform faces).
static __global__ void k_shear_mean(const double *__restrict__ shear, int nx,
                                    const double *__restrict__ wlid, double *__restrict__ out)
{
    __shared__ double red[kMaxWarps * kRedSlots];
    __shared__ double tot[1];
    double a[1] = {0.0};
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        a[0] += wlid ? shear[i] * wlid[i] * nx : shear[i];
        out[i] = shear[i];
    }
    block_reduce<1, double>(a, red, tot);
    if (threadIdx.x == 0) out[nx] = tot[0] / nx;
}

// ---------------------------------------------------------------------
// Free streaming (Eq. streaming2D), first-order upwind, conservative.
// ---------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R upwind_node(const Geo &g, const R *__restrict__ h,
                                         const R *__restrict__ ghost, int c, int ix, int iy,
                                         int64_t j, int jx, int jy, R cux, R cuy)
{
    const int64_t nvt = g.nvt;
    R h0 = h[(int64_t)c * nvt + j];
    R hx = h0, hy = h0;
    if (cux > R(0)) {
        hx = ix > 0 ? h[(int64_t)(c - 1) * nvt + j] : ghost[iy * g.nv + jy];
    } else if (cux < R(0)) {
        hx = ix < g.nx - 1 ? h[(int64_t)(c + 1) * nvt + j] : ghost[(g.ny + iy) * g.nv + jy];
    }
    if (cuy > R(0)) {
        hy = iy > 0 ? h[(int64_t)(c - g.nx) * nvt + j] : ghost[(2 * g.ny + ix) * g.nv + jx];
    } else if (cuy < R(0)) {
        hy = iy < g.ny - 1 ? h[(int64_t)(c + g.nx) * nvt + j]
                           : ghost[(2 * g.ny + g.nx + ix) * g.nv + jx];
    }
    R ax = fabs(cux), ay = fabs(cuy);
    return h0 - ax * (h0 - hx) - ay * (h0 - hy);
}

// One CTA per cell, threads over the slab.
template <typename R>
__global__ void k_stream(Geo g, const R *__restrict__ h, const R *__restrict__ ghost,
                         R *__restrict__ ht)
{
    __shared__ R cu[kMaxN];
    const int N = g.nv, N2 = N * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) cu[i] = (R)(g.axv[i] * g.dt / g.dx);
    __syncthreads();
    const R ry = (R)(g.dx / g.dy);
    for (int c = blockIdx.x; c < g.nr; c += gridDim.x) {
        const int ix = c % g.nx, iy = c / g.nx;
        // Courant numbers of this cell: its own widths on stretched grids.
        const R fx = g.sx ? (R)g.sx[ix] : R(1), fy = g.sy ? (R)g.sy[iy] : ry;
        for (int j = threadIdx.x; j < g.nvt; j += blockDim.x) {
            int jx = j / N2, jy = (j / N) % N;
            ht[(int64_t)c * g.nvt + j] =
                upwind_node<R>(g, h, ghost, c, ix, iy, j, jx, jy, cu[jx] * fx, cu[jy] * fy);
        }
    }
}

// ---------------------------------------------------------------------
// Per-cell relaxation (Eqs. monteCarloInt, collision_step, rinorm_a,
// correzione) and moments, optionally with streaming fused into the load.
// ---------------------------------------------------------------------
template <typename R>
struct AxisTab {       // per-axis tables in shared memory, N entries each
    R *A, *IA, *v, *v2, *v3, *v4, *Av, *Av2, *cx, *cu;
};

template <typename R>
__device__ __noinline__ void chol_or_ge(R G[5][5], R b[5], R x[5], int *fallback, bool force_ge = false)
{
    R L[5][5];
    bool ok = !force_ge;
    for (int i = 0; i < 5 && ok; ++i) {
        for (int j = 0; j <= i; ++j) {
            R s = G[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > R(0))) { ok = false; break; }
                L[i][i] = sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    }
    if (ok) {
        R y[5];
        for (int i = 0; i < 5; ++i) {
            R s = b[i];
            for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
            y[i] = s / L[i][i];
        }
        for (int i = 4; i >= 0; --i) {
            R s = y[i];
            for (int k = i + 1; k < 5; ++k) s -= L[k][i] * x[k];
            x[i] = s / L[i][i];
        }
        return;
    }
    ++*fallback;
    // Gaussian elimination with partial pivoting.
    R A[5][6];
    for (int i = 0; i < 5; ++i) {
        for (int j = 0; j < 5; ++j) A[i][j] = G[i][j];
        A[i][5] = b[i];
    }
    for (int k = 0; k < 5; ++k) {
        int p = k;
        for (int i = k + 1; i < 5; ++i)
            if (fabs(A[i][k]) > fabs(A[p][k])) p = i;
        if (A[p][k] == R(0)) {
            for (int i = 0; i < 5; ++i) x[i] = R(0);
            return;
        }
        for (int j = 0; j < 6; ++j) {
            R t = A[k][j]; A[k][j] = A[p][j]; A[p][j] = t;
        }
        for (int i = k + 1; i < 5; ++i) {
            R m = A[i][k] / A[k][k];
            for (int j = k; j < 6; ++j) A[i][j] -= m * A[k][j];
        }
    }
    for (int i = 4; i >= 0; --i) {
        R s = A[i][5];
        for (int j = i + 1; j < 5; ++j) s -= A[i][j] * x[j];
        x[i] = s / A[i][i];
    }
}

// Correction of Eqs. rinorm_a / correzione for one cell.  P holds the reduced
// sums: P[0..13] moments of the post-collision N_c over the monomials
// 1, vx, vy, vz, vx2, vy2, vz2, vxvy, vxvz, vyvz, vx v2, vy v2, vz v2, v4 and
// P[14..18] the moments D of the collision increment N_c - N over the
// invariants 1, vx, vy, vz, v2.  Solves G mu = -D (the correction restores the
// invariants of the pre-collision N) with G = sum_j w_j (1 + eps h_c,j) psi
// psi^T.
template <typename R>
__device__ __noinline__ void correction_solve(const Geo &g, const double *Pd, double *mu,
                                              int *fallback)
{
    // Solved in the state precision: G is close to the equilibrium Gram matrix
    // (condition number ~30), so FP32 keeps the correction to ~1e-6 of itself.
    R P[19];
    for (int k = 0; k < 19; ++k) P[k] = (R)Pd[k];
    const R e = (R)g.eps;
    R post[5] = {P[0], P[1], P[2], P[3], P[4] + P[5] + P[6]};
    R rhs[5];
    for (int a = 0; a < 5; ++a) rhs[a] = (R)(-Pd[14 + a]);
    const R m[5][5] = {
        {P[0], P[1], P[2], P[3], post[4]},
        {P[1], P[4], P[7], P[8], P[10]},
        {P[2], P[7], P[5], P[9], P[11]},
        {P[3], P[8], P[9], P[6], P[12]},
        {post[4], P[10], P[11], P[12], P[13]}};
    R M[5][5];
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b)
            M[a][b] = (sizeof(R) == 8 ? (R)g.G0[a * 5 + b] : (R)g.G0f[a * 5 + b]) + e * m[a][b];
    R x[5];
    chol_or_ge<R>(M, rhs, x, fallback, g.solve_fb != 0);
    for (int a = 0; a < 5; ++a) mu[a] = (double)x[a];
}

// Eqs. densita..sforzi in V0 units from the ten sums m = sum w h {1, v_x,
// v_y, v_z, v_x^2, v_y^2, v_z^2, v_x v_y, v_x v_z, v_y v_z}.
template <typename R>
__device__ __noinline__ void finalize_moments(const double *md, R e, double *o)
{
    R m[10];
    for (int k = 0; k < 10; ++k) m[k] = (R)md[k];
    R rho = m[0], n = R(1) + e * rho;
    R u[3] = {m[1] / n, m[2] / n, m[3] / n};
    o[0] = rho;
    o[1] = u[0];
    o[2] = u[1];
    o[3] = u[2];
    o[4] = ((R(2) / R(3)) * (m[4] + m[5] + m[6]) - rho) / n -
           (R(2) * e / R(3)) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k) o[5 + k] = R(2) * m[4 + k] - R(2) * e * n * u[pa[k]] * u[pb[k]];
}

// Dynamic shared memory layout of the per-cell kernels.
template <typename R>
struct CellSmem {
    R *slab;           // nvt
    R *gw;             // nt (or nullptr when the products live in global scratch)
    void *sidx;        // nt node-index records of the cell's own samples (per-cell sets)
    AxisTab<R> tab;    // 10 * N
    double *red;       // kMaxWarps * kRedSlots
    double *tot;       // kRedSlots
    double *mu;        // 8
};

template <typename R>
__device__ __forceinline__ CellSmem<R> carve(char *base, const Geo &g, bool gw_in_smem)
{
    CellSmem<R> s;
    size_t off = 0;
    s.red = (double *)(base + off); off += sizeof(double) * kMaxWarps * kRedSlots;
    s.tot = (double *)(base + off); off += sizeof(double) * kRedSlots;
    s.mu = (double *)(base + off); off += sizeof(double) * 8;
    R *t = (R *)(base + off);
    const int N = g.nv;
    s.tab.A = t; s.tab.IA = t + N; s.tab.v = t + 2 * N; s.tab.v2 = t + 3 * N;
    s.tab.v3 = t + 4 * N; s.tab.v4 = t + 5 * N; s.tab.Av = t + 6 * N; s.tab.Av2 = t + 7 * N;
    s.tab.cx = t + 8 * N; s.tab.cu = t + 9 * N;
    off += sizeof(R) * 10 * N;
    off = (off + 15) & ~(size_t)15;
    s.slab = (R *)(base + off); off += sizeof(R) * g.nvt;
    off = (off + 15) & ~(size_t)15;
    s.gw = gw_in_smem ? (R *)(base + off) : nullptr;
    if (gw_in_smem) off += sizeof(R) * g.nt;
    off = (off + 15) & ~(size_t)15;
    s.sidx = base + off;
    return s;
}

// idx_bytes: bytes per sample of the per-cell sample records (0 for the
// shared set, whose records stay in global memory).
template <typename R>
__host__ __device__ inline size_t cell_smem_bytes(int nv, int nvt, int nt, bool gw_in_smem,
                                                  size_t idx_bytes = 0)
{
    size_t off = sizeof(double) * (kMaxWarps * kRedSlots + kRedSlots + 8) + sizeof(R) * 10 * nv;
    off = (off + 15) & ~(size_t)15;
    off += sizeof(R) * nvt;
    off = (off + 15) & ~(size_t)15;
    if (gw_in_smem) off += sizeof(R) * nt;
    off = (off + 15) & ~(size_t)15;
    off += idx_bytes * nt;
    return off;
}

// FUSED: the slab is filled by streaming h^n (Eq. streaming2D) instead of
// loading h~ from global memory.  PC: every cell draws its own sample set
// (Philox counter word 2 = the cell index, step from *stepp) in the gather
// phase and keeps its node indices in shared memory; pidx and pa are unused.
template <typename R, bool FUSED, typename I, bool PC = false>
__global__ void __launch_bounds__(kMaxThreads, 1)
k_cell(Geo g, const R *__restrict__ hin, const R *__restrict__ ghost,
       const typename Idx4<I>::type *__restrict__ pidx, const PlanA<R, I> *__restrict__ pa,
       R *__restrict__ gw_global,
       R *__restrict__ hout, double *__restrict__ mom, unsigned long long *__restrict__ stats,
       int gw_in_smem, const int64_t *__restrict__ stepp = nullptr)
{
    extern __shared__ __align__(16) char smem_raw[];
    CellSmem<R> S = carve<R>(smem_raw, g, gw_in_smem != 0);
    using V4 = typename Idx4<I>::type;
    V4 *sidx = reinterpret_cast<V4 *>(S.sidx);
    const int64_t step = PC ? *stepp : 0;
    const int N = g.nv, N2 = N * N, nvt = g.nvt, T = blockDim.x, t = threadIdx.x;
    const R eps = (R)g.eps;
    R *gw = S.gw ? S.gw : gw_global + (int64_t)blockIdx.x * g.nt;

    for (int i = t; i < N; i += T) {
        double v = g.axv[i], A = g.axA[i];
        S.tab.A[i] = (R)A;
        S.tab.IA[i] = (R)(1.0 / A);
        S.tab.v[i] = (R)v;
        S.tab.v2[i] = (R)(v * v);
        S.tab.v3[i] = (R)(v * v * v);
        S.tab.v4[i] = (R)(v * v * v * v);
        S.tab.Av[i] = (R)(A * v);
        S.tab.Av2[i] = (R)(A * v * v);
        S.tab.cu[i] = (R)(v * g.dt / g.dx);
    }
    __syncthreads();
    const R ry = (R)(g.dx / g.dy);
    int fallback = 0;

    for (int kc = blockIdx.x; kc < g.nr; kc += gridDim.x) {
        const int c = cell_of(g, kc);
        const int ix = c % g.nx, iy = c / g.nx;
        // ---- fill the slab with h~ ----------------------------------------
        if (FUSED) {
            // Eq. streaming2D with the upwind sources hoisted per thread: the
            // sign of v_x changes once along jx (negative half reads the right
            // neighbour, positive half the left one), the sign of v_y is fixed
            // per thread; at a wall the source is the face's ghost value.
            const int64_t nvt64 = nvt;
            const R *own = hin + (int64_t)c * nvt64;
            // Courant factors of this cell (its own widths on stretched grids).
            const R fx = g.sx ? (R)g.sx[ix] : R(1), fy = g.sy ? (R)g.sy[iy] : ry;
            const int nneg = N / 2, npos = (N + 1) / 2;
            for (int p = t; p < N2; p += T) {
                const int jy = p / N;
                const R cuy = S.tab.cu[jy] * fy, ay = fabs(cuy);
                const R *ys = own;
                int ystr = N2, yoff = p;
                if (cuy > R(0)) {
                    if (iy > 0) ys = own - (int64_t)g.nx * nvt64;
                    else { ys = ghost + (2 * g.ny + ix) * N; ystr = 1; yoff = 0; }
                } else if (cuy < R(0)) {
                    if (iy < g.ny - 1) ys = own + (int64_t)g.nx * nvt64;
                    else { ys = ghost + (2 * g.ny + g.nx + ix) * N; ystr = 1; yoff = 0; }
                }
                // v_x < 0: right neighbour or right-wall ghost (constant in jx)
                const R *xs = ix < g.nx - 1 ? own + nvt64 + p : ghost + (g.ny + iy) * N + jy;
                int xstr = ix < g.nx - 1 ? N2 : 0;
#pragma unroll 4
                for (int jx = 0; jx < nneg; ++jx) {
                    const int j = jx * N2 + p;
                    R h0 = own[j], hx = xs[jx * xstr], hy = ys[jx * ystr + yoff];
                    R ax = fabs(S.tab.cu[jx]) * fx;
                    S.slab[j] = h0 - ax * (h0 - hx) - ay * (h0 - hy);
                }
                for (int jx = nneg; jx < npos; ++jx) {       // v_x = 0 (odd N)
                    const int j = jx * N2 + p;
                    R h0 = own[j], hy = ys[jx * ystr + yoff];
                    S.slab[j] = h0 - ay * (h0 - hy);
                }
                // v_x > 0: left neighbour or left-wall ghost
                xs = ix > 0 ? own - nvt64 + p : ghost + iy * N + jy;
                xstr = ix > 0 ? N2 : 0;
#pragma unroll 4
                for (int jx = npos; jx < N; ++jx) {
                    const int j = jx * N2 + p;
                    R h0 = own[j], hx = xs[jx * xstr], hy = ys[jx * ystr + yoff];
                    R ax = fabs(S.tab.cu[jx]) * fx;
                    S.slab[j] = h0 - ax * (h0 - hx) - ay * (h0 - hy);
                }
            }
        } else {
            const R *src = hin + (int64_t)c * nvt;
            for (int j = t; j < nvt; j += T) S.slab[j] = src[j];
        }
        if (PC && t == 0) reinterpret_cast<int *>(S.red)[0] = 0;     // redraw queue
        __syncthreads();

        // ---- phase A: g_l W_l from the pre-collision values (Jacobi) -------
        // Plan entries are loaded four at a time to keep L2 requests in flight.
        if constexpr (PC) {
            // The cell's own samples (Sec. 4.2 / Algorithm 2 with the cell in
            // the Philox counter), node selection equal to the FP64
            // computation's.  FP32 states on uniform grids draw in FP32; a
            // sample near a velocity-cell face is queued in the reduction
            // scratch (idle until the increment sums) and drawn again in
            // FP64 after the loop by all threads, so the warps stay together
            // (a full queue redraws in place).
            const bool fast = sizeof(R) == 4 && !g.axe;
            int *rq = reinterpret_cast<int *>(S.red);
            const int rcap = g.redraw_cap < 0 ? kMaxWarps * kRedSlots * 2 - 1
                                              : min(g.redraw_cap, kMaxWarps * kRedSlots * 2 - 1);
            auto put = [&](int l, const SampleOut &o) {
                sidx[l] = Idx4<I>::make(o.idx);
                const R ha = o.idx[0] >= 0 ? S.slab[o.idx[0]] : R(0);
                const R hb = o.idx[1] >= 0 ? S.slab[o.idx[1]] : R(0);
                gw[l] = (ha + hb + eps * ha * hb) * (R)o.W;
            };
            auto count = [&](bool act, const SampleOut &o) {
                if (stats) {
                    const unsigned mo = __ballot_sync(0xFFFFFFFFu, act && o.outside);
                    const unsigned mn = __ballot_sync(0xFFFFFFFFu, act && o.near);
                    if ((t & 31) == 0) {
                        if (mo) atomicAdd(stats + 1, (unsigned long long)__popc(mo));
                        if (mn) atomicAdd(stats + 2, (unsigned long long)__popc(mn));
                    }
                }
            };
            for (int l0 = 0; l0 < g.nt; l0 += T) {
                const int l = l0 + t;
                bool act = l < g.nt;
                SampleOut o = {};
                if (act) {
                    bool redo = true;
                    if (fast) o = draw_sample_fast(g, step, (uint32_t)c, (uint32_t)l, &redo);
                    if (redo) {
                        const int k = fast ? atomicAdd(rq, 1) : rcap;
                        if (k < rcap) {
                            rq[1 + k] = l;
                            act = false;
                        } else {
                            o = draw_sample(g, step, (uint32_t)c, (uint32_t)l);
                        }
                    }
                    if (act) put(l, o);
                }
                count(act, o);
            }
            if (fast) {
                __syncthreads();
                const int nq = min(rq[0], rcap);
                for (int i0 = 0; i0 < nq; i0 += T) {
                    const bool act = i0 + t < nq;
                    SampleOut o = {};
                    if (act) {
                        const int l = rq[1 + i0 + t];
                        o = draw_sample(g, step, (uint32_t)c, (uint32_t)l);
                        put(l, o);
                    }
                    count(act, o);
                }
            }
        } else {
            int l = t;
            for (; l + 3 * T < g.nt; l += 4 * T) {
                PlanA<R, I> q[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) q[u] = pa[l + u * T];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int a = q[u].a(), b = q[u].b();
                    R ha = a >= 0 ? S.slab[a] : R(0);
                    R hb = b >= 0 ? S.slab[b] : R(0);
                    gw[l + u * T] = (ha + hb + eps * ha * hb) * q[u].W;
                }
            }
            for (; l < g.nt; l += T) {
                const PlanA<R, I> q = pa[l];
                const int a = q.a(), b = q.b();
                R ha = a >= 0 ? S.slab[a] : R(0);
                R hb = b >= 0 ? S.slab[b] : R(0);
                gw[l] = (ha + hb + eps * ha * hb) * q.W;
            }
        }
        __syncthreads();
        const V4 *pix = PC ? sidx : pidx;

        // ---- N = w h~ in place, and the conserved moments of h~ ------------
        R pre[5] = {R(0), R(0), R(0), R(0), R(0)};
        for (int p = t; p < N2; p += T) {
            const int jy = p / N, jz = p % N;
            const R Ayz = S.tab.A[jy] * S.tab.A[jz];
            R s0 = R(0), s1 = R(0), s2 = R(0);
            for (int jx = 0; jx < N; ++jx) {
                const int j = jx * N2 + p;
                R n = S.slab[j] * S.tab.A[jx] * Ayz;
                S.slab[j] = n;
                s0 += n;
                s1 += n * S.tab.v[jx];
                s2 += n * S.tab.v2[jx];
            }
            const R vy = S.tab.v[jy], vz = S.tab.v[jz], q = vy * vy + vz * vz;
            pre[0] += s0;
            pre[1] += s1;
            pre[2] += vy * s0;
            pre[3] += vz * s0;
            pre[4] += s2 + q * s0;
        }
        __syncthreads();

        // ---- phase B: scatter the gains and losses (Eq. monteCarloInt) -----
        {
            auto scatter = [&](const V4 &q, R r) {
                if (r != R(0)) {
                    const int a = idx_of(q.x), b = idx_of(q.y), as = idx_of(q.z), bs = idx_of(q.w);
                    if (as >= 0) atomicAdd(S.slab + as, r);
                    if (bs >= 0) atomicAdd(S.slab + bs, r);
                    if (a >= 0) atomicAdd(S.slab + a, -r);
                    if (b >= 0) atomicAdd(S.slab + b, -r);
                }
            };
            int l = t;
            for (; l + 3 * T < g.nt; l += 4 * T) {
                V4 q[4];
                R r[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    q[u] = pix[l + u * T];
                    r[u] = gw[l + u * T];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) scatter(q[u], r[u]);
            }
            for (; l < g.nt; l += T) scatter(pix[l], gw[l]);
        }
        __syncthreads();

        // ---- moments of the post-collision N_c for the correction ----------
        R acc[19];
#pragma unroll
        for (int k = 0; k < 19; ++k) acc[k] = R(0);
        for (int p = t; p < N2; p += T) {
            const int jy = p / N, jz = p % N;
            R s0 = R(0), s1 = R(0), s2 = R(0), s3 = R(0), s4 = R(0);
            for (int jx = 0; jx < N; ++jx) {
                R n = S.slab[jx * N2 + p];
                s0 += n;
                s1 += n * S.tab.v[jx];
                s2 += n * S.tab.v2[jx];
                s3 += n * S.tab.v3[jx];
                s4 += n * S.tab.v4[jx];
            }
            const R vy = S.tab.v[jy], vz = S.tab.v[jz], q = vy * vy + vz * vz;
            acc[0] += s0;                  // 1
            acc[1] += s1;                  // vx
            acc[2] += vy * s0;             // vy
            acc[3] += vz * s0;             // vz
            acc[4] += s2;                  // vx^2
            acc[5] += vy * vy * s0;        // vy^2
            acc[6] += vz * vz * s0;        // vz^2
            acc[7] += vy * s1;             // vx vy
            acc[8] += vz * s1;             // vx vz
            acc[9] += vy * vz * s0;        // vy vz
            acc[10] += s3 + q * s1;        // vx v^2
            acc[11] += vy * (s2 + q * s0); // vy v^2
            acc[12] += vz * (s2 + q * s0); // vz v^2
            acc[13] += s4 + R(2) * q * s2 + q * q * s0;   // v^4
        }
        // The thread's share of the increment sums D: post minus pre over its
        // own nodes, so only thread-sized partial sums cancel.
        acc[14] = acc[0] - pre[0];
        acc[15] = acc[1] - pre[1];
        acc[16] = acc[2] - pre[2];
        acc[17] = acc[3] - pre[3];
        acc[18] = (acc[4] + acc[5] + acc[6]) - pre[4];
        block_reduce<19, R>(acc, S.red, S.tot);

        // ---- 5x5 solve: G mu = -D, G = sum w (1 + eps h_c) psi psi
        if (t == 0) correction_solve<R>(g, S.tot, S.mu, &fallback);
        __syncthreads();
        {
            const R mx = (R)S.mu[1], m4 = (R)S.mu[4];
            for (int i = t; i < N; i += T) {
                const R v = S.tab.v[i];
                S.tab.cx[i] = mx * v + m4 * S.tab.v2[i];
            }
        }
        __syncthreads();

        // ---- corrected write-back and output moments ----------------------
        R mo[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) mo[k] = R(0);
        R *dst = hout + (int64_t)c * nvt;
        for (int p = t; p < N2; p += T) {
            const int jy = p / N, jz = p % N;
            const R IAyz = S.tab.IA[jy] * S.tab.IA[jz];
            const R vy = S.tab.v[jy], vz = S.tab.v[jz];
            const R ct = (R)S.mu[0] + (R)S.mu[2] * vy + (R)S.mu[3] * vz +
                         (R)S.mu[4] * (vy * vy + vz * vz);
            R t0 = R(0), t1 = R(0), t2 = R(0);
            for (int jx = 0; jx < N; ++jx) {
                const int j = jx * N2 + p;
                R hc = S.slab[j] * S.tab.IA[jx] * IAyz;
                R corr = ct + S.tab.cx[jx];
                R hn = hc + (R(1) + eps * hc) * corr;
                dst[j] = hn;
                t0 += hn * S.tab.A[jx];
                t1 += hn * S.tab.Av[jx];
                t2 += hn * S.tab.Av2[jx];
            }
            const R Ayz = S.tab.A[jy] * S.tab.A[jz];
            mo[0] += Ayz * t0;
            mo[1] += Ayz * t1;
            mo[2] += Ayz * vy * t0;
            mo[3] += Ayz * vz * t0;
            mo[4] += Ayz * t2;
            mo[5] += Ayz * vy * vy * t0;
            mo[6] += Ayz * vz * vz * t0;
            mo[7] += Ayz * vy * t1;
            mo[8] += Ayz * vz * t1;
            mo[9] += Ayz * vy * vz * t0;
        }
        block_reduce<10, R>(mo, S.red, S.tot);
        if (t == 0 && mom) finalize_moments<R>(S.tot, (R)g.eps, mom + (int64_t)c * 11);
        // red/tot reuse is protected by the barriers inside block_reduce; the
        // next cell's first writes to the slab happen after this point only.
        __syncthreads();
    }
    if (fallback && stats) atomicAdd(stats + 3, (unsigned long long)fallback);
}

// Moments of an arbitrary state (Eqs. densita..sforzi), one CTA per cell.
template <typename R>
__global__ void k_moments(Geo g, const R *__restrict__ h, double *__restrict__ mom)
{
    __shared__ double red[kMaxWarps * kRedSlots];
    __shared__ double tot[kRedSlots];
    const int N = g.nv, N2 = N * N;
    for (int c = blockIdx.x; c < g.nr; c += gridDim.x) {
        double mo[10];
        for (int k = 0; k < 10; ++k) mo[k] = 0.0;
        const R *src = h + (int64_t)c * g.nvt;
        for (int j = threadIdx.x; j < g.nvt; j += blockDim.x) {
            int jx = j / N2, jy = (j / N) % N, jz = j % N;
            double vx = g.axv[jx], vy = g.axv[jy], vz = g.axv[jz];
            double wh = g.axA[jx] * g.axA[jy] * g.axA[jz] * (double)src[j];
            mo[0] += wh;
            mo[1] += wh * vx;
            mo[2] += wh * vy;
            mo[3] += wh * vz;
            mo[4] += wh * vx * vx;
            mo[5] += wh * vy * vy;
            mo[6] += wh * vz * vz;
            mo[7] += wh * vx * vy;
            mo[8] += wh * vx * vz;
            mo[9] += wh * vy * vz;
        }
        block_reduce<10, double>(mo, red, tot);
        if (threadIdx.x == 0) {
            const double *m = tot, e = g.eps;
            double rho = m[0], n = 1.0 + e * rho;
            double u[3] = {m[1] / n, m[2] / n, m[3] / n};
            double *o = mom + (int64_t)c * 11;
            o[0] = rho;
            o[1] = u[0];
            o[2] = u[1];
            o[3] = u[2];
            o[4] = ((2.0 / 3.0) * (m[4] + m[5] + m[6]) - rho) / n -
                   (2.0 * e / 3.0) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
            const double m2[6] = {m[4], m[5], m[6], m[7], m[8], m[9]};
            for (int k = 0; k < 6; ++k) o[5 + k] = 2.0 * m2[k] - 2.0 * e * n * u[pa[k]] * u[pb[k]];
        }
        __syncthreads();
    }
}

// Count of non-finite values in an array of doubles (flag only).
static __global__ void k_nonfinite(const double *__restrict__ x, int64_t n, int *__restrict__ flag)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) *flag = 1;
}

}  // namespace bzk
