// bz_adjoint.cuh -- adjoint of one time step with the sample stream fixed.
//
// With the samples of step n fixed, h^{n+1} = C(T(h^n; U)) is a smooth map:
// the free streaming T (Eq. streaming2D) is linear in h^n except for the wall
// ghosts (Eq. bcMax), which are affine in the outgoing flux of their face and
// nonlinear in the lid speed U; the Monte Carlo update (Eqs. monteCarloInt,
// collision_step) is bilinear in h~; the correction (Eqs. rinorm_a,
// correzione) is differentiated through its 5x5 solve.  Given
// lam = dJ/dh^{n+1} the three kernels below produce dJ/dh^n and add dJ/dU_i
// for J containing wD * D_n, D_n the mean lid shear of h^n (Sec. 5.2):
//   k_adj_cell    recomputes h~, h_c and mu of each cell in shared memory and
//                 applies the transposed correction and Monte Carlo update
//   k_adj_walls   per face, the ghost sensitivities -> outgoing-flux and lid
//                 speed terms
//   k_adj_stream  the transposed upwind stencil (a downwind gather) plus the
//                 outgoing-flux and lid-shear terms.
#pragma once

#include "bz_kernels.cuh"

namespace bzk {

template <typename R>
struct AdjSmem {
    R *A;            // h~ of the cell (kept for the bilinear term)
    R *B;            // N = w h~ -> N_c -> h_c -> q = lam_c / w
    R *C;            // dJ/dh~ accumulator
    R *gw;           // nt: g_l W_l
    AxisTab<R> tab;  // 10 N
    R *cxi;          // N: xi_x v + xi_4 v^2
    double *red, *tot, *mu, *xi, *P;
};

template <typename R>
__host__ __device__ inline size_t adj_smem_bytes(int nv, int nvt, int nt)
{
    size_t off = sizeof(double) * (kMaxWarps * kRedSlots + kRedSlots + 8 + 8 + 24);
    off += sizeof(R) * 11 * nv;
    off = (off + 15) & ~(size_t)15;
    off += 3 * sizeof(R) * nvt;
    off = (off + 15) & ~(size_t)15;
    off += sizeof(R) * nt;
    return off;
}

template <typename R>
__device__ __forceinline__ AdjSmem<R> carve_adj(char *base, const Geo &g)
{
    AdjSmem<R> s;
    size_t off = 0;
    s.red = (double *)(base + off); off += sizeof(double) * kMaxWarps * kRedSlots;
    s.tot = (double *)(base + off); off += sizeof(double) * kRedSlots;
    s.mu = (double *)(base + off); off += sizeof(double) * 8;
    s.xi = (double *)(base + off); off += sizeof(double) * 8;
    s.P = (double *)(base + off); off += sizeof(double) * 24;
    R *t = (R *)(base + off);
    const int N = g.nv;
    s.tab.A = t; s.tab.IA = t + N; s.tab.v = t + 2 * N; s.tab.v2 = t + 3 * N;
    s.tab.v3 = t + 4 * N; s.tab.v4 = t + 5 * N; s.tab.Av = t + 6 * N; s.tab.Av2 = t + 7 * N;
    s.tab.cx = t + 8 * N; s.tab.cu = t + 9 * N; s.cxi = t + 10 * N;
    off += sizeof(R) * 11 * N;
    off = (off + 15) & ~(size_t)15;
    s.A = (R *)(base + off); off += sizeof(R) * g.nvt;
    s.B = (R *)(base + off); off += sizeof(R) * g.nvt;
    s.C = (R *)(base + off); off += sizeof(R) * g.nvt;
    off = (off + 15) & ~(size_t)15;
    s.gw = (R *)(base + off);
    return s;
}

// G of the correction from the reduced sums P[0..13] (see correction_solve).
template <typename R>
__device__ __forceinline__ void gram_of(const Geo &g, const double *P, R G[5][5])
{
    const double e = g.eps, p4 = P[4] + P[5] + P[6];
    const double m[5][5] = {
        {P[0], P[1], P[2], P[3], p4},
        {P[1], P[4], P[7], P[8], P[10]},
        {P[2], P[7], P[5], P[9], P[11]},
        {P[3], P[8], P[9], P[6], P[12]},
        {p4, P[10], P[11], P[12], P[13]}};
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b)
            G[a][b] = (sizeof(R) == 8 ? (R)g.G0[a * 5 + b] : (R)g.G0f[a * 5 + b]) +
                      (R)e * (R)m[a][b];
}

// Sets the step counter read by the forward kernels of the adjoint.
static __global__ void k_set_step(int64_t *__restrict__ stepp, int64_t step) { *stepp = step; }

template <typename R>
__global__ void __launch_bounds__(kMaxThreads, 1)
k_adj_cell(Geo g, const R *__restrict__ hin, const R *__restrict__ ghost,
           const int4 *__restrict__ pidx, const PlanA<R, int> *__restrict__ pa,
           const R *__restrict__ lam_in, R *__restrict__ lt, unsigned long long *__restrict__ stats)
{
    extern __shared__ __align__(16) char smem_raw[];
    AdjSmem<R> S = carve_adj<R>(smem_raw, g);
    const int N = g.nv, N2 = N * N, nvt = g.nvt, T = blockDim.x, t = threadIdx.x;
    const R eps = (R)g.eps;
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
        // ---- forward: h~ ------------------------------------------------------
        for (int p = t; p < N2; p += T) {
            const int jy = p / N;
            const R cuy = S.tab.cu[jy] * ry;
            for (int jx = 0; jx < N; ++jx) {
                const int j = jx * N2 + p;
                S.A[j] = upwind_node<R>(g, hin, ghost, c, ix, iy, j, jx, jy, S.tab.cu[jx], cuy);
            }
        }
        __syncthreads();
        // ---- forward: g_l W_l ---------------------------------------------------
        for (int l = t; l < g.nt; l += T) {
            const int4 q = pidx[l];
            const R ha = q.x >= 0 ? S.A[q.x] : R(0);
            const R hb = q.y >= 0 ? S.A[q.y] : R(0);
            S.gw[l] = (ha + hb + eps * ha * hb) * pa[l].W;
        }
        __syncthreads();
        // ---- forward: N = w h~ and the invariants of h~ ------------------------
        R pre[5] = {R(0), R(0), R(0), R(0), R(0)};
        for (int p = t; p < N2; p += T) {
            const int jy = p / N, jz = p % N;
            const R Ayz = S.tab.A[jy] * S.tab.A[jz];
            R s0 = R(0), s1 = R(0), s2 = R(0);
            for (int jx = 0; jx < N; ++jx) {
                const int j = jx * N2 + p;
                const R n = S.A[j] * S.tab.A[jx] * Ayz;
                S.B[j] = n;
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
        // ---- forward: Monte Carlo gains and losses -----------------------------
        for (int l = t; l < g.nt; l += T) {
            const R r = S.gw[l];
            if (r != R(0)) {
                const int4 q = pidx[l];
                if (q.z >= 0) atomicAdd(S.B + q.z, r);
                if (q.w >= 0) atomicAdd(S.B + q.w, r);
                if (q.x >= 0) atomicAdd(S.B + q.x, -r);
                if (q.y >= 0) atomicAdd(S.B + q.y, -r);
            }
        }
        __syncthreads();
        // ---- forward: correction sums, G and mu --------------------------------
        R acc[19];
#pragma unroll
        for (int k = 0; k < 19; ++k) acc[k] = R(0);
        for (int p = t; p < N2; p += T) {
            const int jy = p / N, jz = p % N;
            R s0 = R(0), s1 = R(0), s2 = R(0), s3 = R(0), s4 = R(0);
            for (int jx = 0; jx < N; ++jx) {
                const R n = S.B[jx * N2 + p];
                s0 += n;
                s1 += n * S.tab.v[jx];
                s2 += n * S.tab.v2[jx];
                s3 += n * S.tab.v3[jx];
                s4 += n * S.tab.v4[jx];
            }
            const R vy = S.tab.v[jy], vz = S.tab.v[jz], q = vy * vy + vz * vz;
            acc[0] += s0;
            acc[1] += s1;
            acc[2] += vy * s0;
            acc[3] += vz * s0;
            acc[4] += s2;
            acc[5] += vy * vy * s0;
            acc[6] += vz * vz * s0;
            acc[7] += vy * s1;
            acc[8] += vz * s1;
            acc[9] += vy * vz * s0;
            acc[10] += s3 + q * s1;
            acc[11] += vy * (s2 + q * s0);
            acc[12] += vz * (s2 + q * s0);
            acc[13] += s4 + R(2) * q * s2 + q * q * s0;
        }
        // The thread's share of the increment sums D (post minus pre).
        acc[14] = acc[0] - pre[0];
        acc[15] = acc[1] - pre[1];
        acc[16] = acc[2] - pre[2];
        acc[17] = acc[3] - pre[3];
        acc[18] = (acc[4] + acc[5] + acc[6]) - pre[4];
        block_reduce<19, R>(acc, S.red, S.tot);
        if (t == 0) {
            for (int k = 0; k < 19; ++k) S.P[k] = S.tot[k];
            correction_solve<R>(g, S.P, S.mu, &fallback);
        }
        __syncthreads();
        for (int i = t; i < N; i += T)
            S.tab.cx[i] = (R)S.mu[1] * S.tab.v[i] + (R)S.mu[4] * S.tab.v2[i];
        // ---- h_c = N_c / w, and nu = sum_j lam_j (1 + eps h_c,j) psi_j --------
        const R *lam = lam_in + (int64_t)c * nvt;
        R nu[5] = {R(0), R(0), R(0), R(0), R(0)};
        for (int p = t; p < N2; p += T) {
            const int jy = p / N, jz = p % N;
            const R IAyz = S.tab.IA[jy] * S.tab.IA[jz];
            R s0 = R(0), s1 = R(0), s2 = R(0);
            for (int jx = 0; jx < N; ++jx) {
                const int j = jx * N2 + p;
                const R hc = S.B[j] * S.tab.IA[jx] * IAyz;
                S.B[j] = hc;
                const R tv = lam[j] * (R(1) + eps * hc);
                s0 += tv;
                s1 += tv * S.tab.v[jx];
                s2 += tv * S.tab.v2[jx];
            }
            const R vy = S.tab.v[jy], vz = S.tab.v[jz], q = vy * vy + vz * vz;
            nu[0] += s0;
            nu[1] += s1;
            nu[2] += vy * s0;
            nu[3] += vz * s0;
            nu[4] += s2 + q * s0;
        }
        block_reduce<5, R>(nu, S.red, S.tot);
        if (t == 0) {
            // xi = G^{-1} nu (G symmetric): dJ/dR = -xi, dJ/dG = -xi mu^T.
            R G[5][5], b[5], x[5];
            gram_of<R>(g, S.P, G);
            for (int a = 0; a < 5; ++a) b[a] = (R)S.tot[a];
            chol_or_ge<R>(G, b, x, &fallback);
            for (int a = 0; a < 5; ++a) S.xi[a] = (double)x[a];
        }
        __syncthreads();
        for (int i = t; i < N; i += T)
            S.cxi[i] = (R)S.xi[1] * S.tab.v[i] + (R)S.xi[4] * S.tab.v2[i];
        __syncthreads();
        // ---- lam_c = (lam - w psi.xi)(1 + eps psi.mu); dJ/dh~ = lam_c + w psi.xi
        for (int p = t; p < N2; p += T) {
            const int jy = p / N, jz = p % N;
            const R vy = S.tab.v[jy], vz = S.tab.v[jz], q = vy * vy + vz * vz;
            const R Ayz = S.tab.A[jy] * S.tab.A[jz], IAyz = S.tab.IA[jy] * S.tab.IA[jz];
            const R cti = (R)S.xi[0] + (R)S.xi[2] * vy + (R)S.xi[3] * vz + (R)S.xi[4] * q;
            const R ctm = (R)S.mu[0] + (R)S.mu[2] * vy + (R)S.mu[3] * vz + (R)S.mu[4] * q;
            for (int jx = 0; jx < N; ++jx) {
                const int j = jx * N2 + p;
                const R w = S.tab.A[jx] * Ayz;
                const R px = cti + S.cxi[jx], pm = ctm + S.tab.cx[jx];
                const R lc = (lam[j] - w * px) * (R(1) + eps * pm);
                S.B[j] = lc * (S.tab.IA[jx] * IAyz);     // lam_c / w
                S.C[j] = lc + w * px;
            }
        }
        __syncthreads();
        // ---- transposed Monte Carlo update (bilinear in h~) ----------------------
        for (int l = t; l < g.nt; l += T) {
            const int4 q = pidx[l];
            R gam = R(0);
            if (q.z >= 0) gam += S.B[q.z];
            if (q.w >= 0) gam += S.B[q.w];
            if (q.x >= 0) gam -= S.B[q.x];
            if (q.y >= 0) gam -= S.B[q.y];
            gam *= pa[l].W;
            if (gam != R(0)) {
                const R ha = q.x >= 0 ? S.A[q.x] : R(0);
                const R hb = q.y >= 0 ? S.A[q.y] : R(0);
                if (q.x >= 0) atomicAdd(S.C + q.x, gam * (R(1) + eps * hb));
                if (q.y >= 0) atomicAdd(S.C + q.y, gam * (R(1) + eps * ha));
            }
        }
        __syncthreads();
        R *dst = lt + (int64_t)c * nvt;
        for (int j = t; j < nvt; j += T) dst[j] = S.C[j];
        __syncthreads();
    }
    if (fallback && stats) atomicAdd(stats + 3, (unsigned long long)fallback);
}

// Per face: the sensitivities of its ghost values, gathered from dJ/dh~ of
// the boundary cell (inflow nodes, weight |Cu_n|) and, on the lid, from the
// shear D_n; turned into dJ/dF (F = outgoing flux sum |v_n| w h) in lF[f] and,
// on the lid, into dJ/dU added to grad_lid.  The factor r = Phi_w / (n_w
// Phi0) depends on v_x only (walls at rest: 1) and is tabulated per face.
template <typename R>
__global__ void k_adj_walls(Geo g, const int64_t *__restrict__ stepp, const R *__restrict__ lt,
                            const double *__restrict__ nw, double *__restrict__ lF,
                            double *__restrict__ grad_lid, double wD)
{
    __shared__ double red[kMaxWarps * kRedSlots];
    __shared__ double tot[4];
    __shared__ R rt[kMaxN], sA[kMaxN], sv[kMaxN], se[kMaxN], sde[kMaxN];
    const int64_t step = *stepp;
    const int f = blockIdx.x;
    const Face F = face_of(g, f, step);
    const int N = g.nv, N2 = N * N;
    const bool lid = f >= 2 * g.ny + g.nx;
    const double cdx = g.dt / (F.nax == 0 ? g.dx : g.dy), U = F.U;
    // Per node of the axis: r = Phi_w / (n_w Phi0) (walls at rest: 1) and the
    // terms of the inflow density D_in(U) and of its U-derivative.
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const R v = (R)g.axv[i], u = (R)U;
        sv[i] = v;
        sA[i] = (R)g.axA[i];
        rt[i] = lid ? exp(R(2) * v * u - u * u) : R(1);
        const R d = v - u, e = (R)(g.dv * 0.5641895835477563) * exp(-d * d);
        se[i] = e;
        sde[i] = e * R(2) * d;
    }
    __syncthreads();
    const R *L = lt + (int64_t)F.cell * g.nvt;
    const R dcoef = (R)(lid && wD != 0.0 ? wD * 2.0 / g.nx : 0.0), rcdx = (R)cdx;
    // Thread t takes node jz = t mod N of every (t div N)-th (jx, jy) row
    // whose normal velocity points into the cell (v_n > 0: the upper half of
    // the normal axis for an inward normal along +e_n, the lower half for
    // -e_n, the axes being symmetric); per-thread sums in the state's
    // precision, the block sum in double.
    R a0 = R(0), a1 = R(0);        // sum lg r, sum lg r v_x
    const int per = blockDim.x / N, jz = threadIdx.x % N, H = N / 2;
    const int jlo = F.nsign > 0.0 ? N - H : 0;
    const int nrow = N * H;        // rows with v_n > 0
    if ((int)threadIdx.x < per * N) {
        // kWallLoads rows at a time: their loads are in flight together.
        for (int r0 = threadIdx.x / N; r0 < nrow; r0 += kWallLoads * per) {
            R ls[kWallLoads];
#pragma unroll
            for (int k = 0; k < kWallLoads; ++k) {
                const int r = r0 + k * per;
                // side walls: jx in the half, jy free; bottom and lid: jy in it
                const int a = r / H, b = r - a * H;
                const int row = F.nax == 0 ? (jlo + r / N) * N + r % N : a * N + jlo + b;
                ls[k] = r < nrow ? L[row * N + jz] : R(0);
            }
#pragma unroll
            for (int k = 0; k < kWallLoads; ++k) {
                const int r = r0 + k * per;
                if (r >= nrow) break;
                const int a = r / H, b = r - a * H;
                const int jx = F.nax == 0 ? jlo + r / N : a, jy = F.nax == 0 ? r % N : jlo + b;
                const R vx = sv[jx], vy = sv[jy];
                const R vn = (F.nax == 0 ? vx : vy) * (R)F.nsign;
                R lg = vn * rcdx * ls[k];
                if (dcoef != R(0)) lg += dcoef * sA[jx] * sA[jy] * sA[jz] * vx * vy;
                const R lr = lg * rt[jx];
                a0 += lr;
                a1 += lr * vx;
            }
        }
    }
    double acc[2] = {(double)a0, (double)a1};
    block_reduce<2, double>(acc, red, tot);
    if (threadIdx.x == 0) {
        double ts = 0.0, dts = 0.0;
        for (int jt = 0; jt < N; ++jt) {
            ts += (double)se[jt];
            dts += (double)sde[jt];
        }
        const double din = g.hn * ts * g.zsum, ddin = g.hn * dts * g.zsum;
        lF[f] = tot[0] / din;
        if (lid && grad_lid)
            grad_lid[f - 2 * g.ny - g.nx] +=
                nw[f] / g.eps * (2.0 * (tot[1] - U * tot[0]) - ddin / din * tot[0]);
    }
}

// dJ/dh^n: the transposed upwind stencil (h^n_c feeds h~ of its downwind
// neighbours) plus, on boundary cells, the outgoing-flux terms of their faces
// and on the lid row the term of the lid shear D_n.
template <typename R>
__global__ void k_adj_stream(Geo g, const R *__restrict__ lt, const double *__restrict__ lF,
                             R *__restrict__ lam_out, double wD)
{
    __shared__ R sv[kMaxN], sax[kMaxN], say[kMaxN];
    const int N = g.nv, N2 = N * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double v = g.axv[i];
        sv[i] = (R)v;
        sax[i] = (R)(fabs(v) * g.dt / g.dx);
        say[i] = (R)(fabs(v) * g.dt / g.dy);
    }
    __syncthreads();
    const int64_t nvt = g.nvt;
    for (int c = blockIdx.x; c < g.nr; c += gridDim.x) {
        const int ix = c % g.nx, iy = c / g.nx;
        const bool edge = ix == 0 || ix == g.nx - 1 || iy == 0 || iy == g.ny - 1;
        const R *Lc = lt + (int64_t)c * nvt;
        R *o = lam_out + (int64_t)c * nvt;
        for (int j = threadIdx.x; j < g.nvt; j += blockDim.x) {
            const int jx = j / N2, jy = (j / N) % N;
            const R vx = sv[jx], vy = sv[jy], ax = sax[jx], ay = say[jy];
            R s = (R(1) - ax - ay) * Lc[j];
            if (vx > R(0) && ix < g.nx - 1) s += ax * Lc[nvt + j];
            if (vx < R(0) && ix > 0) s += ax * Lc[j - nvt];
            if (vy > R(0) && iy < g.ny - 1) s += ay * Lc[g.nx * nvt + j];
            if (vy < R(0) && iy > 0) s += ay * Lc[j - g.nx * nvt];
            if (edge) {
                const int jz = j % N;
                const double w = g.axA[jx] * g.axA[jy] * g.axA[jz];
                const double dvx = g.axv[jx], dvy = g.axv[jy];
                double extra = 0.0;
                if (ix == 0 && dvx < 0.0) extra -= lF[iy] * dvx * w;
                if (ix == g.nx - 1 && dvx > 0.0) extra += lF[g.ny + iy] * dvx * w;
                if (iy == 0 && dvy < 0.0) extra -= lF[2 * g.ny + ix] * dvy * w;
                if (iy == g.ny - 1 && dvy > 0.0) {
                    extra += lF[2 * g.ny + g.nx + ix] * dvy * w;
                    extra += wD * 2.0 * w * dvx * dvy / g.nx;
                }
                s += (R)extra;
            }
            o[j] = s;
        }
    }
}

}  // namespace bzk
