/*
 * bz_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see the
 * header).  Every function cites the passage of Frezzotti, Ghiroldi &
 * Gibelli, "Solving the Boltzmann equation on GPUs", that it follows.
 * Compiled with -O2 -ffp-contract=off; OpenMP over spatial cells only.
 *
 * Readings where the paper is silent or inconsistent (kept in sync with the
 * design notes of the repository):
 *  - post-collision map with v_r = v1 - v (Algorithm 2), which conserves
 *    energy; the Sec. 2 text writes v_r = v - v1 with the same map, which
 *    does not;
 *  - Jacobi evaluation of the collision sum on the post-streaming h~
 *    (Eq. collision_step) rather than Algorithm 3's in-place sequence;
 *  - the 1/Nt factor of Eq. monteCarloInt is kept in the weights;
 *  - h := 0 outside the velocity box, and chi terms of nodes outside the box
 *    are dropped (the correction restores the conserved moments);
 *  - moments written from their definitions in V0 = sqrt(2RT0) units;
 *  - K = n0 sigma^2 lambda0 from the hard-sphere viscosity with the
 *    Chapman-Cowling factor 1.016034 (caller supplies K).
 */
#include "bz_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define BZO_TWO_PI 6.283185307179586
#define BZO_PI 3.141592653589793

/* ------------------------------------------------------------------ */
/* Grid and derived quantities (Sec. 3, Sec. 5.1)                      */
/* ------------------------------------------------------------------ */

double bzo_dv(const bzo_problem *p) { return (2.0 * p->vmax) / (double)p->nv; }
double bzo_dx(const bzo_problem *p) { return (1.0 / p->kn) / (double)p->nx; }
double bzo_dy(const bzo_problem *p) { return (1.0 / p->kn) / (double)p->ny; }

static int stretched(double r) { return r > 0.0 && r != 1.0; }

/* Velocity cell edges (Sec. 5.1).  Uniform: -vmax + k dv.  Stretched with
 * ratio rv: the nv/2 cells of each half axis have widths d0, d0/rv, d0/rv^2,
 * ... outward from the origin (the smallest cells at the origin), summing to
 * vmax; the edges are symmetric about 0. */
double bzo_axis_edge(const bzo_problem *p, int32_t k)
{
    if (!stretched(p->rv)) return -p->vmax + (double)k * bzo_dv(p);
    int32_t m = p->nv / 2;
    double q = 1.0 / p->rv;
    double d0 = p->vmax * (q - 1.0) / (pow(q, (double)m) - 1.0);
    int32_t i = k >= m ? k - m : m - k;           /* edge index from the origin */
    double e = d0 * (pow(q, (double)i) - 1.0) / (q - 1.0);
    return k >= m ? e : -e;
}

double bzo_axis_width(const bzo_problem *p, int32_t j)
{
    if (!stretched(p->rv)) return bzo_dv(p);
    return bzo_axis_edge(p, j + 1) - bzo_axis_edge(p, j);
}

/* Node velocity of axis index j: the centre of its cell. */
double bzo_node_v(const bzo_problem *p, int32_t j)
{
    if (!stretched(p->rv)) return -p->vmax + ((double)j + 0.5) * bzo_dv(p);
    return 0.5 * (bzo_axis_edge(p, j) + bzo_axis_edge(p, j + 1));
}

/* Spatial cell widths (Sec. 5.1, stretched physical grid): widths shrink by
 * rx per cell toward each side wall and by ry per cell toward the lid (the
 * smallest cells at the upper corners), normalised to the side L. */
static double stretched_width(int32_t n, int32_t d, int32_t i, double r, double L)
{
    /* cell i has distance d(i) (in cells) from the refined end(s); width ~ r^-d */
    double sum = 0.0;
    for (int32_t k = 0; k < n; ++k) {
        int32_t dk = d < 0 ? (k < n - 1 - k ? k : n - 1 - k) : n - 1 - k;
        sum += pow(1.0 / r, (double)dk);
    }
    int32_t di = d < 0 ? (i < n - 1 - i ? i : n - 1 - i) : n - 1 - i;
    return L * pow(1.0 / r, (double)di) / sum;
}

double bzo_cell_dx(const bzo_problem *p, int32_t ix)
{
    if (!stretched(p->rx)) return bzo_dx(p);
    return stretched_width(p->nx, -1, ix, p->rx, 1.0 / p->kn);
}

double bzo_cell_dy(const bzo_problem *p, int32_t iy)
{
    if (!stretched(p->ry)) return bzo_dy(p);
    return stretched_width(p->ny, 1, iy, p->ry, 1.0 / p->kn);
}

/* Time step from the maximum Courant number per direction (Sec. 5.1), with
 * the fastest node and the narrowest cell. */
double bzo_dt(const bzo_problem *p)
{
    double vtop = bzo_node_v(p, p->nv - 1);
    double h = bzo_cell_dx(p, 0);
    for (int32_t i = 1; i < p->nx; ++i)
        if (bzo_cell_dx(p, i) < h) h = bzo_cell_dx(p, i);
    for (int32_t i = 0; i < p->ny; ++i)
        if (bzo_cell_dy(p, i) < h) h = bzo_cell_dy(p, i);
    return p->cfl * h / vtop;
}

static void node_velocity(const bzo_problem *p, int32_t j, double v[3])
{
    int32_t n = p->nv;
    int32_t jz = j % n, jy = (j / n) % n, jx = j / (n * n);
    v[0] = bzo_node_v(p, jx);
    v[1] = bzo_node_v(p, jy);
    v[2] = bzo_node_v(p, jz);
}

/* dV_j of node j: the product of its three axis widths. */
static double node_volume(const bzo_problem *p, int32_t j)
{
    int32_t n = p->nv;
    int32_t jz = j % n, jy = (j / n) % n, jx = j / (n * n);
    return bzo_axis_width(p, jx) * bzo_axis_width(p, jy) * bzo_axis_width(p, jz);
}

/* Equilibrium Maxwellian Phi0 in V0 units with n0 = 1 (Eq. MaxwellDist). */
static double phi0(const double v[3])
{
    return pow(BZO_PI, -1.5) * exp(-(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
}

/* N_j ~ dV_j Phi0_j h_j (Sec. 3): the node weight dV_j Phi0_j. */
double bzo_weight(const bzo_problem *p, int32_t j)
{
    double v[3];
    node_velocity(p, j, v);
    return node_volume(p, j) * phi0(v);
}

/* Lid speed of lid face ix at the start of step `step`. */
double bzo_lid_speed(const bzo_problem *p, int32_t ix, int64_t step)
{
    double base = p->lid_profile ? p->lid_profile[ix] : p->lid_u0;
    double t = (double)step * bzo_dt(p);
    if (p->lid_period > 0.0)
        base += p->lid_amp * sin(BZO_TWO_PI * t / p->lid_period);
    return base;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from the definition in Salmon et al. (SC'11)         */
/* ------------------------------------------------------------------ */

void bzo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* ------------------------------------------------------------------ */
/* Sampling (Eq. coll8Dim / monteCarloInt; Sec. 4.2 sampling kernel)   */
/* ------------------------------------------------------------------ */

static double uniform01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

/* chi_j support: the node whose velocity cell holds v, or -1. */
int32_t bzo_node_of(const bzo_problem *p, const double v[3], int32_t *near_face)
{
    double dv = bzo_dv(p);
    int32_t id[3], inside = 1, near = 0;
    if (stretched(p->rv)) {
        /* the cell whose edges hold v (a value on an edge goes to the upper cell) */
        for (int c = 0; c < 3; ++c) {
            if (!(v[c] >= bzo_axis_edge(p, 0)) || v[c] >= bzo_axis_edge(p, p->nv)) {
                inside = 0;
                id[c] = -1;
                continue;
            }
            int32_t k = 0;
            while (v[c] >= bzo_axis_edge(p, k + 1)) ++k;
            double w = bzo_axis_width(p, k);
            if (v[c] - bzo_axis_edge(p, k) < 1e-9 * w || bzo_axis_edge(p, k + 1) - v[c] < 1e-9 * w)
                near = 1;
            id[c] = k;
        }
        if (near_face) *near_face = near;
        if (!inside) return -1;
        return (id[0] * p->nv + id[1]) * p->nv + id[2];
    }
    for (int c = 0; c < 3; ++c) {
        double t = (v[c] + p->vmax) / dv;
        double fl = floor(t);
        double fr = t - fl;
        if (fr < 1e-9 || fr > 1.0 - 1e-9) near = 1;
        if (!(t >= 0.0) || fl >= (double)p->nv) {
            inside = 0;
            id[c] = -1;
        } else {
            id[c] = (int32_t)fl;
        }
    }
    if (near_face) *near_face = near;
    if (!inside) return -1;
    return (id[0] * p->nv + id[1]) * p->nv + id[2];
}

void bzo_sample(const bzo_problem *p, int64_t step, uint32_t cellword, int64_t l,
                bzo_sample_t *o)
{
    uint32_t key[2] = {p->seed, p->instance};
    uint32_t x[8];
    for (uint32_t d = 0; d < 2; ++d) {
        uint32_t ctr[4] = {(uint32_t)l, (uint32_t)step, cellword, d};
        bzo_philox4x32_10(ctr, key, x + 4 * d);
    }
    double u[8];
    for (int i = 0; i < 8; ++i) u[i] = uniform01(x[i]);

    /* v, v1 ~ Phi0 by Box-Muller: each pair of uniforms gives two normals of
     * variance 1/2 (Phi0 = pi^{-3/2} e^{-v^2}). */
    double r0 = sqrt(-log(u[0])), t0 = BZO_TWO_PI * u[1];
    double r1 = sqrt(-log(u[2])), t1 = BZO_TWO_PI * u[3];
    double r2 = sqrt(-log(u[4])), t2 = BZO_TWO_PI * u[5];
    o->v[0] = r0 * cos(t0);
    o->v[1] = r0 * sin(t0);
    o->v[2] = r1 * cos(t1);
    o->v1[0] = r1 * sin(t1);
    o->v1[1] = r2 * cos(t2);
    o->v1[2] = r2 * sin(t2);

    /* k uniform on the unit sphere through (k_z, phi) as in Eq. coll8Dim. */
    double kz = 1.0 - 2.0 * u[6];
    double ph = BZO_TWO_PI * u[7];
    double st = sqrt(1.0 - kz * kz);
    o->k[0] = st * cos(ph);
    o->k[1] = st * sin(ph);
    o->k[2] = kz;

    /* Post-collision velocities with v_r = v1 - v (Algorithm 2). */
    double vr[3];
    for (int c = 0; c < 3; ++c) vr[c] = o->v1[c] - o->v[c];
    double s = (vr[0] * o->k[0] + vr[1] * o->k[1]) + vr[2] * o->k[2];
    for (int c = 0; c < 3; ++c) {
        o->vs[c] = o->v[c] + s * o->k[c];
        o->v1s[c] = o->v1[c] - s * o->k[c];
    }
    o->s = s;

    /* Eq. monteCarloInt prefactor n0^2 d^2 pi / Nt becomes pi K / Nt in
     * lambda0/V0 units; times dt for the explicit update (Eq. collision_step). */
    double cw = BZO_PI * p->kcoll * bzo_dt(p) / (double)p->nt;
    o->W = cw * fabs(s);

    int32_t nf, near = 0;
    o->idx[0] = bzo_node_of(p, o->v, &nf);   near |= nf;
    o->idx[1] = bzo_node_of(p, o->v1, &nf);  near |= nf;
    o->idx[2] = bzo_node_of(p, o->vs, &nf);  near |= nf;
    o->idx[3] = bzo_node_of(p, o->v1s, &nf); near |= nf;
    o->near_face = near;
}

void bzo_sample_all(const bzo_problem *p, int64_t step, uint32_t cellword,
                    bzo_sample_t *out)
{
    for (int64_t l = 0; l < p->nt; ++l) bzo_sample(p, step, cellword, l, out + l);
}

/* ------------------------------------------------------------------ */
/* Maxwell diffuse walls (Eq. bcMax and the n_w condition, Sec. 2)     */
/* ------------------------------------------------------------------ */

int32_t bzo_num_faces(const bzo_problem *p) { return 2 * p->nx + 2 * p->ny; }

/* Face geometry: boundary cell, inward normal, wall velocity. */
static void face_info(const bzo_problem *p, int64_t step, int32_t f, int32_t *cell,
                      double nrm[3], double vw[3])
{
    int32_t nx = p->nx, ny = p->ny;
    nrm[0] = nrm[1] = nrm[2] = 0.0;
    vw[0] = vw[1] = vw[2] = 0.0;
    if (f < ny) {                       /* left wall x = -L/2 */
        *cell = f * nx;
        nrm[0] = 1.0;
    } else if (f < 2 * ny) {            /* right wall x = +L/2 */
        *cell = (f - ny) * nx + (nx - 1);
        nrm[0] = -1.0;
    } else if (f < 2 * ny + nx) {       /* bottom wall y = 0 */
        *cell = f - 2 * ny;
        nrm[1] = 1.0;
    } else {                            /* lid y = L, moving along +x */
        int32_t ix = f - 2 * ny - nx;
        *cell = (ny - 1) * nx + ix;
        nrm[1] = -1.0;
        vw[0] = bzo_lid_speed(p, ix, step);
    }
}

static double wall_maxwellian(const double v[3], const double vw[3])
{
    double d0 = v[0] - vw[0], d1 = v[1] - vw[1], d2 = v[2] - vw[2];
    return pow(BZO_PI, -1.5) * exp(-(d0 * d0 + d1 * d1 + d2 * d2));
}

/* n_w from zero net mass flux through the face; integrals become sums over the
 * velocity nodes with the same weights as everywhere else. */
static double face_density(const bzo_problem *p, int64_t step, int32_t f, const double *hcell)
{
    int32_t nvt = p->nv * p->nv * p->nv;
    int32_t cell;
    double nrm[3], vw[3], v[3];
    face_info(p, step, f, &cell, nrm, vw);
    double out = 0.0, in = 0.0;
    for (int32_t j = 0; j < nvt; ++j) {
        node_velocity(p, j, v);
        double vn = v[0] * nrm[0] + v[1] * nrm[1] + v[2] * nrm[2];
        if (vn < 0.0)
            out += -vn * bzo_weight(p, j) * (1.0 + p->eps * hcell[j]);
        else if (vn > 0.0)
            in += vn * node_volume(p, j) * wall_maxwellian(v, vw);
    }
    return out / in;
}

void bzo_wall_density(const bzo_problem *p, int64_t step, const double *h, double *nw)
{
    int32_t nf = bzo_num_faces(p), nvt = p->nv * p->nv * p->nv;
    for (int32_t f = 0; f < nf; ++f) {
        int32_t cell;
        double nrm[3], vw[3];
        face_info(p, step, f, &cell, nrm, vw);
        nw[f] = face_density(p, step, f, h + (int64_t)cell * nvt);
    }
}

/* Emitted distribution n_w Phi_w written as Phi0 (1 + eps h_w). */
double bzo_ghost(const bzo_problem *p, int64_t step, int32_t f, double nw, int32_t j)
{
    int32_t cell;
    double nrm[3], vw[3], v[3];
    face_info(p, step, f, &cell, nrm, vw);
    node_velocity(p, j, v);
    return (nw * wall_maxwellian(v, vw) / phi0(v) - 1.0) / p->eps;
}

/* ------------------------------------------------------------------ */
/* Free streaming: first-order explicit upwind scheme (Eq. streaming2D) */
/* ------------------------------------------------------------------ */

/* Eq. streaming2D for every node of cell c.  nb[0] is the cell's own slab,
 * nb[1..4] the left, right, lower and upper neighbours (NULL at a wall, where
 * the diffusely emitted ghost value of that face is used). */
static void stream_cell(const bzo_problem *p, int64_t step, int32_t c, const double *nb[5],
                        const double *nw, double *out)
{
    int32_t nx = p->nx, ny = p->ny, n = p->nv;
    int32_t ix = c % nx, iy = c / nx;
    int64_t nvt = (int64_t)n * n * n;
    /* Each cell uses its own widths: the upwind finite-volume update of a
     * cell of width dx_i (uniform widths give Eq. streaming2D as printed). */
    double dt = bzo_dt(p), dx = bzo_cell_dx(p, ix), dy = bzo_cell_dy(p, iy);
    for (int64_t j = 0; j < nvt; ++j) {
        double v[3];
        node_velocity(p, (int32_t)j, v);
        double cux = v[0] * dt / dx, cuy = v[1] * dt / dy;
        double h0 = nb[0][j];
        double hx = h0, hy = h0;
        if (v[0] > 0.0) {           /* upwind neighbour on the left */
            hx = nb[1] ? nb[1][j] : bzo_ghost(p, step, iy, nw[iy], (int32_t)j);
        } else if (v[0] < 0.0) {    /* upwind neighbour on the right */
            hx = nb[2] ? nb[2][j] : bzo_ghost(p, step, ny + iy, nw[ny + iy], (int32_t)j);
        }
        if (v[1] > 0.0) {           /* upwind neighbour below */
            hy = nb[3] ? nb[3][j] : bzo_ghost(p, step, 2 * ny + ix, nw[2 * ny + ix], (int32_t)j);
        } else if (v[1] < 0.0) {    /* upwind neighbour above (lid) */
            hy = nb[4] ? nb[4][j]
                       : bzo_ghost(p, step, 2 * ny + nx + ix, nw[2 * ny + nx + ix], (int32_t)j);
        }
        double ax = fabs(cux), ay = fabs(cuy);
        out[j] = (1.0 - ax - ay) * h0 + ax * hx + ay * hy;
    }
}

void bzo_stream(const bzo_problem *p, int64_t step, const double *h, double *ht)
{
    int32_t nx = p->nx, ny = p->ny, n = p->nv;
    int64_t nvt = (int64_t)n * n * n;
    int32_t nf = bzo_num_faces(p);
    double *nw = (double *)malloc(sizeof(double) * nf);
    bzo_wall_density(p, step, h, nw);

#pragma omp parallel for schedule(static)
    for (int32_t c = 0; c < nx * ny; ++c) {
        const double *nb[5];
        nb[0] = h + (int64_t)c * nvt;
        nb[1] = c % nx > 0 ? h + (int64_t)(c - 1) * nvt : NULL;
        nb[2] = c % nx < nx - 1 ? h + (int64_t)(c + 1) * nvt : NULL;
        nb[3] = c / nx > 0 ? h + (int64_t)(c - nx) * nvt : NULL;
        nb[4] = c / nx < ny - 1 ? h + (int64_t)(c + nx) * nvt : NULL;
        stream_cell(p, step, c, nb, nw, ht + (int64_t)c * nvt);
    }
    free(nw);
}

/* ------------------------------------------------------------------ */
/* Homogeneous relaxation (Eqs. monteCarloInt, collision_step,          */
/* rinorm_a, correzione) and macroscopic quantities (Eqs. densita..sforzi) */
/* ------------------------------------------------------------------ */

/* Collision invariants psi = 1, v, v^2 used by the correction. */
static void invariants(const double v[3], double phi[5])
{
    phi[0] = 1.0;
    phi[1] = v[0];
    phi[2] = v[1];
    phi[3] = v[2];
    phi[4] = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
}

/* Gaussian elimination with partial pivoting on a 5x5 system. */
static int solve5(double A[5][5], double b[5], double x[5])
{
    for (int k = 0; k < 5; ++k) {
        int piv = k;
        for (int i = k + 1; i < 5; ++i)
            if (fabs(A[i][k]) > fabs(A[piv][k])) piv = i;
        if (A[piv][k] == 0.0) return -1;
        if (piv != k) {
            for (int j = 0; j < 5; ++j) {
                double t = A[k][j];
                A[k][j] = A[piv][j];
                A[piv][j] = t;
            }
            double t = b[k];
            b[k] = b[piv];
            b[piv] = t;
        }
        for (int i = k + 1; i < 5; ++i) {
            double m = A[i][k] / A[k][k];
            for (int j = k; j < 5; ++j) A[i][j] -= m * A[k][j];
            b[i] -= m * b[k];
        }
    }
    for (int i = 4; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < 5; ++j) s -= A[i][j] * x[j];
        x[i] = s / A[i][i];
    }
    return 0;
}

static void cell_moments(const bzo_problem *p, const double *hc, const double *w,
                         const double *vel, double *m)
{
    int64_t nvt = (int64_t)p->nv * p->nv * p->nv;
    double m0 = 0, m1[3] = {0, 0, 0}, m2[3][3] = {{0}};
    for (int64_t j = 0; j < nvt; ++j) {
        double wh = w[j] * hc[j];
        const double *v = vel + 3 * j;
        m0 += wh;
        for (int a = 0; a < 3; ++a) {
            m1[a] += wh * v[a];
            for (int b = 0; b < 3; ++b) m2[a][b] += wh * v[a] * v[b];
        }
    }
    double eps = p->eps;
    double rho = m0, n = 1.0 + eps * rho;
    double u[3] = {m1[0] / n, m1[1] / n, m1[2] / n};
    double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double tr = m2[0][0] + m2[1][1] + m2[2][2];
    m[0] = rho;
    m[1] = u[0];
    m[2] = u[1];
    m[3] = u[2];
    m[4] = ((2.0 / 3.0) * tr - rho) / n - (2.0 * eps / 3.0) * u2;
    static const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
    for (int q = 0; q < 6; ++q)
        m[5 + q] = 2.0 * m2[pa[q]][pb[q]] - 2.0 * eps * n * u[pa[q]] * u[pb[q]];
}

static void tables(const bzo_problem *p, double **w, double **vel)
{
    int64_t nvt = (int64_t)p->nv * p->nv * p->nv;
    *w = (double *)malloc(sizeof(double) * nvt);
    *vel = (double *)malloc(sizeof(double) * 3 * nvt);
    for (int64_t j = 0; j < nvt; ++j) {
        (*w)[j] = bzo_weight(p, (int32_t)j);
        node_velocity(p, (int32_t)j, *vel + 3 * j);
    }
}

void bzo_moments(const bzo_problem *p, const double *h, double *mom)
{
    int64_t nvt = (int64_t)p->nv * p->nv * p->nv;
    double *w, *vel;
    tables(p, &w, &vel);
#pragma omp parallel for schedule(static)
    for (int32_t c = 0; c < p->nx * p->ny; ++c)
        cell_moments(p, h + (int64_t)c * nvt, w, vel, mom + 11 * (int64_t)c);
    free(w);
    free(vel);
}

/* Relaxation of one cell (Eqs. monteCarloInt, collision_step, rinorm_a,
 * correzione) from h (= h~) into o, with scratch dN, hc of nv^3 doubles. */
static void collide_cell(const bzo_problem *p, const bzo_sample_t *smp, const double *w,
                         const double *vel, const double *h, double *o, double *stage,
                         double *dN, double *hc)
{
    int64_t nvt = (int64_t)p->nv * p->nv * p->nv;
    double eps = p->eps;
    /* Moments of h~ to be preserved (Eq. correzione, right side). */
    double pre[5] = {0, 0, 0, 0, 0}, phi[5];
    for (int64_t j = 0; j < nvt; ++j) {
        invariants(vel + 3 * j, phi);
        for (int a = 0; a < 5; ++a) pre[a] += w[j] * h[j] * phi[a];
    }
    /* Eq. monteCarloInt evaluated on h~ (Eq. collision_step). */
    memset(dN, 0, sizeof(double) * nvt);
    for (int64_t l = 0; l < p->nt; ++l) {
        const bzo_sample_t *q = smp + l;
        double ha = q->idx[0] >= 0 ? h[q->idx[0]] : 0.0;
        double hb = q->idx[1] >= 0 ? h[q->idx[1]] : 0.0;
        double g = ha + hb + eps * ha * hb;
        double r = q->W * g;
        if (q->idx[2] >= 0) dN[q->idx[2]] += r;
        if (q->idx[3] >= 0) dN[q->idx[3]] += r;
        if (q->idx[0] >= 0) dN[q->idx[0]] -= r;
        if (q->idx[1] >= 0) dN[q->idx[1]] -= r;
    }
    for (int64_t j = 0; j < nvt; ++j) hc[j] = h[j] + dN[j] / w[j];
    if (stage) memcpy(stage, hc, sizeof(double) * nvt);

    /* Correction of the full distribution (Eqs. rinorm_a, correzione):
     * Phi0 (1 + eps h^{n+1}) = Phi0 (1 + eps h_c) (1 + eps mu.psi), so
     * sum_b [sum_j w (1 + eps h_c) psi_a psi_b] mu_b = -(post_a - pre_a). */
    double G[5][5] = {{0}}, R[5] = {0, 0, 0, 0, 0}, mu[5];
    for (int64_t j = 0; j < nvt; ++j) {
        invariants(vel + 3 * j, phi);
        double f = w[j] * (1.0 + eps * hc[j]);
        for (int a = 0; a < 5; ++a) {
            R[a] += w[j] * hc[j] * phi[a];
            for (int b = 0; b < 5; ++b) G[a][b] += f * phi[a] * phi[b];
        }
    }
    double rhs[5];
    for (int a = 0; a < 5; ++a) rhs[a] = -(R[a] - pre[a]);
    if (solve5(G, rhs, mu) != 0) mu[0] = mu[1] = mu[2] = mu[3] = mu[4] = 0.0;
    for (int64_t j = 0; j < nvt; ++j) {
        invariants(vel + 3 * j, phi);
        double corr = mu[0] * phi[0] + mu[1] * phi[1] + mu[2] * phi[2] +
                      mu[3] * phi[3] + mu[4] * phi[4];
        o[j] = hc[j] + (1.0 + eps * hc[j]) * corr;
    }
}

void bzo_collide(const bzo_problem *p, int64_t step, const bzo_sample_t *samples,
                 const double *ht, double *hout, double *mom, double *stage)
{
    int32_t nr = p->nx * p->ny;
    int64_t nvt = (int64_t)p->nv * p->nv * p->nv;
    double *w, *vel;
    tables(p, &w, &vel);

    bzo_sample_t *shared = NULL;
    if (!samples && !p->per_cell) {
        shared = (bzo_sample_t *)malloc(sizeof(bzo_sample_t) * p->nt);
        bzo_sample_all(p, step, 0xFFFFFFFFu, shared);
        samples = shared;
    }

#pragma omp parallel
    {
        double *dN = (double *)malloc(sizeof(double) * nvt);
        double *hc = (double *)malloc(sizeof(double) * nvt);
        bzo_sample_t *own = NULL;
        if (!samples) own = (bzo_sample_t *)malloc(sizeof(bzo_sample_t) * p->nt);
#pragma omp for schedule(static)
        for (int32_t c = 0; c < nr; ++c) {
            const bzo_sample_t *smp = samples;
            if (!smp) {
                bzo_sample_all(p, step, (uint32_t)c, own);
                smp = own;
            }
            collide_cell(p, smp, w, vel, ht + (int64_t)c * nvt, hout + (int64_t)c * nvt,
                         stage ? stage + (int64_t)c * nvt : NULL, dN, hc);
            if (mom) cell_moments(p, hout + (int64_t)c * nvt, w, vel, mom + 11 * (int64_t)c);
        }
        free(dN);
        free(hc);
        free(own);
    }
    free(shared);
    free(w);
    free(vel);
}

/* Time splitting (Sec. 3): h^n -> free streaming -> h~ -> relaxation -> h^{n+1}. */
void bzo_step(const bzo_problem *p, int64_t step, const double *h, double *hnext,
              double *mom)
{
    int64_t tot = (int64_t)p->nx * p->ny * p->nv * p->nv * p->nv;
    double *ht = (double *)malloc(sizeof(double) * tot);
    bzo_stream(p, step, h, ht);
    bzo_collide(p, step, NULL, ht, hnext, mom, NULL);
    free(ht);
}

/* One full step of a single cell from its own slab and its four neighbours
 * (NULL where the cell touches a wall): the wall densities of its own
 * boundary faces, Eq. streaming2D, and the relaxation with the step's sample
 * set.  Gives the same values as bzo_step for that cell. */
void bzo_step_cell(const bzo_problem *p, int64_t step, int32_t c, const double *own,
                   const double *left, const double *right, const double *below,
                   const double *above, double *out, double *mom)
{
    int32_t nx = p->nx, ny = p->ny, nf = bzo_num_faces(p);
    int64_t nvt = (int64_t)p->nv * p->nv * p->nv;
    int32_t ix = c % nx, iy = c / nx;
    double *nw = (double *)calloc((size_t)nf, sizeof(double));
    if (ix == 0) nw[iy] = face_density(p, step, iy, own);
    if (ix == nx - 1) nw[ny + iy] = face_density(p, step, ny + iy, own);
    if (iy == 0) nw[2 * ny + ix] = face_density(p, step, 2 * ny + ix, own);
    if (iy == ny - 1) nw[2 * ny + nx + ix] = face_density(p, step, 2 * ny + nx + ix, own);
    const double *nb[5] = {own, ix > 0 ? left : NULL, ix < nx - 1 ? right : NULL,
                           iy > 0 ? below : NULL, iy < ny - 1 ? above : NULL};
    double *ht = (double *)malloc(sizeof(double) * nvt);
    stream_cell(p, step, c, nb, nw, ht);
    double *w, *vel;
    tables(p, &w, &vel);
    bzo_sample_t *smp = (bzo_sample_t *)malloc(sizeof(bzo_sample_t) * p->nt);
    bzo_sample_all(p, step, p->per_cell ? (uint32_t)c : 0xFFFFFFFFu, smp);
    double *dN = (double *)malloc(sizeof(double) * nvt);
    double *hc = (double *)malloc(sizeof(double) * nvt);
    collide_cell(p, smp, w, vel, ht, out, NULL, dN, hc);
    if (mom) cell_moments(p, out, w, vel, mom);
    free(nw); free(ht); free(w); free(vel); free(smp); free(dN); free(hc);
}

/* Wall shear on the lid (D of Sec. 5.2): x-momentum flux through each lid
 * face, 2 sum_j w_j v_x v_y h_face,j with the cell value for v_y > 0 and the
 * emitted (ghost) value for v_y < 0. */
void bzo_lid_shear(const bzo_problem *p, int64_t step, const double *h, double *out)
{
    int32_t nx = p->nx, ny = p->ny;
    int64_t nvt = (int64_t)p->nv * p->nv * p->nv;
    int32_t nf = bzo_num_faces(p);
    double *nw = (double *)malloc(sizeof(double) * nf);
    bzo_wall_density(p, step, h, nw);
    double mean = 0.0;
    for (int32_t ix = 0; ix < nx; ++ix) {
        int32_t f = 2 * ny + nx + ix;
        int64_t c = (int64_t)(ny - 1) * nx + ix;
        double s = 0.0, v[3];
        for (int64_t j = 0; j < nvt; ++j) {
            node_velocity(p, (int32_t)j, v);
            double hf;
            if (v[1] > 0.0) hf = h[c * nvt + j];
            else if (v[1] < 0.0) hf = bzo_ghost(p, step, f, nw[f], (int32_t)j);
            else continue;
            s += bzo_weight(p, (int32_t)j) * v[0] * v[1] * hf;
        }
        out[ix] = 2.0 * s;
        mean += out[ix] * bzo_cell_dx(p, ix);
    }
    out[nx] = mean * p->kn;                     /* (1/L) sum_ix dx_ix shear_ix */
    free(nw);
}

/* ------------------------------------------------------------------ */
/* Monte Carlo estimate of Eq. coll8Dim for one cell, split into gain    */
/* (chi_j(v*) + chi_j(v1*)) and loss (chi_j(v) + chi_j(v1)) parts        */
/* ------------------------------------------------------------------ */

void bzo_mc_dNdt(const bzo_problem *p, int64_t step, const double *h, double *gain,
                 double *loss)
{
    int64_t nvt = (int64_t)p->nv * p->nv * p->nv;
    double eps = p->eps, dt = bzo_dt(p);
    memset(gain, 0, sizeof(double) * nvt);
    memset(loss, 0, sizeof(double) * nvt);
    for (int64_t l = 0; l < p->nt; ++l) {
        bzo_sample_t q;
        bzo_sample(p, step, 0xFFFFFFFFu, l, &q);
        double ha = q.idx[0] >= 0 ? h[q.idx[0]] : 0.0;
        double hb = q.idx[1] >= 0 ? h[q.idx[1]] : 0.0;
        double r = q.W / dt * (ha + hb + eps * ha * hb);
        if (q.idx[2] >= 0) gain[q.idx[2]] += r;
        if (q.idx[3] >= 0) gain[q.idx[3]] += r;
        if (q.idx[0] >= 0) loss[q.idx[0]] += r;
        if (q.idx[1] >= 0) loss[q.idx[1]] += r;
    }
}

int32_t bzo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Adjoint of one time step (fixed sample stream)                      */
/* ------------------------------------------------------------------ */
/* With the samples of a step fixed, the step h^n -> h^{n+1} is a smooth map
 * of h^n and of the lid speeds: streaming is linear in h^n apart from the
 * wall ghosts, which are affine in the outgoing flux and nonlinear in U;
 * the Monte Carlo update is bilinear in h~ (Eq. monteCarloInt); the
 * correction (Eqs. rinorm_a, correzione) is differentiated through its 5x5
 * solve.  Objective of interest: J = sum_n wD_n D_n, D_n the lid shear of
 * h^n (Sec. 5.2).  Given lam = dJ/dh^{n+1}, bzo_adjoint_step returns
 * dJ/dh^n (including wD dD_n/dh^n) and adds dJ/dU_i to grad_lid[i]. */

/* Phi_w / Phi0 at node velocity v for wall velocity vw: exp(|v|^2 - |v - vw|^2). */
static double ratio_w0(const double v[3], const double vw[3])
{
    double a = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double d0 = v[0] - vw[0], d1 = v[1] - vw[1], d2 = v[2] - vw[2];
    return exp(a - (d0 * d0 + d1 * d1 + d2 * d2));
}

/* For face f: D_in = sum_{vn>0} vn dV Phi_w and its derivative in the
 * tangential wall speed (x component). */
static void face_influx(const bzo_problem *p, int64_t step, int32_t f, double *din, double *ddin)
{
    int32_t cell, nvt = p->nv * p->nv * p->nv;
    double nrm[3], vw[3], v[3];
    face_info(p, step, f, &cell, nrm, vw);
    double s = 0.0, ds = 0.0;
    for (int32_t j = 0; j < nvt; ++j) {
        node_velocity(p, j, v);
        double vn = v[0] * nrm[0] + v[1] * nrm[1] + v[2] * nrm[2];
        if (vn > 0.0) {
            double m = vn * node_volume(p, j) * wall_maxwellian(v, vw);
            s += m;
            ds += m * 2.0 * (v[0] - vw[0]);
        }
    }
    *din = s;
    *ddin = ds;
}

void bzo_adjoint_step(const bzo_problem *p, int64_t step, const double *h, const double *lam_in,
                      double *lam_out, double *grad_lid, double wD)
{
    int32_t nx = p->nx, ny = p->ny, nr = nx * ny, n = p->nv, nf = bzo_num_faces(p);
    int64_t nvt = (int64_t)n * n * n;
    double eps = p->eps, dt = bzo_dt(p);
    double *w, *vel;
    tables(p, &w, &vel);

    /* ---- forward recompute: walls, streaming, samples ---- */
    double *nw = (double *)malloc(sizeof(double) * nf);
    bzo_wall_density(p, step, h, nw);
    double *ht = (double *)malloc(sizeof(double) * nr * nvt);
    bzo_stream(p, step, h, ht);
    bzo_sample_t *smp = (bzo_sample_t *)malloc(sizeof(bzo_sample_t) * p->nt);
    bzo_sample_all(p, step, 0xFFFFFFFFu, smp);

    /* ---- collision adjoint, cell by cell: lam^{n+1} -> lam~ ---- */
    double *lt = (double *)calloc((size_t)nr * nvt, sizeof(double));
#pragma omp parallel
    {
        double *dN = (double *)malloc(sizeof(double) * nvt);
        double *hc = (double *)malloc(sizeof(double) * nvt);
        double *lc = (double *)malloc(sizeof(double) * nvt);
#pragma omp for schedule(static)
        for (int32_t c = 0; c < nr; ++c) {
            const double *hh = ht + (int64_t)c * nvt;
            const double *lam = lam_in + (int64_t)c * nvt;
            double *out = lt + (int64_t)c * nvt;
            double phi[5];
            /* forward: h_c, G, mu exactly as bzo_collide */
            double pre[5] = {0, 0, 0, 0, 0};
            for (int64_t j = 0; j < nvt; ++j) {
                invariants(vel + 3 * j, phi);
                for (int a = 0; a < 5; ++a) pre[a] += w[j] * hh[j] * phi[a];
            }
            memset(dN, 0, sizeof(double) * nvt);
            for (int64_t l = 0; l < p->nt; ++l) {
                const bzo_sample_t *q = smp + l;
                double ha = q->idx[0] >= 0 ? hh[q->idx[0]] : 0.0;
                double hb = q->idx[1] >= 0 ? hh[q->idx[1]] : 0.0;
                double r = q->W * (ha + hb + eps * ha * hb);
                if (q->idx[2] >= 0) dN[q->idx[2]] += r;
                if (q->idx[3] >= 0) dN[q->idx[3]] += r;
                if (q->idx[0] >= 0) dN[q->idx[0]] -= r;
                if (q->idx[1] >= 0) dN[q->idx[1]] -= r;
            }
            for (int64_t j = 0; j < nvt; ++j) hc[j] = hh[j] + dN[j] / w[j];
            double G[5][5] = {{0}}, R[5] = {0, 0, 0, 0, 0}, mu[5], Gs[5][5];
            for (int64_t j = 0; j < nvt; ++j) {
                invariants(vel + 3 * j, phi);
                double f = w[j] * (1.0 + eps * hc[j]);
                for (int a = 0; a < 5; ++a) {
                    R[a] += w[j] * hc[j] * phi[a];
                    for (int b = 0; b < 5; ++b) G[a][b] += f * phi[a] * phi[b];
                }
            }
            memcpy(Gs, G, sizeof(G));
            double rhs[5];
            for (int a = 0; a < 5; ++a) rhs[a] = -(R[a] - pre[a]);
            if (solve5(G, rhs, mu) != 0) mu[0] = mu[1] = mu[2] = mu[3] = mu[4] = 0.0;
            /* nu = d J / d mu = sum_j lam_j (1 + eps h_c,j) psi_j ; xi = G^{-1} nu */
            double nu[5] = {0, 0, 0, 0, 0}, xi[5];
            for (int64_t j = 0; j < nvt; ++j) {
                invariants(vel + 3 * j, phi);
                for (int a = 0; a < 5; ++a) nu[a] += lam[j] * (1.0 + eps * hc[j]) * phi[a];
            }
            if (solve5(Gs, nu, xi) != 0) xi[0] = xi[1] = xi[2] = xi[3] = xi[4] = 0.0;
            /* dJ/dh_c and the direct dJ/dh~ of the moments of h~ */
            for (int64_t j = 0; j < nvt; ++j) {
                invariants(vel + 3 * j, phi);
                double px = 0.0, pm = 0.0;
                for (int a = 0; a < 5; ++a) {
                    px += phi[a] * xi[a];
                    pm += phi[a] * mu[a];
                }
                lc[j] = (lam[j] - w[j] * px) * (1.0 + eps * pm);
                out[j] = lc[j] + w[j] * px;
            }
            /* transposed Monte Carlo update: h_c = h~ + S(h~)/w, S bilinear */
            for (int64_t l = 0; l < p->nt; ++l) {
                const bzo_sample_t *q = smp + l;
                double gam = 0.0;
                if (q->idx[2] >= 0) gam += lc[q->idx[2]] / w[q->idx[2]];
                if (q->idx[3] >= 0) gam += lc[q->idx[3]] / w[q->idx[3]];
                if (q->idx[0] >= 0) gam -= lc[q->idx[0]] / w[q->idx[0]];
                if (q->idx[1] >= 0) gam -= lc[q->idx[1]] / w[q->idx[1]];
                gam *= q->W;
                double ha = q->idx[0] >= 0 ? hh[q->idx[0]] : 0.0;
                double hb = q->idx[1] >= 0 ? hh[q->idx[1]] : 0.0;
                if (q->idx[0] >= 0) out[q->idx[0]] += gam * (1.0 + eps * hb);
                if (q->idx[1] >= 0) out[q->idx[1]] += gam * (1.0 + eps * ha);
            }
        }
        free(dN);
        free(hc);
        free(lc);
    }

    /* ---- streaming adjoint: lam~ -> lam^n, ghosts collected per face ---- */
    double *lg = (double *)calloc((size_t)nf * nvt, sizeof(double)); /* dJ/d ghost_f(j) */
    memset(lam_out, 0, sizeof(double) * nr * nvt);
    for (int32_t c = 0; c < nr; ++c) {
        int32_t ix = c % nx, iy = c / nx;
        double dxc = bzo_cell_dx(p, ix), dyc = bzo_cell_dy(p, iy);
        for (int64_t j = 0; j < nvt; ++j) {
            double v[3];
            node_velocity(p, (int32_t)j, v);
            double ax = fabs(v[0] * dt / dxc), ay = fabs(v[1] * dt / dyc);
            double L = lt[(int64_t)c * nvt + j];
            lam_out[(int64_t)c * nvt + j] += (1.0 - ax - ay) * L;
            if (v[0] > 0.0) {
                if (ix > 0) lam_out[(int64_t)(c - 1) * nvt + j] += ax * L;
                else lg[(int64_t)iy * nvt + j] += ax * L;
            } else if (v[0] < 0.0) {
                if (ix < nx - 1) lam_out[(int64_t)(c + 1) * nvt + j] += ax * L;
                else lg[(int64_t)(ny + iy) * nvt + j] += ax * L;
            } else {
                lam_out[(int64_t)c * nvt + j] += ax * L;
            }
            if (v[1] > 0.0) {
                if (iy > 0) lam_out[(int64_t)(c - nx) * nvt + j] += ay * L;
                else lg[(int64_t)(2 * ny + ix) * nvt + j] += ay * L;
            } else if (v[1] < 0.0) {
                if (iy < ny - 1) lam_out[(int64_t)(c + nx) * nvt + j] += ay * L;
                else lg[(int64_t)(2 * ny + nx + ix) * nvt + j] += ay * L;
            } else {
                lam_out[(int64_t)c * nvt + j] += ay * L;
            }
        }
    }

    /* ---- lid shear D_n: its own ghost sensitivities ---- */
    if (wD != 0.0) {
        for (int32_t ix = 0; ix < nx; ++ix) {
            int32_t f = 2 * ny + nx + ix;
            int64_t c = (int64_t)(ny - 1) * nx + ix;
            for (int64_t j = 0; j < nvt; ++j) {
                double v[3];
                node_velocity(p, (int32_t)j, v);
                double coef = wD * 2.0 * w[j] * v[0] * v[1] * bzo_cell_dx(p, ix) * p->kn;
                if (v[1] > 0.0) lam_out[c * nvt + j] += coef;
                else if (v[1] < 0.0) lg[(int64_t)f * nvt + j] += coef;
            }
        }
    }

    /* ---- ghosts -> outgoing flux of each face, and the lid speeds ---- */
    for (int32_t f = 0; f < nf; ++f) {
        int32_t cell;
        double nrm[3], vw[3], v[3];
        face_info(p, step, f, &cell, nrm, vw);
        double din, ddin;
        face_influx(p, step, f, &din, &ddin);
        double lF = 0.0, lU = 0.0;
        for (int64_t j = 0; j < nvt; ++j) {
            double L = lg[(int64_t)f * nvt + j];
            if (L == 0.0) continue;
            node_velocity(p, (int32_t)j, v);
            double r = ratio_w0(v, vw);
            /* ghost = (n_w r - 1)/eps, n_w = out/in: d/dF = r/in (F: outgoing h-flux) */
            lF += L * r / din;
            /* d/dU = (n_w r / eps) [2 (v_x - U) - din'/din] */
            lU += L * (nw[f] * r / eps) * (2.0 * (v[0] - vw[0]) - ddin / din);
        }
        for (int64_t j = 0; j < nvt; ++j) {
            node_velocity(p, (int32_t)j, v);
            double vn = v[0] * nrm[0] + v[1] * nrm[1] + v[2] * nrm[2];
            if (vn < 0.0) lam_out[(int64_t)cell * nvt + j] += lF * (-vn) * w[j];
        }
        if (f >= 2 * ny + nx && grad_lid) grad_lid[f - 2 * ny - nx] += lU;
    }
    free(lg);
    free(lt);
    free(ht);
    free(nw);
    free(smp);
    free(w);
    free(vel);
}
