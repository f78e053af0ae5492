/*
 * bz_oracle.h -- plain FP64 CPU oracle for the semi-regular Boltzmann step of
 * Frezzotti, Ghiroldi & Gibelli, "Solving the Boltzmann equation on GPUs".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or constant with the CUDA
 * path.  It is deliberately slow and written to be read against the paper:
 * every function follows the equations in the order the paper states them,
 * in double precision, compiled without FMA contraction.
 *
 * Units (Sec. 5.1): velocities in V0 = sqrt(2 R T0), lengths in lambda0,
 * times in lambda0/V0, n0 = 1, so Phi0(v) = pi^{-3/2} exp(-|v|^2).
 *
 * Array layout shared with the library's public state format (an interface,
 * not code): h[cell][j], cell = iy*nx + ix (x fastest), velocity node
 * j = (jx*nv + jy)*nv + jz.
 */
#ifndef BZ_ORACLE_H
#define BZ_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Problem statement (Sec. 2, Sec. 5.1).  The oracle derives dt, dx, the
 * velocity nodes and the weights itself from these inputs. */
typedef struct {
    int32_t nx, ny;            /* spatial cells; cavity [-L/2,L/2] x [0,L] */
    double kn;                 /* Knudsen number; cavity side L = 1/kn (lambda0) */
    int32_t nv;                /* velocity nodes per axis */
    double vmax;               /* velocity box [-vmax, vmax]^3 */
    double eps;                /* deviation parameter epsilon, > 0 */
    double cfl;                /* maximum Courant number per direction */
    double kcoll;              /* collision constant K = n0 sigma^2 lambda0 */
    int64_t nt;                /* Monte Carlo samples per step */
    uint32_t seed, instance;   /* Philox key */
    int32_t per_cell;          /* 0: one sample set shared by all cells; 1: per cell */
    double lid_u0, lid_amp, lid_period; /* U(t) = base + amp sin(2 pi t / period) */
    const double *lid_profile; /* nx per-face base lid speeds, or NULL => lid_u0 */
    /* Stretched grids (Sec. 5.1; 0 or 1 = uniform).  rv: velocity cells grow
     * outward from the origin by 1/rv per cell (nv even).  rx: spatial cells
     * shrink by rx per cell toward each side wall; ry: toward the lid. */
    double rv, rx, ry;
} bzo_problem;

/* One Monte Carlo collision sample (Eq. monteCarloInt, Sec. 4.2 sampling). */
typedef struct {
    double v[3], v1[3], k[3];  /* drawn velocities and unit vector */
    double vs[3], v1s[3];      /* post-collision velocities v*, v1* */
    double s;                  /* (v1 - v) . k */
    double W;                  /* pi K dt |s| / Nt */
    int32_t idx[4];            /* node of v, v1, v*, v1*; -1 outside the box */
    int32_t near_face;         /* 1 if a component lies within 1e-9 dv of a face */
} bzo_sample_t;

/* Derived quantities.  bzo_dv/dx/dy are the uniform spacings (2 vmax / nv,
 * L / nx, L / ny); on stretched grids the per-node and per-cell widths are
 * bzo_axis_width, bzo_cell_dx and bzo_cell_dy. */
double bzo_dv(const bzo_problem *p);
double bzo_dx(const bzo_problem *p);
double bzo_dy(const bzo_problem *p);
double bzo_dt(const bzo_problem *p);
double bzo_node_v(const bzo_problem *p, int32_t jaxis);
/* Velocity cell edge k (0..nv) of one axis and the width of cell j. */
double bzo_axis_edge(const bzo_problem *p, int32_t k);
double bzo_axis_width(const bzo_problem *p, int32_t jaxis);
/* Width of spatial column ix and of row iy. */
double bzo_cell_dx(const bzo_problem *p, int32_t ix);
double bzo_cell_dy(const bzo_problem *p, int32_t iy);
double bzo_weight(const bzo_problem *p, int32_t j);        /* dV Phi0(v_j) */
double bzo_lid_speed(const bzo_problem *p, int32_t ix, int64_t step);

/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11). */
void bzo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Node index of a velocity (chi_j support), -1 outside the box. */
int32_t bzo_node_of(const bzo_problem *p, const double v[3], int32_t *near_face);

/* Draw sample l of step `step` for the given cell word (0xFFFFFFFF = shared). */
void bzo_sample(const bzo_problem *p, int64_t step, uint32_t cellword, int64_t l,
                bzo_sample_t *out);
void bzo_sample_all(const bzo_problem *p, int64_t step, uint32_t cellword,
                    bzo_sample_t *out /* nt */);

/* Diffuse walls (Eq. bcMax and the zero-mass-flux condition).
 * Faces: [0,ny) left, [ny,2ny) right, [2ny,2ny+nx) bottom, [2ny+nx,2ny+2nx) lid.
 * nw[f] is the wall density of face f computed from h (state at step start). */
int32_t bzo_num_faces(const bzo_problem *p);
void bzo_wall_density(const bzo_problem *p, int64_t step, const double *h, double *nw);
/* Ghost value h_w of face f at node j (only meaningful for inflow nodes). */
double bzo_ghost(const bzo_problem *p, int64_t step, int32_t f, double nw, int32_t j);

/* Free streaming with the first-order upwind scheme (Eq. streaming2D). */
void bzo_stream(const bzo_problem *p, int64_t step, const double *h, double *ht);

/* Homogeneous relaxation of every cell with an explicit sample table
 * (Eqs. monteCarloInt, collision_step, rinorm_a, correzione).  When
 * samples == NULL the sample sets are drawn from Philox for `step`.
 * mom (nullable): nr*11 moments of the result (densita..sforzi).
 * stage (nullable): nr*nv values of the uncorrected post-collision h_c. */
void bzo_collide(const bzo_problem *p, int64_t step, const bzo_sample_t *samples,
                 const double *ht, double *hout, double *mom, double *stage);

/* One full time step: walls from h^n, streaming, collision + correction. */
void bzo_step(const bzo_problem *p, int64_t step, const double *h, double *hnext,
              double *mom);

/* One full step of the single cell c (same values as bzo_step for it) from
 * its own slab and its left/right/lower/upper neighbours (NULL at walls).
 * out: nv^3 values; mom (nullable): 11 moments. */
void bzo_step_cell(const bzo_problem *p, int64_t step, int32_t c, const double *own,
                   const double *left, const double *right, const double *below,
                   const double *above, double *out, double *mom);

/* Macroscopic quantities of every cell (Eqs. densita..sforzi, V0 units):
 * [rho, ux, uy, uz, theta, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz]. */
void bzo_moments(const bzo_problem *p, const double *h, double *mom);

/* x-momentum flux through each lid face (wall shear), nx values, and D: their
 * mean over the lid, weighted by the face widths (out[nx]). */
void bzo_lid_shear(const bzo_problem *p, int64_t step, const double *h, double *out);

/* Monte Carlo estimate of Eq. coll8Dim (Eq. monteCarloInt) for one cell with
 * the shared sample set of `step`: dN_j/dt = gain_j - loss_j, where gain holds
 * the chi_j(v*) + chi_j(v1*) terms and loss the chi_j(v) + chi_j(v1) terms. */
void bzo_mc_dNdt(const bzo_problem *p, int64_t step, const double *h, double *gain,
                 double *loss);

/* Adjoint of step `step` with its sample set fixed: given h (= h^n) and
 * lam_in = dJ/dh^{n+1}, writes lam_out = dJ/dh^n and adds dJ/dU_i (lid face
 * speeds at t_n) to grad_lid[i] (nullable), for J containing wD * D_n, D_n
 * the mean lid shear of h^n (bzo_lid_shear). */
void bzo_adjoint_step(const bzo_problem *p, int64_t step, const double *h, const double *lam_in,
                      double *lam_out, double *grad_lid, double wD);

/* Number of OpenMP threads the oracle uses. */
int32_t bzo_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
