/*
 * bz.h -- C ABI of a GB300-native (sm_103a) semi-regular Boltzmann solver.
 *
 * Method: Frezzotti, Ghiroldi & Gibelli, "Solving the Boltzmann equation on
 * GPUs".  The deviational distribution h, f = Phi0 (1 + eps h) (Sec. 2,
 * Eq. definition), is advanced on a 2D driven cavity by time splitting
 * (Sec. 3): first-order upwind free streaming with Maxwell diffuse walls
 * (Eqs. streaming2D, bcMax), then a Monte Carlo evaluation of the hard-sphere
 * collision integral on a Cartesian velocity grid (Eqs. coll8Dim,
 * monteCarloInt, collision_step) and the Aristov-Tcheremissine conservation
 * correction (Eqs. rinorm_a, correzione).
 *
 * Units: velocities in V0 = sqrt(2 R T0); lengths in lambda0 =
 * (mu0/p0) V0 with mu0 the hard-sphere viscosity; times in lambda0/V0; n0 = 1;
 * Phi0(v) = pi^{-3/2} exp(-|v|^2).  Geometry (Sec. 5.1): the cavity is
 * [-L/2, L/2] x [0, L] with L = 1/kn; the lid y = L moves along +x; all
 * walls are at T0.
 *
 * State layout (device memory, owned by the handle): h[cell][node] with
 * cell = iy*nx + ix (x fastest) and node j = (jx*nv + jy)*nv + jz; element
 * type float (BZ_F32) or double (BZ_F64).  Node velocities are the cell
 * centres v = -vmax + (j + 1/2) dv, dv = 2 vmax / nv.
 *
 * Conventions:
 *  - every call returns a bz_status; nothing is thrown across the ABI;
 *  - a `stream` argument is a cudaStream_t passed as void* (NULL = legacy
 *    default stream); device work is enqueued on it asynchronously and errors
 *    of that work surface at the next call that synchronises;
 *  - pointer arguments documented as "host or device" may be either (the copy
 *    uses unified addressing); all other pointers are as documented;
 *  - inputs are copied at the call; the library never keeps caller pointers;
 *  - a handle is not thread-safe; distinct handles are independent;
 *  - bz_last_error() returns a thread-local message for the last failure.
 */
#ifndef BZ_H
#define BZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bz_handle bz_handle;

typedef enum {
    BZ_OK = 0,
    BZ_EINVAL = 1,        /* invalid argument (message says which) */
    BZ_ENOMEM = 2,        /* device allocation failed */
    BZ_ECUDA = 3,         /* a CUDA runtime call failed (message has the text) */
    BZ_EDEVICE = 4,       /* a kernel reported an inconsistency (error word) */
    BZ_ETIMEOUT = 5,      /* a bounded device wait gave up */
    BZ_ENONFINITE = 6,    /* a non-finite moment was produced */
    BZ_ESTATE = 7,        /* call not valid in the handle's current state */
    BZ_EUNSUPPORTED = 8   /* configuration outside what the kernels support */
} bz_status;

enum { BZ_F32 = 0, BZ_F64 = 1 };             /* state element type */
enum { BZ_SHARED = 0, BZ_PER_CELL = 1 };     /* Monte Carlo sample sets */

/* Sub-step selection for bz_step_ex (tests and profiling). */
enum {
    BZ_DO_STREAM = 1u,     /* walls + free streaming into h~ (Eq. streaming2D) */
    BZ_DO_COLLIDE = 2u,    /* sampling + collision + correction on the state */
    BZ_SPLIT = 4u          /* full step as separate stream and collide kernels */
};

/* Spatial grid (Sec. 3, Sec. 5.1): nx x ny cells on the square cavity of
 * side L = 1/kn (Knudsen number kn = 1/delta).  rx, ry: stretched cells
 * (Sec. 5.1; 0 or 1 = uniform): column widths shrink by the factor rx per
 * cell toward each side wall, row heights by ry per cell toward the lid, the
 * smallest cells at the lid corners; widths sum to L.  The time step then
 * follows from the narrowest cell. */
typedef struct {
    int32_t nx, ny;
    double kn;
    double rx, ry;
} bz_space;

/* Velocity grid (Sec. 3): nv^3 nodes on the cube [-vmax, vmax]^3 (V0 units).
 * rv: stretched cells (Sec. 5.1; 0 or 1 = uniform; nv even): along each axis
 * the cell widths grow by 1/rv per cell outward from the origin (the
 * smallest cells at the origin), edges symmetric about 0; a node sits at the
 * centre of its cell and its weight is its cell volume times Phi0. */
typedef struct {
    int32_t nv;
    double vmax;
    double rv;
} bz_vel;

/* Walls (Sec. 2 Eq. bcMax, Sec. 5.1): the lid speed of lid face ix at time
 * t is U_ix(t) = base_ix + lid_amp sin(2 pi t / lid_period) (the sine term
 * only when lid_period > 0), with base_ix = lid_profile[ix] when lid_profile
 * is non-NULL (host pointer to nx doubles, copied) and lid_u0 otherwise.
 * All other walls are at rest; every wall is at T0. */
typedef struct {
    double lid_u0, lid_amp, lid_period;
    const double *lid_profile;
} bz_walls;

/* Method parameters.
 *   n_pairs     Monte Carlo samples per step, Nt of Eq. monteCarloInt (>= 1)
 *   seed        Philox4x32-10 key word 0; instance = key word 1
 *   eps         deviation parameter of Eq. definition; 0 => max |U| (1 if
 *               the lid never moves)
 *   cfl         maximum Courant number per direction (Sec. 5.1); 0 => 0.5
 *   kcoll       K = n0 sigma^2 lambda0; 0 => hard-sphere value
 *               (5 * 1.016034 / 16) sqrt(2/pi) (Sec. 5.1, lambda0)
 *   dtype       BZ_F32 or BZ_F64 state
 *   sample_mode BZ_SHARED: one sample set per step for all cells (Sec. 3,
 *               "the same set of collisions"); BZ_PER_CELL: independent sets */
typedef struct {
    int64_t n_pairs;
    uint32_t seed, instance;
    double eps, cfl, kcoll;
    int32_t dtype;
    int32_t sample_mode;
} bz_params;

/* Derived quantities of a handle. */
typedef struct {
    double dt, dx, dy, dv, eps, kcoll;
    int64_t nodes;          /* nx*ny*nv^3 */
    int64_t state_bytes;    /* one state buffer */
    int64_t step;           /* steps taken so far (time t = step * dt) */
    int32_t nr, nvt;        /* cells, velocity nodes */
    int32_t dtype;
    int32_t threads_per_cell, smem_bytes;  /* per-cell kernel launch shape */
    int32_t kernel_variant;  /* 0: generic per-cell kernel; 1: FP32 4-node-vector kernel;
                                2: FP32 active-node kernel with deferred correction */
    int32_t plan_batch;      /* active-node kernel: the sample plans of this many
                                consecutive steps are built together, by the first step
                                that needs a plan the last batch does not hold; 0: each
                                step builds its own plan, or another kernel runs */
    int64_t plan_end;        /* with plan_batch > 0: the first step the built plans do not
                                cover (a step from there on builds the next batch) */
} bz_info;

/* Create a solver for the driven cavity.  Validates every argument
 * (BZ_EINVAL), rejects grids whose velocity slab does not fit one SM's
 * shared memory (BZ_EUNSUPPORTED), allocates two state buffers and the
 * per-step scratch on the current device (BZ_ENOMEM), and sets h = 0, the
 * uniform equilibrium n0, T0 of Sec. 5.1.  *out is NULL on failure. */
bz_status bz_create(const bz_space *space, const bz_vel *vel, const bz_walls *walls,
                    const bz_params *params, bz_handle **out);

/* Release a handle and all device memory it owns (NULL is accepted). */
bz_status bz_destroy(bz_handle *h);

/* Advance nsteps >= 0 time steps (Sec. 3 time splitting): per step the
 * wall densities from h^n (Eq. bcMax), the shared sample set (Sec. 4.2,
 * Algorithm 2), and one fused kernel that streams (Eq. streaming2D),
 * collides (Eq. collision_step), corrects (Eqs. rinorm_a, correzione) and
 * reduces the moments.  On the FP32 active-node path the sample sets of
 * bz_info.plan_batch steps are built ahead in one batch (they depend on the
 * step number only), so the step that starts a batch carries its cost.
 * Asynchronous on `stream`. */
bz_status bz_step(bz_handle *h, int32_t nsteps, void *stream);

/* Like bz_step with the sub-steps chosen by `flags` (BZ_DO_STREAM,
 * BZ_DO_COLLIDE, BZ_SPLIT).  BZ_DO_STREAM alone replaces the state by h~
 * without advancing the step counter; BZ_DO_COLLIDE alone applies the
 * relaxation of step `step` to the current state and advances the counter;
 * both (or BZ_SPLIT) take one full step with separate kernels. */
bz_status bz_step_ex(bz_handle *h, int32_t nsteps, uint32_t flags, void *stream);

/* Macroscopic quantities of every cell (Eqs. densita..sforzi, written in V0
 * units): out[cell*11 + k], k = rho, ux, uy, uz, theta, Pxx, Pyy, Pzz, Pxy,
 * Pxz, Pyz, as doubles; `out` (nx*ny*11 doubles, host or device) is written
 * on `stream` (synchronously when it is pageable host memory).
 * BZ_ENONFINITE if any value is not finite (the values are still written). */
bz_status bz_moments(bz_handle *h, double *out, void *stream);

/* Wall shear on the lid (D of Sec. 5.2): out[ix] for ix < nx is the
 * x-momentum flux 2 sum_j w_j v_x v_y h_face,j through lid face ix of the
 * current state, with h_face the cell value for v_y > 0 and the diffusely
 * emitted value for v_y < 0; out[nx] is their mean D.  out: nx+1 doubles,
 * host or device. */
bz_status bz_lid_shear(bz_handle *h, double *out, void *stream);

/* Copy the state out of / into the handle (layout above; dtype of the
 * handle).  dst/src: host or device, nx*ny*nv^3 elements.  get returns the
 * step counter in *step (nullable); set overwrites it with `step`. */
bz_status bz_get_state(bz_handle *h, void *dst, int64_t *step, void *stream);
bz_status bz_set_state(bz_handle *h, const void *src, int64_t step, void *stream);

/* Replace the lid motion (same meaning as bz_walls; profile host, copied).
 * The deviation parameter eps is not changed. */
bz_status bz_set_lid(bz_handle *h, double lid_u0, double lid_amp, double lid_period,
                     const double *lid_profile);

bz_status bz_get_info(const bz_handle *h, bz_info *out);

/* Counters since creation: [0] steps, [1] samples with a node outside the
 * velocity box, [2] samples within 1e-9 dv of a cell face, [3] correction
 * solves that fell back from Cholesky to pivoted elimination, [4] kernel
 * launches issued; on the active-node path (bz_info.kernel_variant 2) [5]
 * steps whose active velocity nodes exceeded the kernel's compact arrays (they
 * ran the fallback kernel), [6] active nodes of the latest step, [7] the
 * compact arrays' capacity; otherwise [5..7] are 0.  Synchronises the device.
 * Returns BZ_ETIMEOUT (out filled all the same) when a bounded device wait
 * of the active-node kernel gave up since the last call (only its optional
 * bulk-copy streaming ring waits on the device; the steps concerned are
 * invalid); the flag is then cleared. */
bz_status bz_stats(bz_handle *h, int64_t out[8]);

/* The Monte Carlo sample set of step `step` (Sec. 4.2, Algorithm 2) as the
 * device computes it: idx[4*l + q] = node of v, v1, v*, v1* (q = 0..3; -1
 * outside the box) and W[l] = pi K dt |(v1 - v).k| / Nt (Eq. monteCarloInt
 * times dt) in double.  Both outputs host or device (4*Nt int32, Nt double).
 * For parity checks; the step path keeps its own copy in device scratch. */
bz_status bz_sample_plan(bz_handle *h, int64_t step, int32_t *idx, double *W, void *stream);

/* The sample set of cell `cell` (0 <= cell < nx*ny, row-major) at step `step`
 * as the BZ_PER_CELL step draws it (Sec. 4.2 with the cell index in the
 * sampler's counter): same layout and units as bz_sample_plan.  For FP32
 * handles the sampler's arithmetic is FP32 except near a velocity-cell face,
 * where the sample is drawn again in double, so idx equals the double-
 * precision node selection and W carries FP32 error (a few 1e-6 of
 * |v1 - v| in |(v1 - v).k|).  Valid whatever the handle's sample mode.
 * BZ_EINVAL on a NULL pointer, a negative step or a cell out of range. */
bz_status bz_sample_plan_cell(bz_handle *h, int64_t step, int32_t cell, int32_t *idx, double *W,
                              void *stream);

/* Adjoint of one time step with its Monte Carlo sample set fixed.  With the
 * samples of step n fixed, the step h^n -> h^{n+1} (upwind streaming with
 * diffuse walls, Eqs. streaming2D and bcMax; the Jacobi Monte Carlo update,
 * Eqs. monteCarloInt and collision_step; the correction, Eqs. rinorm_a and
 * correzione) is a smooth function of h^n and of the lid face speeds U_i at
 * t_n.  The paper has no adjoint: this call transposes those equations so
 * that gradients of a wall-shear objective (D of Sec. 5.2) with respect to
 * the lid profile and the initial state can be taken through many steps.
 *
 * h_n: device, the state at step `step` (nx*ny*nv^3 elements of the handle's
 * dtype, layout above).  lam_in: device, the same shape, dJ/dh^{n+1}.
 * lam_out: device, the same shape, receives dJ/dh^n; it may be lam_in itself
 * but must not overlap h_n.  grad_lid: device, nx doubles, or NULL; dJ/dU_i
 * is ADDED to grad_lid[i].  wD: weight of the lid shear D_n of h^n in J
 * (D_n as bz_lid_shear's out[nx]); its terms are added to lam_out and
 * grad_lid.  The lid motion is the handle's (bz_set_lid).  The handle's
 * state, step counter and moments are not touched; the adjoint scratch (the
 * sample set, the ghost values and one state-sized buffer) is allocated on
 * the first call (BZ_ENOMEM on failure).  BZ_EUNSUPPORTED when three
 * velocity slabs and the per-sample products do not fit one block's shared
 * memory.  Asynchronous on `stream`. */
bz_status bz_adjoint_step(bz_handle *h, int64_t step, const void *h_n, const void *lam_in,
                          void *lam_out, double *grad_lid, double wD, void *stream);

/* Device Philox4x32-10 (Salmon et al., SC'11) words for n counters
 * (ctr: 4*n uint32, host or device) under key (k0, k1); out: 4*n uint32,
 * host or device.  Synchronous.  For cross-checks of the generator. */
bz_status bz_philox(uint32_t k0, uint32_t k1, const uint32_t *ctr, int64_t n, uint32_t *out);

/* ---------------------------------------------------------------------
 * Batches: many independent cavity instances (each with its own grids, Kn,
 * lid, sample count and Philox key) advanced together, every step one CUDA
 * graph launch.  Three schedules: persistent kernels (one launch per kernel
 * class and step over the cells of all instances, the FP32 4-node-vector
 * per-cell kernel); fan-out (every instance's own active-node step, the
 * instances spread over up to 8 concurrent graph branches); persistent
 * active-node kernels (one launch per kernel class over all instances, the
 * active-node kernel claiming (instance, group of four cells) segments from
 * a work list, one launch per velocity-grid size; available when every
 * instance runs the active-node path with four cells per group).  The two
 * active-node schedules copy every instance's sample plans from the batches
 * built ahead (built between steps, before the step's graph launch, when an
 * instance's step leaves its last batch).  bz_batch_tune chooses.  Every instance must be FP32 with nv a multiple of 4 and >= 12,
 * at most 32768 samples per step, the shared sample set and uniform grids
 * (BZ_EUNSUPPORTED otherwise).  The batch owns its instances; instance i is
 * addressed by its index.  The state of an instance at step n lives in one of
 * its two buffers chosen by the parity of n, so the per-instance calls below
 * are the way to read and write it. */
typedef struct bz_batch bz_batch;

bz_status bz_batch_create(int32_t n, const bz_space *spaces, const bz_vel *vels,
                          const bz_walls *walls, const bz_params *params, bz_batch **out);
bz_status bz_batch_destroy(bz_batch *b);
/* Advance every instance by nsteps (asynchronous on stream). */
bz_status bz_batch_step(bz_batch *b, int32_t nsteps, void *stream);
bz_status bz_batch_set_state(bz_batch *b, int32_t i, const void *src, int64_t step, void *stream);
bz_status bz_batch_get_state(bz_batch *b, int32_t i, void *dst, int64_t *step, void *stream);
/* Moments of instance i's current state (as bz_moments). */
bz_status bz_batch_moments(bz_batch *b, int32_t i, double *out, void *stream);
/* Autotuner: times `trial_steps` recomputations of the current step (the
 * state is not advanced) for every schedule (persistent kernels: threads per
 * CTA 512 or 1024, CTAs per SM, cell-strip width 4, 8 or 16; fan-out: 1, 2, 4
 * or 8 branches, as a graph; the persistent active-node schedule where
 * available), keeps the fastest and returns its index in *choice (nullable)
 * and the milliseconds per step of every schedule in ms[0..ncand) (nullable,
 * up to 16 entries). */
bz_status bz_batch_tune(bz_batch *b, int32_t trial_steps, void *stream, int32_t *choice,
                        double *ms, int32_t *ncand);
/* Schedule in use: out[0..2] the persistent kernels' threads per CTA,
 * persistent CTAs and strip width; out[3] the fan-out branches, 0 when the
 * persistent 4-node-vector kernels run and -1 when the persistent
 * active-node kernels run. */
bz_status bz_batch_schedule(const bz_batch *b, int32_t out[4]);

/* Per-kernel timing with CUDA events recorded on the launching stream around
 * every kernel the handle launches while enabled (enable != 0); disabling
 * keeps what was recorded.  On the active-node path the fused steps keep
 * running as two-step CUDA graphs: enable == 1 captures one in which the
 * per-cell kernel's launches (class 2 only) are bracketed by event record
 * nodes, and every replay first gives those nodes fresh events.
 * bz_profile_read synchronises, returns per kernel
 * class k (0 walls, 1 sampling, 2 per-cell step or collision, 3 streaming)
 * the summed device time ms[k] and the launch count launches[k] since the
 * last read, and clears the record.  No counterpart in the paper (its timings
 * are host-side, Sec. 5.2); used by the benchmark. */
bz_status bz_profile(bz_handle *h, int32_t enable);
bz_status bz_profile_read(bz_handle *h, double ms[4], int64_t launches[4]);

/* Phase trace of the FP32 per-cell kernel, recorded while bz_profile(h, 2)
 * is on: SM clock (clock64) at up to 9 phase points of the first 8 work
 * items of CTA 0 in the latest launch.  For the quad kernel (kernel variant
 * 1) an item is a cell and the points are: cell start, after streaming,
 * gather, N = w h~, scatter, correction sums, solve, write-back, cell end.
 * For the active-node kernel (variant 2) an item is an iteration of its two
 * roles and the points are: iteration start, streaming done, collision
 * terms done, their sums done, write-back done, correction and moments of
 * the group two back done (the first two from a streaming thread, the next
 * three from a collision thread).  out: at least 72 int64, host; row-major
 * [item][point].  BZ_ESTATE if not enabled. */
bz_status bz_phase_clocks(bz_handle *h, int64_t *out, int32_t n);

/* ---------------------------------------------------------------------
 * Collision step without device allocation.  The paper has no counterpart.
 * This entry point is for callers that cannot call cudaMalloc: applications
 * whose device memory is all owned by their own pool allocator and that
 * forbid allocation while they run, and latency-critical loops in which a
 * cudaMalloc or cudaFree would synchronise the device.
 *
 * It computes what bz_step_ex(h, 1, BZ_DO_COLLIDE, ...) computes on a handle
 * holding h_in at step `step` (the step's shared Monte Carlo sample set, the
 * collision update and the conservation correction, no streaming), up to
 * floating-point summation order, and writes the result to h_out and, when
 * mom is non-NULL, its moments to mom (nx*ny*11 doubles, as bz_moments).
 * h_in and h_out are caller-owned device arrays of nx*ny*nv^3 elements of
 * params->dtype in the layout above; their byte ranges must not overlap
 * (BZ_EINVAL).  No walls are needed; params->eps must be given (> 0); cfl and
 * kcoll keep their defaults at 0; uniform grids and the shared sample set
 * only (BZ_EUNSUPPORTED otherwise).
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its only
 * scratch (the sample set, the per-axis velocity tables and the step number)
 * is a file-scope device array of BZ_NOALLOC_SCRATCH_BYTES, which every GPU
 * that loads the library holds until the process exits.  Hence n_pairs <=
 * BZ_NOALLOC_MAX_PAIRS (larger values return BZ_EINVAL), and the velocity slab
 * and the per-sample products must fit one block's shared memory (else
 * BZ_EUNSUPPORTED).  The first call on a device looks up the device address of
 * that array, with that device current.  Every call on a device uses the same
 * array, which keeps the last call's contents: calls on one device that
 * overlap in time (on different streams) race and give wrong results, so
 * serialise them; calls on different devices use different arrays.
 * Asynchronous on `stream`; errors as elsewhere. */
#define BZ_NOALLOC_MAX_PAIRS 65536
#define BZ_NOALLOC_SCRATCH_BYTES ((2u << 20) + 4096u)
bz_status bz_collide_noalloc(const bz_space *space, const bz_vel *vel, const bz_params *params,
                             int64_t step, const void *h_in, void *h_out, double *mom,
                             void *stream);

/* Thread-local text of the last failure on this thread ("" if none). */
const char *bz_last_error(void);

/* Library version string. */
const char *bz_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BZ_H */
