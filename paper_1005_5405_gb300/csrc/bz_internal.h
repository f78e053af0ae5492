// bz_internal.h -- helpers shared by the library's translation units.
#pragma once

#include "bz.h"

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

namespace bzk {
struct Geo;
}

// Stores the text returned by bz_last_error() on this thread.
void bz_record_error(const char *msg);

// Host tables of a discretised problem: velocity cell edges (nv + 1), node
// velocities, cell widths and weight factors A_j = width_j pi^-1/2
// exp(-v_j^2) per axis (nv each), and the spatial column and row widths.
struct bz_grid_tables {
    std::vector<double> edges, axv, axw, axA, cdx, cdy;
};

// The discretisation of a validated problem statement (Sec. 3, Sec. 5.1):
// fills every scalar field of g (sizes, dv, dx, dy, dt from the Courant
// number, the collision prefactor cw, eps, the Philox key, the lid motion,
// the wall flux constants, the equilibrium Gram matrix G0) and the host
// tables; device pointers of g are left untouched.  walls may be NULL (lid at
// rest; params->eps must then be > 0).  The one rule for bz_create and
// bz_collide_noalloc.
void bz_discretise(const bz_space *space, const bz_vel *vel, const bz_walls *walls,
                   const bz_params *params, bzk::Geo &g, bz_grid_tables &tb);

// A kernel's dynamic shared-memory limit is one setting for the whole
// process, shared by every handle that launches it: it is raised to the most
// the device allows next to the kernel's static shared memory, so that no
// handle can lower it below another handle's need.
template <typename Kernel>
cudaError_t bz_allow_max_smem(Kernel kernel, int optin)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

// Scratch of bz_adjoint_step (bz_adjoint.cu), owned by a handle.
struct bz_adj_scratch {
    int4 *pidx;          // sample node indices, logical order
    void *pa;            // gather records (a, b, W)
    void *ghost;         // ghost values of the forward walls of step n
    void *lt;            // dJ/dh~, one state
    double *nw, *lF;     // wall densities, dJ/d(outgoing flux) per face
    int64_t *step;       // device step counter of the recomputed step
    int threads, grid;
    size_t smem;
    // FP32 fast path (quad kernel): 16-bit plan in the shared-memory order,
    // the destination-sorted scatter list of the step, the quad mapping.
    bool fast;
    void *pidx16, *pa16;
    int *sc_count, *sc_cursor, *sc_meta;   // counts and cursors of both lists, 2 x nvt;
    uint32_t *sc_ent;                      // headers: forward list, then the loss list
    uint4 *lrec;         // the loss-term records of the transposed update
    int map[3];          // Q, K, J
    // The fast path's plan runs on a side stream beside the forward walls.
    cudaStream_t side;
    cudaEvent_t fork, join;
    // A second plan set (the b fields), built on the side stream while a
    // step's walls and streaming run, for the step the next call is expected
    // to take (the next in the direction of the last two calls, backward at
    // first); pre_step is that step (-1: none), step2 its device counter.
    void *pidx16b, *pa16b;
    int *sc_countb, *sc_cursorb, *sc_metab;
    uint32_t *sc_entb;
    uint4 *lrecb;
    int64_t *step2;
    int64_t pre_step, last_step;
    cudaEvent_t cell_done;
};

// Allocates the scratch and sets up the kernels on the first call.
bz_status bz_adj_prepare(bz_adj_scratch *a, const bzk::Geo &g, int dtype, int nsm, int smem_optin);
// The launches of one adjoint step (see bz_adjoint_step in bz.h).
bz_status bz_adj_launch(bz_adj_scratch *a, const bzk::Geo &g, int dtype, int64_t step,
                        const void *hn, const void *lam_in, void *lam_out, double *grad_lid,
                        double wD, unsigned long long *stats, cudaStream_t s, long long *launches);
void bz_adj_release(bz_adj_scratch *a);
