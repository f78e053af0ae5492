// bz_adjoint.cu -- host side of bz_adjoint_step: scratch and launch sequence.
//
// One adjoint step recomputes what the forward step n produced and the
// adjoint needs (the wall densities and ghosts of h^n, the sample set of step
// n; h~, h_c and mu per cell inside the cell kernel) and then runs the
// transposed collision, the wall terms and the transposed streaming.
#include "bz.h"
#include "bz_internal.h"
#include "bz_adjoint.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <string>

namespace {

bz_status err(bz_status st, const char *msg)
{
    bz_record_error(msg);
    return st;
}

bz_status cuda_err(cudaError_t e, const char *what)
{
    char buf[300];
    snprintf(buf, sizeof(buf), "%s failed: %s", what, cudaGetErrorString(e));
    bz_record_error(buf);
    return e == cudaErrorMemoryAllocation ? BZ_ENOMEM : BZ_ECUDA;
}

template <typename R>
bz_status prepare(bz_adj_scratch *a, const bzk::Geo &g, int nsm, int optin)
{
    const int n2 = g.nv * g.nv;
    const int threads = std::min(bzk::kMaxThreads, (n2 + 31) / 32 * 32);
    const size_t smem = bzk::adj_smem_bytes<R>(g.nv, g.nvt, g.nt);
    if (smem > (size_t)optin) {
        char buf[300];
        snprintf(buf, sizeof(buf),
                 "the adjoint keeps three velocity slabs and %d per-sample products in shared "
                 "memory: %zu bytes, the device offers %d", g.nt, smem, optin);
        return err(BZ_EUNSUPPORTED, buf);
    }
    cudaError_t e = cudaFuncSetAttribute(bzk::k_adj_cell<R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_err(e, "cudaFuncSetAttribute");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bzk::k_adj_cell<R>, threads, smem);
    if (e != cudaSuccess) return cuda_err(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (occ < 1) return err(BZ_EUNSUPPORTED, "adjoint cell kernel cannot be resident");
    bz_adj_scratch t{};
    t.threads = threads;
    t.smem = smem;
    t.grid = std::min(g.nr, nsm * occ);
    const size_t bytes[7] = {sizeof(int4) * (size_t)g.nt,
                             sizeof(bzk::PlanA<R, int>) * (size_t)g.nt,
                             sizeof(R) * (size_t)g.nfaces * g.nv,
                             sizeof(double) * g.nfaces,
                             sizeof(double) * g.nfaces,
                             sizeof(int64_t),
                             sizeof(R) * (size_t)g.nr * g.nvt};
    void **dst[7] = {(void **)&t.pidx, &t.pa, &t.ghost, (void **)&t.nw, (void **)&t.lF,
                     (void **)&t.step, &t.lt};
    for (int k = 0; k < 7; ++k) {
        e = getenv("BZ_FAULT") && std::string(getenv("BZ_FAULT")) == "alloc"
                ? cudaErrorMemoryAllocation
                : cudaMalloc(dst[k], bytes[k]);
        if (e != cudaSuccess) {
            for (int m = 0; m < k; ++m) cudaFree(*dst[m]);
            return cuda_err(e, "adjoint scratch allocation");
        }
    }
    *a = t;
    return BZ_OK;
}

template <typename R>
bz_status launch(bz_adj_scratch *a, const bzk::Geo &g0, int64_t step, const R *hn,
                 const R *lam_in, R *lam_out, double *grad_lid, double wD,
                 unsigned long long *stats, cudaStream_t s, long long *launches)
{
    bzk::Geo g = g0;
    g.swz = 0;                                   // logical node order
    int n = 0;
    auto check = [&]() {
        ++n;
        return cudaGetLastError();
    };
    bzk::k_set_step<<<1, 1, 0, s>>>(a->step, step);
    cudaError_t e = check();
    // Forward quantities of step n: wall densities and ghosts of h^n, the samples.
    if (e == cudaSuccess) {
        bzk::k_walls<R><<<g.nfaces, 256, 0, s>>>(g, a->step, hn, (R *)a->ghost, a->nw, nullptr);
        e = check();
    }
    if (e == cudaSuccess) {
        const int pb = 256, pg = (g.nt + pb - 1) / pb;
        bzk::k_plan<R, int><<<pg, pb, 0, s>>>(g, a->step, a->pidx, (bzk::PlanA<R, int> *)a->pa,
                                              nullptr, nullptr);
        e = check();
    }
    if (e == cudaSuccess) {
        bzk::k_adj_cell<R><<<a->grid, a->threads, a->smem, s>>>(
            g, hn, (const R *)a->ghost, a->pidx, (const bzk::PlanA<R, int> *)a->pa, lam_in,
            (R *)a->lt, stats);
        e = check();
    }
    if (e == cudaSuccess) {
        bzk::k_adj_walls<R><<<g.nfaces, 256, 0, s>>>(g, a->step, (const R *)a->lt, a->nw, a->lF,
                                                     grad_lid, wD);
        e = check();
    }
    if (e == cudaSuccess) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int grid = std::min(g.nr, nsm * 8);
        bzk::k_adj_stream<R><<<grid, 256, 0, s>>>(g, (const R *)a->lt, a->lF, lam_out, wD);
        e = check();
    }
    if (launches) *launches += n;
    if (e != cudaSuccess) return cuda_err(e, "adjoint kernel launch");
    return BZ_OK;
}

}  // namespace

bz_status bz_adj_prepare(bz_adj_scratch *a, const bzk::Geo &g, int dtype, int nsm, int optin)
{
    if (a->lt) return BZ_OK;
    return dtype == BZ_F64 ? prepare<double>(a, g, nsm, optin) : prepare<float>(a, g, nsm, optin);
}

bz_status bz_adj_launch(bz_adj_scratch *a, const bzk::Geo &g, int dtype, int64_t step,
                        const void *hn, const void *lam_in, void *lam_out, double *grad_lid,
                        double wD, unsigned long long *stats, cudaStream_t s, long long *launches)
{
    if (dtype == BZ_F64)
        return launch<double>(a, g, step, (const double *)hn, (const double *)lam_in,
                              (double *)lam_out, grad_lid, wD, stats, s, launches);
    return launch<float>(a, g, step, (const float *)hn, (const float *)lam_in, (float *)lam_out,
                         grad_lid, wD, stats, s, launches);
}

void bz_adj_release(bz_adj_scratch *a)
{
    void *ptrs[] = {a->pidx, a->pa, a->ghost, a->lt, a->nw, a->lF, a->step};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    *a = bz_adj_scratch{};
}
