// bz_adjoint.cu -- host side of bz_adjoint_step: scratch and launch sequence.
//
// One adjoint step recomputes what the forward step n produced and the
// adjoint needs (the wall densities and ghosts of h^n, the sample set of step
// n; h~, h_c and mu per cell inside the cell kernel) and then runs the
// transposed collision, the wall terms and the transposed streaming.
#include "bz.h"
#include "bz_internal.h"
#include "bz_adjoint.cuh"
#include "bz_cell4.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <string>

namespace {

bool alloc_fault()
{
    const char *f = getenv("BZ_FAULT");
    return f && std::string(f) == "alloc";
}

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

// Buffers used by both kernels of the cell phase.
template <typename R>
bz_status alloc_common(bz_adj_scratch *t, const bzk::Geo &g)
{
    const size_t bytes[7] = {sizeof(int4) * (size_t)g.nt,
                             sizeof(bzk::PlanA<R, int>) * (size_t)g.nt,
                             sizeof(R) * (size_t)g.nfaces * g.nv,
                             sizeof(double) * g.nfaces,
                             sizeof(double) * g.nfaces,
                             sizeof(int64_t),
                             sizeof(R) * (size_t)g.nr * g.nvt};
    void **dst[7] = {(void **)&t->pidx, &t->pa, &t->ghost, (void **)&t->nw, (void **)&t->lF,
                     (void **)&t->step, &t->lt};
    for (int k = 0; k < 7; ++k) {
        cudaError_t e = alloc_fault() ? cudaErrorMemoryAllocation : cudaMalloc(dst[k], bytes[k]);
        if (e != cudaSuccess) return cuda_err(e, "adjoint scratch allocation");
    }
    return BZ_OK;
}

// Launch shape of the generic cell kernel (three slabs and the per-sample
// products in shared memory).
template <typename R>
bz_status setup_generic(bz_adj_scratch *a, const bzk::Geo &g, int nsm, int optin)
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
    // The limit is a property of the kernel, shared by every handle: set it to
    // the device maximum so that no handle lowers it below another's need.
    cudaError_t e = bz_allow_max_smem(bzk::k_adj_cell<R>, optin);
    if (e != cudaSuccess) return cuda_err(e, "cudaFuncSetAttribute");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bzk::k_adj_cell<R>, threads, smem);
    if (e != cudaSuccess) return cuda_err(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (occ < 1) return err(BZ_EUNSUPPORTED, "adjoint cell kernel cannot be resident");
    a->threads = threads;
    a->smem = smem;
    a->grid = std::min(g.nr, nsm * occ);
    return BZ_OK;
}

// The FP32 quad kernel applies when the forward fast path's conditions hold
// (velocity axis a multiple of 4, 16-bit node indices, 15-bit sample
// indices) and the two extra slabs fit in shared memory.
bz_status prepare_fast(bz_adj_scratch *a, const bzk::Geo &g, int nsm, int optin)
{
    const int N = g.nv, Q = N * N / 4;
    const char *force = getenv("BZ_KERNEL");
    if (force && std::string(force) == "generic") return BZ_OK;
    if (N % 4 != 0 || N < 12 || g.nvt >= 65535 || g.nt > 32768 || Q > 1024) return BZ_OK;
    const size_t smem = bzk::adj4_smem_bytes(N, g.nvt, g.nt);
    if (smem > (size_t)optin) return BZ_OK;
    // Two CTAs of up to 512 threads per SM when their shared memory fits, so
    // that one CTA's serial sections (the 5x5 solves) overlap the other's work.
    int smem_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int maxt = (int)smem <= smem_sm / 2 - 1024 && Q <= 512 ? 512 : 1024;
    int K = 1;
    for (int k = 1; k <= N; ++k)
        if (N % k == 0 && Q * k <= maxt) K = k;
    const int T = (Q * K + 31) / 32 * 32;
    cudaError_t e = maxt == 512 ? bz_allow_max_smem(bzk::k_adj_cell4<512>, optin)
                                : bz_allow_max_smem(bzk::k_adj_cell4<1024>, optin);
    if (e != cudaSuccess) return cuda_err(e, "cudaFuncSetAttribute");
    int occ = 0;
    e = maxt == 512
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bzk::k_adj_cell4<512>, T, smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bzk::k_adj_cell4<1024>, T, smem);
    if (e != cudaSuccess) return cuda_err(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (occ < 1) return BZ_OK;
    const size_t bytes[7] = {sizeof(ushort4) * (size_t)g.nt,
                             sizeof(bzk::PlanA<float, uint16_t>) * (size_t)g.nt,
                             sizeof(int) * 2 * (size_t)g.nvt,
                             sizeof(int) * 2 * (size_t)g.nvt,
                             sizeof(int) * 4,
                             sizeof(uint32_t) * ((size_t)4 * g.nt + bzk::kMaxThreads),
                             sizeof(uint4) * ((size_t)2 * g.nt + bzk::kMaxThreads)};
    void **dst[7] = {&a->pidx16, &a->pa16, (void **)&a->sc_count, (void **)&a->sc_cursor,
                     (void **)&a->sc_meta, (void **)&a->sc_ent, (void **)&a->lrec};
    void **dstb[7] = {&a->pidx16b, &a->pa16b, (void **)&a->sc_countb, (void **)&a->sc_cursorb,
                      (void **)&a->sc_metab, (void **)&a->sc_entb, (void **)&a->lrecb};
    for (int k = 0; k < 7; ++k) {
        e = alloc_fault() ? cudaErrorMemoryAllocation : cudaMalloc(dst[k], bytes[k]);
        if (e == cudaSuccess) e = cudaMalloc(dstb[k], bytes[k]);
        if (e != cudaSuccess) return cuda_err(e, "adjoint scratch allocation");
    }
    e = cudaMalloc(&a->step2, sizeof(int64_t));
    if (e != cudaSuccess) return cuda_err(e, "adjoint scratch allocation");
    a->pre_step = a->last_step = -1;
    a->fast = true;
    a->threads = T;
    a->smem = smem;
    a->grid = std::min(g.nr, nsm * occ);
    a->map[0] = Q;
    a->map[1] = K;
    a->map[2] = N / K;
    return BZ_OK;
}

// The fast path's plan of the step in *stepp into one plan set, on stream sp:
// the 16-bit plan in the shared-memory order and the destination-sorted
// forward and loss lists, as the forward step builds them (64-thread blocks
// spread the FP64 sampling over every SM).
cudaError_t fast_plan(const bzk::Geo &g, const int64_t *stepp, int threads, void *pidx16, void *pa16,
                      int *sc_count, int *sc_cursor, int *sc_meta, uint32_t *sc_ent, uint4 *lrec,
                      cudaStream_t sp, int *n)
{
    bzk::Geo gs = g;
    gs.swz = 1;
    const int pb = 256, pg = (g.nt + pb - 1) / pb;
    const ushort4 *pi = (const ushort4 *)pidx16;
    bzk::k_plan<float, uint16_t><<<(g.nt + 63) / 64, 64, 0, sp>>>(
        gs, stepp, (ushort4 *)pidx16, (bzk::PlanA<float, uint16_t> *)pa16, nullptr, nullptr);
    ++*n;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(sc_count, 0, sizeof(int) * 2 * g.nvt, sp);
    if (e != cudaSuccess) return e;
    bzk::k_adj_count2<<<pg, pb, 0, sp>>>(g.nt, g.nvt, pi, sc_count);
    bzk::k_adj_scan2<<<2, 1024, 0, sp>>>(g.nvt, threads, sc_count, sc_cursor, sc_meta);
    bzk::k_adj_fill2<<<pg, pb, 0, sp>>>(g.nt, g.nvt, threads, pi, (const bzk::PlanA<float, uint16_t> *)pa16,
                                        sc_cursor, sc_meta, sc_ent, lrec);
    *n += 3;
    return cudaGetLastError();
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
    const int pb = 256, pg = (g.nt + pb - 1) / pb;
    bool fast = false;
    if constexpr (sizeof(R) == 4) fast = a->fast;
    // The fast path's plan depends on the step only: it runs on the side
    // stream while the walls run (after everything before it on s), unless
    // the previous call already built it there (then s waits for that).
    const cudaStream_t sp = fast ? a->side : s;
    if (fast && a->pre_step == step) {
        std::swap(a->pidx16, a->pidx16b);
        std::swap(a->pa16, a->pa16b);
        std::swap(a->sc_count, a->sc_countb);
        std::swap(a->sc_cursor, a->sc_cursorb);
        std::swap(a->sc_meta, a->sc_metab);
        std::swap(a->sc_ent, a->sc_entb);
        std::swap(a->lrec, a->lrecb);
    } else if (fast) {
        if (e == cudaSuccess) e = cudaEventRecord(a->fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sp, a->fork, 0);
        if (e == cudaSuccess)
            e = fast_plan(g, a->step, a->threads, a->pidx16, a->pa16, a->sc_count, a->sc_cursor, a->sc_meta,
                          a->sc_ent, a->lrec, sp, &n);
        if (e == cudaSuccess) e = cudaEventRecord(a->join, sp);
    }
    // Forward quantities of step n: wall densities and ghosts of h^n.
    if (e == cudaSuccess) {
        bzk::k_walls<R><<<g.nfaces, bzk::kWallThreads, 0, s>>>(g, a->step, hn, (R *)a->ghost, a->nw, nullptr);
        e = check();
    }
    if (fast && e == cudaSuccess) e = cudaStreamWaitEvent(s, a->join, 0);
    if (fast) {
        const ushort4 *pi = (const ushort4 *)a->pidx16;
        bzk::Geo gs = g;
        gs.swz = 1;
        if (e == cudaSuccess) {
            const bzk::Map4 m{a->map[0], a->map[1], a->map[2]};
            if (a->threads <= 512)
                bzk::k_adj_cell4<512><<<a->grid, a->threads, a->smem, s>>>(
                    gs, m, (const float *)hn, (const float *)a->ghost, pi,
                    (const bzk::PlanA<float, uint16_t> *)a->pa16, a->sc_ent, a->sc_meta, a->lrec,
                    a->sc_meta + 2, (const float *)lam_in, (float *)a->lt, stats);
            else
                bzk::k_adj_cell4<1024><<<a->grid, a->threads, a->smem, s>>>(
                    gs, m, (const float *)hn, (const float *)a->ghost, pi,
                    (const bzk::PlanA<float, uint16_t> *)a->pa16, a->sc_ent, a->sc_meta, a->lrec,
                    a->sc_meta + 2, (const float *)lam_in, (float *)a->lt, stats);
            e = check();
        }
        // The plan of the step the next call is expected to take, into the
        // other set, on the side stream once this step's cell kernel is done
        // with its plan (it runs beside this step's walls and streaming).
        const int64_t dir = a->last_step >= 0 && a->last_step != step ? (step > a->last_step ? 1 : -1) : -1;
        const int64_t guess = step + dir;
        a->last_step = step;
        a->pre_step = -1;
        if (guess >= 0 && e == cudaSuccess) {
            e = cudaEventRecord(a->cell_done, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(sp, a->cell_done, 0);
            if (e == cudaSuccess) {
                bzk::k_set_step<<<1, 1, 0, sp>>>(a->step2, guess);
                e = check();
            }
            if (e == cudaSuccess)
                e = fast_plan(g, a->step2, a->threads, a->pidx16b, a->pa16b, a->sc_countb, a->sc_cursorb,
                              a->sc_metab, a->sc_entb, a->lrecb, sp, &n);
            if (e == cudaSuccess) e = cudaEventRecord(a->join, sp);
            if (e == cudaSuccess) a->pre_step = guess;
        }
    } else {
        if (e == cudaSuccess) {
            bzk::k_plan<R, int><<<(g.nt + 63) / 64, 64, 0, s>>>(g, a->step, a->pidx,
                                                                (bzk::PlanA<R, int> *)a->pa, nullptr, nullptr);
            e = check();
        }
        if (e == cudaSuccess) {
            bzk::k_adj_cell<R><<<a->grid, a->threads, a->smem, s>>>(
                g, hn, (const R *)a->ghost, a->pidx, (const bzk::PlanA<R, int> *)a->pa, lam_in,
                (R *)a->lt, stats);
            e = check();
        }
    }
    if (e == cudaSuccess) {
        bzk::k_adj_walls<R><<<g.nfaces, bzk::kWallThreads, 0, s>>>(g, a->step, (const R *)a->lt, a->nw, a->lF,
                                                     grad_lid, wD);
        e = check();
    }
    if (e == cudaSuccess) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (fast) {
            const int Q = g.nv * g.nv / 4;
            const int blk = Q * std::max(1, 512 / Q);
            const int grid = std::min(g.nr, nsm * std::max(1, 2048 / blk));
            bzk::k_adj_stream4<<<grid, blk, 0, s>>>(g, (const float *)a->lt, a->lF,
                                                     (float *)lam_out, wD);
        } else {
            const int grid = std::min(g.nr, nsm * 8);
            bzk::k_adj_stream<R><<<grid, 256, 0, s>>>(g, (const R *)a->lt, a->lF, lam_out, wD);
        }
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
    bz_adj_scratch t{};
    bz_status st = dtype == BZ_F64 ? alloc_common<double>(&t, g) : alloc_common<float>(&t, g);
    if (st == BZ_OK && dtype == BZ_F32) st = prepare_fast(&t, g, nsm, optin);
    if (st == BZ_OK && !t.fast)
        st = dtype == BZ_F64 ? setup_generic<double>(&t, g, nsm, optin)
                             : setup_generic<float>(&t, g, nsm, optin);
    if (st == BZ_OK && t.fast) {
        // A chain of small latency-bound kernels: highest priority.
        int least = 0, greatest = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&t.side, cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t.join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t.cell_done, cudaEventDisableTiming);
        if (e != cudaSuccess) st = cuda_err(e, "adjoint side stream");
    }
    if (st != BZ_OK) {
        bz_adj_release(&t);
        return st;
    }
    *a = t;
    return BZ_OK;
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
    void *ptrs[] = {a->pidx, a->pa, a->ghost, a->lt, a->nw, a->lF, a->step,
                    a->pidx16, a->pa16, a->sc_count, a->sc_cursor, a->sc_meta, a->sc_ent,
                    a->lrec, a->pidx16b, a->pa16b, a->sc_countb, a->sc_cursorb, a->sc_metab,
                    a->sc_entb, a->lrecb, a->step2};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (a->side) cudaStreamDestroy(a->side);
    if (a->fork) cudaEventDestroy(a->fork);
    if (a->join) cudaEventDestroy(a->join);
    if (a->cell_done) cudaEventDestroy(a->cell_done);
    *a = bz_adj_scratch{};
}
