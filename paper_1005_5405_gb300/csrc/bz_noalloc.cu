// bz_noalloc.cu -- a collision step that allocates no device memory.
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// owned entirely by their own pool allocator and that forbid run-time
// allocation, and latency-critical loops in which cudaMalloc/cudaFree would
// synchronise the device.  bz_collide_noalloc serves them: the caller passes
// the input and output states, and the only scratch the step needs (the Monte
// Carlo sample set of the step and the per-axis velocity tables) lives in the
// file-scope device array below, which every GPU that loads the library keeps
// until the process exits.
#include "bz.h"
#include "bz_internal.h"
#include "bz_kernels.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace {

constexpr int kNoallocMaxPairs = BZ_NOALLOC_MAX_PAIRS;
constexpr int kNoallocMaxDevices = 64;
// Scratch layout: sample node indices (int4), gather records (16 bytes each),
// per-axis velocity nodes and weights (kMaxN doubles each), the step number.
constexpr size_t kIdxBytes = sizeof(int4) * (size_t)kNoallocMaxPairs;
constexpr size_t kRecBytes = 16 * (size_t)kNoallocMaxPairs;
constexpr size_t kTabBytes = sizeof(double) * bzk::kMaxN;
constexpr size_t kScratchBytes = kIdxBytes + kRecBytes + 2 * kTabBytes + sizeof(int64_t);
static_assert(kScratchBytes <= BZ_NOALLOC_SCRATCH_BYTES, "scratch size");

// Shared by every call on a device; its contents are those of the last call.
static __device__ __align__(256) unsigned char bz_noalloc_scratch[BZ_NOALLOC_SCRATCH_BYTES];

// Per-axis velocity nodes and weight factors and the step number, passed to
// the set-up kernel by value.
struct NoallocTables {
    double axv[bzk::kMaxN], axA[bzk::kMaxN];
    int64_t step;
};

// Writes the tables into the scratch (one block of kMaxN threads).
__global__ void k_noalloc_tables(NoallocTables t, int n, double *axv, double *axA, int64_t *step)
{
    const int i = threadIdx.x;
    if (i < n) {
        axv[i] = t.axv[i];
        axA[i] = t.axA[i];
    }
    if (i == 0) *step = t.step;
}

std::mutex g_mutex;
void *g_scratch[kNoallocMaxDevices] = {};

bz_status err(bz_status st, const char *fmt, ...)
{
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    bz_record_error(buf);
    return st;
}

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
bz_status scratch_address(int dev, unsigned char **out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (dev < 0 || dev >= kNoallocMaxDevices) return err(BZ_EINVAL, "device %d out of range", dev);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, bz_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return err(BZ_ECUDA, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        g_scratch[dev] = p;
    }
    *out = (unsigned char *)g_scratch[dev];
    return BZ_OK;
}

template <typename R>
bz_status run(const bzk::Geo &g0, unsigned char *scr, const void *hin, void *hout, double *mom,
              cudaStream_t s)
{
    bzk::Geo g = g0;
    int4 *pidx = (int4 *)scr;
    bzk::PlanA<R, int> *pa = (bzk::PlanA<R, int> *)(scr + kIdxBytes);
    double *axv = (double *)(scr + kIdxBytes + kRecBytes);
    double *axA = axv + bzk::kMaxN;
    const int64_t *stepp = (const int64_t *)(axA + bzk::kMaxN);
    g.axv = axv;
    g.axA = axA;
    int dev = 0, nsm = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t smem = bzk::cell_smem_bytes<R>(g.nv, g.nvt, g.nt, true);
    if (smem > (size_t)optin)
        return err(BZ_EUNSUPPORTED,
                   "the velocity slab and the %d per-sample products need %zu bytes of shared "
                   "memory; the device offers %d", g.nt, smem, optin);
    const int threads = std::min(bzk::kMaxThreads, (g.nv * g.nv + 31) / 32 * 32);
    cudaError_t e = bz_allow_max_smem(bzk::k_cell<R, false, int>, optin);
    int occ = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bzk::k_cell<R, false, int>,
                                                          threads, smem);
    if (e != cudaSuccess) return err(BZ_ECUDA, "kernel set-up failed: %s", cudaGetErrorString(e));
    if (occ < 1) return err(BZ_EUNSUPPORTED, "collision kernel cannot be resident");
    const int grid = std::min(g.nr, nsm * occ);
    const int pb = 256, pg = (g.nt + pb - 1) / pb;
    bzk::k_plan<R, int><<<pg, pb, 0, s>>>(g, stepp, pidx, pa, nullptr, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return err(BZ_ECUDA, "sampling launch failed: %s", cudaGetErrorString(e));
    bzk::k_cell<R, false, int><<<grid, threads, smem, s>>>(g, (const R *)hin, nullptr, pidx,
                                                           pa, nullptr, (R *)hout, mom, nullptr, 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return err(BZ_ECUDA, "collision launch failed: %s", cudaGetErrorString(e));
    return BZ_OK;
}

}  // namespace

extern "C" bz_status bz_collide_noalloc(const bz_space *space, const bz_vel *vel,
                                        const bz_params *params, int64_t step, const void *h_in,
                                        void *h_out, double *mom, void *stream)
{
    bz_record_error("");
    if (!space || !vel || !params || !h_in || !h_out) return err(BZ_EINVAL, "NULL argument");
    if (space->nx < 1 || space->ny < 1 || (int64_t)space->nx * space->ny > (1 << 30))
        return err(BZ_EINVAL, "invalid spatial grid");
    if (!(space->kn > 0.0) || !std::isfinite(space->kn)) return err(BZ_EINVAL, "kn must be > 0");
    if (vel->nv < 2 || vel->nv > bzk::kMaxN) return err(BZ_EINVAL, "nv must be in [2, %d]", bzk::kMaxN);
    if (!(vel->vmax > 0.0) || !std::isfinite(vel->vmax)) return err(BZ_EINVAL, "vmax must be > 0");
    if (params->n_pairs < 1 || params->n_pairs > kNoallocMaxPairs)
        return err(BZ_EINVAL, "n_pairs must be in [1, %d] (size of the static scratch)",
                   kNoallocMaxPairs);
    if (!(params->eps > 0.0) || !std::isfinite(params->eps))
        return err(BZ_EINVAL, "eps must be given (> 0): there is no lid to derive it from");
    if (!(params->cfl >= 0.0 && params->cfl <= 1.0)) return err(BZ_EINVAL, "cfl must be in [0, 1]");
    if (!(params->kcoll >= 0.0) || !std::isfinite(params->kcoll))
        return err(BZ_EINVAL, "kcoll must be >= 0");
    if (params->dtype != BZ_F32 && params->dtype != BZ_F64) return err(BZ_EINVAL, "dtype");
    if (params->sample_mode != BZ_SHARED)
        return err(BZ_EUNSUPPORTED, "only the shared sample set is implemented");
    if ((vel->rv > 0.0 && vel->rv < 1.0) || (space->rx > 0.0 && space->rx < 1.0) ||
        (space->ry > 0.0 && space->ry < 1.0))
        return err(BZ_EUNSUPPORTED, "uniform grids only");
    if (step < 0) return err(BZ_EINVAL, "step must be >= 0");

    // Discretisation: the same rules, in the same code, as bz_create.
    bzk::Geo g{};
    bz_grid_tables tb;
    bz_discretise(space, vel, nullptr, params, g, tb);
    const int N = vel->nv;
    const size_t esz = params->dtype == BZ_F64 ? 8 : 4;
    const size_t bytes = esz * (size_t)g.nr * (size_t)g.nvt;
    const uintptr_t a0 = (uintptr_t)h_in, b0 = (uintptr_t)h_out;
    if (a0 < b0 + bytes && b0 < a0 + bytes) return err(BZ_EINVAL, "h_in and h_out must not overlap");
    // The tables travel as a kernel argument (copied at launch), not through
    // a host buffer.
    NoallocTables tabs{};
    for (int j = 0; j < N; ++j) {
        tabs.axv[j] = tb.axv[j];
        tabs.axA[j] = tb.axA[j];
    }
    tabs.step = step;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(BZ_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    unsigned char *scr = nullptr;
    bz_status st = scratch_address(dev, &scr);
    if (st != BZ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double *axv = (double *)(scr + kIdxBytes + kRecBytes);
    k_noalloc_tables<<<1, bzk::kMaxN, 0, s>>>(tabs, N, axv, axv + bzk::kMaxN,
                                              (int64_t *)(axv + 2 * bzk::kMaxN));
    e = cudaGetLastError();
    if (e != cudaSuccess) return err(BZ_ECUDA, "table set-up launch failed: %s", cudaGetErrorString(e));
    return params->dtype == BZ_F64 ? run<double>(g, scr, h_in, h_out, mom, s)
                                   : run<float>(g, scr, h_in, h_out, mom, s);
}
