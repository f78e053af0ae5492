// bz_api.cu -- host side of the C ABI declared in include/bz.h.
//
// Owns device memory, derives the discretisation of the paper's problem
// statement (Sec. 3, Sec. 5.1), and sequences the kernels of one time step on
// the caller's stream.  No host computation is on the step path: the host only
// validates arguments, builds per-axis tables once at creation and launches.
#include "bz.h"
#include "bz_internal.h"
#include "bz_kernels.cuh"
#include "bz_cell4.cuh"
#include "bz_batch.cuh"
#include "bz_lazy.cuh"
#include "bz_ahead.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using bzk::Geo;

namespace {

thread_local std::string g_last_error;

bz_status fail(bz_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define BZ_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(e_ == cudaErrorMemoryAllocation ? BZ_ENOMEM : BZ_ECUDA,        \
                        "%s failed: %s", #call, cudaGetErrorString(e_));               \
    } while (0)

#define BZ_LAUNCHED(hd)                                                                \
    do {                                                                               \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess)                                                         \
            return fail(BZ_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e_)); \
        (hd)->launches++;                                                              \
    } while (0)

bool fault_injected(const char *what)
{
    const char *f = getenv("BZ_FAULT");
    return f && strcmp(f, what) == 0;
}

}  // namespace

void bz_record_error(const char *msg) { g_last_error = msg; }

struct bz_handle {
    Geo g{};
    int dtype = BZ_F32;
    size_t esz = 4;
    void *h[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t step = 0;                   // host mirror of the device step counter
    int64_t *d_step = nullptr;          // device step counter read by the kernels
    cudaStream_t cap_stream = nullptr;  // stream used to capture step graphs
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // two fused steps, by buffer parity
    long long graph_launches = 0;
    // Profiled graphs: the event record nodes of each timed launch (kernel
    // class k), found in the graph they were captured into (kept for that),
    // which get fresh events before every replay.
    struct ProfNode {
        int k;
        cudaGraphNode_t a, b;
    };
    cudaGraph_t gtmpl[2] = {nullptr, nullptr};
    std::vector<ProfNode> gprof[2];
    std::vector<cudaEvent_t> gplace;    // the events recorded while capturing
    bool capturing = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> cap_ev;
    void *ht = nullptr;                 // h~ for the unfused path (lazy)
    void *pidx = nullptr;               // sample plan: node indices (16- or 32-bit)
    bool idx16 = true;
    void *pa = nullptr;                 // sample plan: (a, b, W) records of the gather phase
    void *ghost = nullptr;              // emitted ghost values per face
    double *nw = nullptr;               // wall densities per face
    double *shear = nullptr;            // lid face shear (nx)
    double *mom = nullptr;              // nr * 11
    bool mom_valid = false;
    void *gw_global = nullptr;          // per-CTA product scratch when it does not fit smem
    int gw_in_smem = 1;
    unsigned long long *stats = nullptr;
    int *flag = nullptr;
    double *axv = nullptr, *axA = nullptr, *profile = nullptr;
    std::vector<double> host_profile;
    int dev = 0, nsm = 0, smem_optin = 0;
    int threads = 0, grid_cell = 0, grid_cell_fused = 0;
    size_t smem_cell = 0;
    long long launches = 0;
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[4];
    // FP32 fast path (bz_cell4.cuh)
    bool fast = false;
    long long *prof_clk = nullptr;      // phase trace of the per-cell kernel (bz_profile level 2)
    bzk::Map4 map{};
    int threads4 = 0, grid4f = 0, grid4c = 0, maxt4 = 1024;
    size_t smem4 = 0;
    int *sc_count = nullptr, *sc_cursor = nullptr, *sc_meta = nullptr;  // scatter-list sort
    uint32_t *sc_ent = nullptr;
    bz_adj_scratch adj{};               // bz_adjoint_step scratch, allocated on first use
    // Active-node path with deferred correction (bz_lazy.cuh).  A buffer with
    // lazy_buf set holds h_c and its cells' pending corrections in mu[buf];
    // mu[buf] is all zero whenever lazy_buf is clear.
    bool per_cell = false;              // every cell draws its own sample set
    bool stretched = false;             // non-uniform velocity or spatial cells
    double *axe = nullptr, *axd = nullptr, *wlid = nullptr;
    double *sx = nullptr, *sy = nullptr;
    bool lazy = false;
    float *mu[2] = {nullptr, nullptr};
    bool lazy_buf[2] = {false, false};
    int4 *lz_idx = nullptr;
    bzk::PlanA<float, int> *lz_pa = nullptr;
    ushort4 *lz_qc = nullptr;
    int *lz_flag = nullptr, *lz_cidx = nullptr, *lz_act = nullptr, *lz_wpre = nullptr;
    int *lz_meta = nullptr, *lz_count = nullptr, *lz_cursor = nullptr, *lz_rowend = nullptr;
    int *lz_dest0 = nullptr;
    uint32_t *lz_mask = nullptr;
    uint2 *lz_rec = nullptr;
    int lz_mcap = 0, lz_G = 0, lz_T = 0, lz_grid = 0, lz_mprobe = 0;
    int lz_cmax = 0, lz_order_tpb = 0;     // bank-aware ordering of the term runs (1: on)
    bool lz_tma = false;                   // streaming sources by bulk copies (G = 4 only)
    // Plans built ahead (bz_ahead.cuh): K slots, covering steps [ahead_lo, ahead_hi).
    int ahead_K = 0;
    bzk::AheadPlans ahead{};
    int64_t ahead_lo = 0, ahead_hi = 0;
    int ahead_chunk = 0;                   // positions per chunk of their term order
    int lz_chunk = 0;                      // positions per chunk of the ordering
    cudaStream_t lz_side = nullptr;        // the sample plan runs here, beside the walls
    cudaEvent_t lz_fork = nullptr, lz_join = nullptr, lz_mid = nullptr;
    size_t lz_smem = 0;
    float lz_e0[bzk::kLzX] = {};
};

namespace {

template <typename T>
bz_status dalloc(T **p, size_t bytes)
{
    if (fault_injected("alloc"))
        return fail(BZ_ENOMEM, "device allocation of %zu bytes failed (BZ_FAULT=alloc)", bytes);
    cudaError_t e = cudaMalloc((void **)p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? BZ_ENOMEM : BZ_ECUDA,
                    "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    return BZ_OK;
}

#define BZ_TRY(x)                          \
    do {                                   \
        bz_status s_ = (x);                \
        if (s_ != BZ_OK) return s_;        \
    } while (0)

double lid_eps(double u0, double amp, const double *profile, int nx)
{
    double m = std::fabs(u0);
    if (profile) {
        m = 0.0;
        for (int i = 0; i < nx; ++i) m = std::max(m, std::fabs(profile[i]));
    }
    m += std::fabs(amp);
    return m > 0.0 ? m : 1.0;
}

// Event pair around one launch of kernel class k when profiling is enabled.
struct ProfScope {
    bz_handle *H;
    int k;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    // While a step graph is captured only the per-cell kernel (class 2) is
    // timed: every event node costs the replayed step a little time.
    ProfScope(bz_handle *H_, int k_, cudaStream_t s_) : H(H_), k(k_), s(s_)
    {
        if (H->prof && (!H->capturing || k == 2) && cudaEventCreate(&a) == cudaSuccess &&
            cudaEventCreate(&b) == cudaSuccess)
            cudaEventRecordWithFlags(a, s, H->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
    }
    ~ProfScope()
    {
        if (a && b) {
            cudaEventRecordWithFlags(b, s, H->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
            if (H->capturing) H->cap_ev.push_back({k, {a, b}});
            else H->ev[k].push_back({a, b});
        }
    }
};

// End of a full step: the device step counter moves on (and its host mirror).
bz_status advance(bz_handle *H, cudaStream_t s)
{
    bzk::k_advance<<<1, 1, 0, s>>>(H->d_step);
    BZ_LAUNCHED(H);
    H->step++;
    return BZ_OK;
}

void drop_graphs(bz_handle *H)
{
    for (auto &g : H->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    for (int p = 0; p < 2; ++p) {
        if (H->gtmpl[p]) cudaGraphDestroy(H->gtmpl[p]);
        H->gtmpl[p] = nullptr;
        H->gprof[p].clear();
    }
    for (cudaEvent_t e : H->gplace) cudaEventDestroy(e);
    H->gplace.clear();
}

// Launch the FP32 fast-path cell kernel; false when the handle does not use it.
template <typename R>
bool launch_cell4(bz_handle *H, cudaStream_t s, bool fused, const R *hin, R *hout)
{
    if constexpr (sizeof(R) != 4) {
        return false;
    } else {
        if (!H->fast) return false;
        const Geo &g = H->g;
        const float *gh = (const float *)H->ghost;
        const ushort4 *pi = (const ushort4 *)H->pidx;
        const bzk::PlanA<float, uint16_t> *pa = (const bzk::PlanA<float, uint16_t> *)H->pa;
        // Destination-sorted scatter list of this step's sample set.
        {
            ProfScope ps1(H, 1, s);
            const int pb = 256, pg = (g.nt + pb - 1) / pb;
            if (cudaMemsetAsync(H->sc_count, 0, sizeof(int) * g.nvt, s) != cudaSuccess) return true;
            bzk::k_scatter_count<<<pg, pb, 0, s>>>(g.nt, pi, H->sc_count);
            bzk::k_scatter_scan<<<1, 1024, 0, s>>>(g.nvt, H->threads4, H->sc_count, H->sc_cursor,
                                                   H->sc_meta);
            bzk::k_scatter_fill<<<pg, pb, 0, s>>>(g.nt, H->threads4, pi, H->sc_cursor, H->sc_meta,
                                                  H->sc_ent);
            H->launches += 3;
        }
        ProfScope ps(H, 2, s);
        const int grid = fused ? H->grid4f : H->grid4c;
#define BZ_C4(F, M)                                                                           \
    bzk::k_cell4<F, M><<<grid, H->threads4, H->smem4, s>>>(g, H->map, hin, gh, pa, H->sc_ent, \
                                                          H->sc_meta, hout, H->mom, H->stats,   \
                                                          H->prof_clk)
        if (H->maxt4 == 512) {
            if (fused) BZ_C4(true, 512); else BZ_C4(false, 512);
        } else {
            if (fused) BZ_C4(true, 1024); else BZ_C4(false, 1024);
        }
#undef BZ_C4
        return true;
    }
}

template <bool F, int M>
bz_status setup_cell4_kernel(bz_handle *H, int *occ)
{
    // Kernel attributes are shared by every handle in the process: the limit
    // is set to the device maximum so that no handle lowers it for another.
    BZ_CUDA(bz_allow_max_smem(bzk::k_cell4<F, M>, H->smem_optin));
    BZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, bzk::k_cell4<F, M>, H->threads4,
                                                          H->smem4));
    return BZ_OK;
}

// Decide whether the FP32 fast path applies and size its launch.
bz_status configure_cell4(bz_handle *H)
{
    const Geo &g = H->g;
    const int N = g.nv;
    const char *force = getenv("BZ_KERNEL");
    H->fast = false;
    if (force && strcmp(force, "generic") == 0) return BZ_OK;
    if (H->per_cell) return BZ_OK;         // the shared-set kernels only
    if (H->dtype != BZ_F32 || !H->idx16 || N % 4 != 0 || N < 12) return BZ_OK;
    if (g.nt > 32768) return BZ_OK;                 // 15-bit sample index in the scatter list
    if (bzk::cell4_smem_bytes(N, g.nvt, g.nt) > (size_t)H->smem_optin) return BZ_OK;
    // Threads per CTA: up to 1024 (64 registers each) or, with
    // BZ_CELL_THREADS=512, up to 512 with twice the registers per thread.
    const char *ct = getenv("BZ_CELL_THREADS");
    const int maxt = (ct && atoi(ct) == 512) ? 512 : 1024;
    const int Q = N * N / 4;
    if (Q > maxt) return BZ_OK;
    int K = 1;
    for (int k = 1; k <= N; ++k)
        if (N % k == 0 && Q * k <= maxt) K = k;
    const int T = (Q * K + 31) / 32 * 32;
    H->map = bzk::Map4{Q, K, N / K};
    H->threads4 = T;
    H->maxt4 = maxt;
    H->smem4 = bzk::cell4_smem_bytes(N, g.nvt, g.nt);
    int of = 0, oc = 0;
    if (maxt == 512) {
        BZ_TRY((setup_cell4_kernel<true, 512>(H, &of)));
        BZ_TRY((setup_cell4_kernel<false, 512>(H, &oc)));
    } else {
        BZ_TRY((setup_cell4_kernel<true, 1024>(H, &of)));
        BZ_TRY((setup_cell4_kernel<false, 1024>(H, &oc)));
    }
    if (of < 1 || oc < 1) return BZ_OK;
    H->grid4f = std::min(g.nr, H->nsm * of);
    H->grid4c = std::min(g.nr, H->nsm * oc);
    BZ_TRY(dalloc(&H->sc_count, sizeof(int) * g.nvt));
    BZ_TRY(dalloc(&H->sc_cursor, sizeof(int) * g.nvt));
    BZ_TRY(dalloc(&H->sc_meta, sizeof(int) * 2));
    BZ_TRY(dalloc(&H->sc_ent, sizeof(uint32_t) * ((size_t)4 * g.nt + bzk::kMaxThreads)));
    H->fast = true;
    H->g.swz = 1;
    return BZ_OK;
}

// ---------------------------------------------------------------------
// Active-node path with deferred correction (bz_lazy.cuh)
// ---------------------------------------------------------------------

// A buffer's pending corrections are applied in place (paths that read
// corrected states call this first).
bz_status materialize_if_lazy(bz_handle *H, int x, cudaStream_t s)
{
    if (!H->lazy_buf[x]) return BZ_OK;
    const Geo &g = H->g;
    bzk::k_lz_materialize<<<std::min(g.nr, H->nsm * 8), 256, 0, s>>>(
        g, nullptr, (const float *)H->h[x], H->mu[x], (float *)H->h[x], nullptr);
    BZ_LAUNCHED(H);
    BZ_CUDA(cudaMemsetAsync(H->mu[x], 0, sizeof(float) * 8 * (size_t)g.nr, s));
    H->lazy_buf[x] = false;
    return BZ_OK;
}

// Buffer x is about to be overwritten by a path that writes corrected states.
bz_status drop_lazy(bz_handle *H, int x, cudaStream_t s)
{
    if (!H->lazy_buf[x]) return BZ_OK;
    BZ_CUDA(cudaMemsetAsync(H->mu[x], 0, sizeof(float) * 8 * (size_t)H->g.nr, s));
    H->lazy_buf[x] = false;
    return BZ_OK;
}

// Value of monomial k of the 30-entry sum vector of bz_lazy.cuh at (x, y, z).
double lz_monomial(int k, double x, double y, double z)
{
    const double v2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return x * x;
    case 5: return y * y;
    case 6: return z * z;
    case 7: return x * y;
    case 8: return x * z;
    case 9: return y * z;
    case 10: return x * x * x;
    case 11: return y * y * y;
    case 12: return z * z * z;
    case 13: return x * x * y;
    case 14: return x * x * z;
    case 15: return x * y * y;
    case 16: return y * y * z;
    case 17: return x * z * z;
    case 18: return y * z * z;
    case 19: return x * y * z;
    case 20: return x * x * v2;
    case 21: return y * y * v2;
    case 22: return z * z * v2;
    case 23: return x * y * v2;
    case 24: return x * z * v2;
    case 25: return y * z * v2;
    case 26: return v2;
    case 27: return x * v2;
    case 28: return y * v2;
    default: return z * v2;
    }
}

// Velocity axes with a kernel specialised on their length (the others run
// the kernel that reads it at run time); stretched grids (per-cell Courant
// factors) have their own instances, specialised for 20 nodes per axis (the
// paper's stretched cavities) and run-time lengths otherwise.
int lz_nv_key(const bz_handle *H) { return H->stretched ? (H->g.nv == 20 ? -20 : -1) : (H->g.nv == 32 || H->g.nv == 20 ? H->g.nv : 0); }

template <int G, int NV, bool SX, bool TMA = false>
bz_status setup_lz_one(bz_handle *H, size_t smem, int *occ)
{
    BZ_CUDA(bz_allow_max_smem(bzk::k_lz<G, NV, SX, TMA>, H->smem_optin));
    BZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, bzk::k_lz<G, NV, SX, TMA>, H->lz_T, smem));
    return BZ_OK;
}

template <int G>
bz_status setup_lz_kernel(bz_handle *H, size_t smem, int *occ)
{
    if (G == 4 && H->lz_tma && lz_nv_key(H) >= 0)
        return lz_nv_key(H) == 32 ? setup_lz_one<4, 32, false, true>(H, smem, occ)
                                  : setup_lz_one<4, 0, false, true>(H, smem, occ);
    switch (lz_nv_key(H)) {
    case 32: return setup_lz_one<G, 32, false>(H, smem, occ);
    case 20: return setup_lz_one<G, 20, false>(H, smem, occ);
    case -1: return setup_lz_one<G, 0, true>(H, smem, occ);
    case -20: return setup_lz_one<G, 20, true>(H, smem, occ);
    default: return setup_lz_one<G, 0, false>(H, smem, occ);
    }
}

template <int G>
void launch_lz_kernel(bz_handle *H, const bzk::LzArgs &a, cudaStream_t s)
{
    if (G == 4 && H->lz_tma && lz_nv_key(H) >= 0) {
        if (lz_nv_key(H) == 32)
            bzk::k_lz<4, 32, false, true><<<H->lz_grid, H->lz_T, H->lz_smem, s>>>(H->g, a);
        else
            bzk::k_lz<4, 0, false, true><<<H->lz_grid, H->lz_T, H->lz_smem, s>>>(H->g, a);
        return;
    }
    switch (lz_nv_key(H)) {
    case 32: bzk::k_lz<G, 32, false><<<H->lz_grid, H->lz_T, H->lz_smem, s>>>(H->g, a); break;
    case 20: bzk::k_lz<G, 20, false><<<H->lz_grid, H->lz_T, H->lz_smem, s>>>(H->g, a); break;
    case -1: bzk::k_lz<G, 0, true><<<H->lz_grid, H->lz_T, H->lz_smem, s>>>(H->g, a); break;
    case -20: bzk::k_lz<G, 20, true><<<H->lz_grid, H->lz_T, H->lz_smem, s>>>(H->g, a); break;
    default: bzk::k_lz<G, 0, false><<<H->lz_grid, H->lz_T, H->lz_smem, s>>>(H->g, a); break;
    }
}

// Decide whether the active-node path applies (FP32 fast path, at most 32
// nodes per axis) and size it: the number of active nodes is measured on the
// sample sets of the first steps (it depends on the grid and the sample count
// only, not on the state) and the compact arrays get a margin above it.  The
// largest group of cells per CTA (4, else 2) whose shared memory fits is
// taken.  Needs the per-axis tables on the device.
bz_status configure_lazy(bz_handle *H)
{
    H->lazy = false;
    const Geo &g = H->g;
    const char *force = getenv("BZ_KERNEL");
    if (force && (strcmp(force, "generic") == 0 || strcmp(force, "cell4") == 0)) return BZ_OK;
    if (!H->fast || g.nv > bzk::kLzMaxN || g.nv % 4 != 0 || g.nvt % 32 != 0) return BZ_OK;
    const int N = g.nv, nvt = g.nvt, nt = g.nt;
    const int P4 = bzk::lz_planes4(N);
    if (P4 == 0) return BZ_OK;
    const size_t mub = sizeof(float) * 8 * (size_t)g.nr;
    BZ_TRY(dalloc(&H->mu[0], mub));
    BZ_TRY(dalloc(&H->mu[1], mub));
    BZ_CUDA(cudaMemset(H->mu[0], 0, mub));
    BZ_CUDA(cudaMemset(H->mu[1], 0, mub));
    BZ_TRY(dalloc(&H->lz_idx, sizeof(int4) * (size_t)nt));
    BZ_TRY(dalloc(&H->lz_pa, sizeof(bzk::PlanA<float, int>) * (size_t)nt));
    BZ_TRY(dalloc(&H->lz_qc, sizeof(ushort4) * (size_t)nt));
    BZ_TRY(dalloc(&H->lz_flag, sizeof(int) * nvt));
    BZ_TRY(dalloc(&H->lz_cidx, sizeof(int) * nvt));
    BZ_TRY(dalloc(&H->lz_act, sizeof(int) * nvt));
    BZ_TRY(dalloc(&H->lz_mask, sizeof(uint32_t) * (nvt / 32)));
    BZ_TRY(dalloc(&H->lz_wpre, sizeof(int) * (nvt / 32)));
    BZ_TRY(dalloc(&H->lz_meta, sizeof(int) * bzk::kLzMetaSize));
    BZ_CUDA(cudaMemset(H->lz_flag, 0, sizeof(int) * nvt));
    BZ_CUDA(cudaMemset(H->lz_meta, 0, sizeof(int) * bzk::kLzMetaSize));

    // Active nodes of the sample sets of steps 0..3.
    int64_t *dstep = nullptr;
    BZ_TRY(dalloc(&dstep, sizeof(int64_t)));
    Geo gl = g;
    gl.swz = 0;
    const int pb = 256, pg = (nt + pb - 1) / pb;
    int mmax = 0;
    cudaError_t e = cudaSuccess;
    for (int64_t st = 0; st < 4 && e == cudaSuccess; ++st) {
        e = cudaMemcpy(dstep, &st, sizeof(int64_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) break;
        bzk::k_plan<float, int><<<pg, pb>>>(gl, dstep, H->lz_idx, H->lz_pa, nullptr, nullptr);
        bzk::k_lz_mark<<<pg, pb>>>(nt, H->lz_idx, H->lz_flag);
        bzk::k_lz_scan<<<1, 1024>>>(nvt, nvt, H->lz_flag, H->lz_cidx, H->lz_act, H->lz_mask,
                                    H->lz_wpre, H->lz_meta);
        int m = 0;
        e = cudaMemcpy(&m, H->lz_meta, sizeof(int), cudaMemcpyDeviceToHost);
        mmax = std::max(mmax, m);
    }
    cudaFree(dstep);
    if (e != cudaSuccess) return fail(BZ_ECUDA, "active-node probe failed: %s", cudaGetErrorString(e));
    H->lz_mprobe = mmax;
    // The count varies little from step to step (it is a sum of many nearly
    // independent node hits); a step above the capacity runs the fallback.
    int mcap = std::min(nvt, (mmax + mmax / 20 + 64 + 31) / 32 * 32);
    if (const char *mc = getenv("BZ_LAZY_MCAP")) mcap = std::max(1, std::min(nvt, atoi(mc)));
    if (const char *tm = getenv("BZ_LAZY_TMA")) H->lz_tma = atoi(tm) != 0;

    // One CTA of two 256-thread roles per SM; the largest group of cells
    // whose shared memory fits.
    H->lz_T = bzk::kLzThreads;
    bool ok = false;
    const char *force_g = getenv("BZ_LAZY_G");
    for (int G : {4, 2}) {
        if (force_g && atoi(force_g) != G) continue;
        // Term records address a compact array with 16-bit byte offsets.
        if ((size_t)mcap * 4 * G > 65535) continue;
        const size_t smem = bzk::lz_offsets(nvt, mcap, G).end;
        if (smem > (size_t)H->smem_optin) continue;
        int occ = 0;
        if (G == 4) BZ_TRY(setup_lz_kernel<4>(H, smem, &occ));
        else BZ_TRY(setup_lz_kernel<2>(H, smem, &occ));
        if (occ < 1) continue;
        H->lz_G = G;
        H->lz_smem = smem;
        H->lz_grid = std::min((g.nr + G - 1) / G, H->nsm);
        if (const char *c = getenv("BZ_LAZY_CTAS")) H->lz_grid = std::max(1, std::min(H->lz_grid, atoi(c)));
        ok = true;
        break;
    }
    if (!ok) return BZ_OK;
    H->lz_mcap = mcap;
    // Bank-aware ordering of the term runs: one warp per phase group of
    // runs, with their records staged in shared memory.
    H->lz_cmax = ((4 * nt + bzk::kLzRoleT - 1) / bzk::kLzRoleT + 7) / 8 * 8;
    {
        const int nb = H->lz_G == 4 ? 8 : 16;
        H->lz_chunk = std::min(H->lz_cmax, 64);
        if (const char *c = getenv("BZ_LAZY_ORDER_CHUNK")) H->lz_chunk = std::max(8, std::min(H->lz_cmax, atoi(c)));
        // The order saves shared-memory replays on every CTA iteration (about
        // 3 us per iteration at 320 positions on a GB300).  Built per step it
        // costs a chain of about 2 x 64 dependent decisions (about 50 us) on
        // the step's critical path: it runs when the iterations per CTA times
        // the run length reach 6144.  With the plans built ahead (below) it
        // runs over whole runs and costs GPU time in proportion to the run
        // length (about 45-65 us per step at 2x10^4 samples, by the batch
        // size), which pays from about 12 iterations per CTA on (measured:
        // 64^2 cells lose 1%, 96^2 and more gain 0.6-9%).
        const int64_t iters = ((int64_t)(g.nr + H->lz_G - 1) / H->lz_G + H->lz_grid - 1) / H->lz_grid;
        const char *ka = getenv("BZ_LAZY_AHEAD");
        const bool per_step = ka && atoi(ka) == 0;
        H->lz_order_tpb = H->lz_chunk <= 32767 && (per_step ? iters * H->lz_cmax >= 6144 : iters >= 12) &&
                          bzk::lz_order_smem(H->lz_chunk, nb) <= (size_t)H->smem_optin ? 1 : 0;
        if (const char *o = getenv("BZ_LAZY_ORDER")) H->lz_order_tpb = atoi(o) != 0 && H->lz_chunk <= 32767 &&
                          bzk::lz_order_smem(H->lz_chunk, nb) <= (size_t)H->smem_optin ? 1 : 0;
        if (getenv("BZ_LAZY_NOORDER")) H->lz_order_tpb = 0;
        if (H->lz_order_tpb > 0)
            BZ_CUDA(bz_allow_max_smem(nb == 8 ? bzk::k_lz_order<8> : bzk::k_lz_order<16>, H->smem_optin));
    }
    BZ_TRY(dalloc(&H->lz_count, sizeof(int) * (size_t)nvt));
    BZ_TRY(dalloc(&H->lz_cursor, sizeof(int) * (size_t)nvt));
    BZ_TRY(dalloc(&H->lz_rowend, sizeof(int) * (size_t)nvt));
    BZ_TRY(dalloc(&H->lz_dest0, sizeof(int) * (size_t)bzk::kLzRoleT));
    BZ_TRY(dalloc(&H->lz_rec, sizeof(uint2) * ((size_t)4 * nt + (size_t)8 * bzk::kLzRoleT)));
    BZ_CUDA(cudaMemset(H->lz_count, 0, sizeof(int) * (size_t)nvt));
    // Plans of K steps built ahead at a time (BZ_LAZY_AHEAD=K sets the
    // count, 0 builds each step's plan in the step), their term order over
    // whole runs.  The order kernel's one-warp CTAs (T / NB per plan and
    // chunk) are bound by their shared memory to a few per SM and take about
    // the same time in every wave.  When 32 plans need more than one wave, K
    // fills the last wave; K is kept even so that the two-step graphs never
    // straddle a batch; at most 64.  (On a 152-SM GB300 at 2x10^4 samples
    // seven CTAs fit an SM, so the 1024 CTAs of 32 plans take one wave.)
    {
        const int nb = H->lz_G == 4 ? 8 : 16;
        H->ahead_chunk = H->lz_cmax;
        if (getenv("BZ_LAZY_ORDER_CHUNK")) H->ahead_chunk = H->lz_chunk;
        if (H->lz_order_tpb > 0 && bzk::lz_order_smem(H->ahead_chunk, nb) > (size_t)H->smem_optin)
            H->ahead_chunk = H->lz_chunk;
        H->ahead_K = 32;
        if (H->lz_order_tpb > 0) {
            const int nch = (H->lz_cmax + H->ahead_chunk - 1) / H->ahead_chunk;
            const int64_t per = (int64_t)(bzk::kLzRoleT / nb) * nch;       // CTAs per plan
            int occ = 0;
            const size_t osm = bzk::lz_order_smem(H->ahead_chunk, nb);
            BZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &occ, nb == 8 ? bzk::k_lz_order<8> : bzk::k_lz_order<16>, 32, osm));
            const int64_t wave = (int64_t)occ * H->nsm;
            if (wave > 0 && 32 * per > wave) {
                const int64_t waves = (32 * per + wave - 1) / wave;
                H->ahead_K = (int)std::min<int64_t>(64, waves * wave / per / 2 * 2);
            }
        }
    }
    if (const char *kk = getenv("BZ_LAZY_AHEAD")) H->ahead_K = std::max(0, std::min(256, atoi(kk)));
    if (H->ahead_K > 0) {
        bzk::AheadPlans &A = H->ahead;
        const int K = H->ahead_K;
        A.K = K;
        A.nt = nt;
        A.nvt = nvt;
        A.mcap = mcap;
        A.osh = H->lz_G == 4 ? 4 : 3;
        A.recn = (int64_t)4 * nt + (int64_t)8 * bzk::kLzRoleT;
        const size_t k = (size_t)K;
        BZ_TRY(dalloc(&A.idx, sizeof(int4) * k * nt));
        BZ_TRY(dalloc(&A.pa, sizeof(bzk::PlanA<float, int>) * k * nt));
        BZ_TRY(dalloc(&A.qc, sizeof(ushort4) * k * nt));
        BZ_TRY(dalloc(&A.flag, sizeof(int) * k * nvt));
        BZ_TRY(dalloc(&A.cidx, sizeof(int) * k * nvt));
        BZ_TRY(dalloc(&A.act, sizeof(int) * k * nvt));
        BZ_TRY(dalloc(&A.mask, sizeof(uint32_t) * k * (nvt / 32)));
        BZ_TRY(dalloc(&A.wpre, sizeof(int) * k * (nvt / 32)));
        BZ_TRY(dalloc(&A.meta, sizeof(int) * k * bzk::kLzMetaSize));
        BZ_TRY(dalloc(&A.count, sizeof(int) * k * nvt));
        BZ_TRY(dalloc(&A.cursor, sizeof(int) * k * nvt));
        BZ_TRY(dalloc(&A.rowend, sizeof(int) * k * nvt));
        BZ_TRY(dalloc(&A.dest0, sizeof(int) * k * bzk::kLzRoleT));
        BZ_TRY(dalloc(&A.rec, sizeof(uint2) * k * (size_t)A.recn));
        BZ_TRY(dalloc(&A.cnt, sizeof(unsigned long long) * 2 * k));
        BZ_CUDA(cudaMemset(A.flag, 0, sizeof(int) * k * nvt));
        BZ_CUDA(cudaMemset(A.count, 0, sizeof(int) * k * nvt));
        H->ahead_lo = H->ahead_hi = 0;
    }
    // Equilibrium sums of the 30 monomials (the moments of h^{n+1} need them).
    std::vector<double> axv(N), axA(N);
    BZ_CUDA(cudaMemcpy(axv.data(), g.axv, sizeof(double) * N, cudaMemcpyDeviceToHost));
    BZ_CUDA(cudaMemcpy(axA.data(), g.axA, sizeof(double) * N, cudaMemcpyDeviceToHost));
    for (int k = 0; k < bzk::kLzX; ++k) {
        double acc = 0.0;
        for (int jx = 0; jx < N; ++jx)
            for (int jy = 0; jy < N; ++jy)
                for (int jz = 0; jz < N; ++jz)
                    acc += axA[jx] * axA[jy] * axA[jz] * lz_monomial(k, axv[jx], axv[jy], axv[jz]);
        H->lz_e0[k] = (float)acc;
    }
    {
        // The plan is a chain of small latency-bound kernels: its blocks go
        // first when the walls' blocks leave room.
        int least = 0, greatest = 0;
        BZ_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        BZ_CUDA(cudaStreamCreateWithPriority(&H->lz_side, cudaStreamNonBlocking, greatest));
    }
    BZ_CUDA(cudaEventCreateWithFlags(&H->lz_fork, cudaEventDisableTiming));
    BZ_CUDA(cudaEventCreateWithFlags(&H->lz_join, cudaEventDisableTiming));
    BZ_CUDA(cudaEventCreateWithFlags(&H->lz_mid, cudaEventDisableTiming));
    H->lazy = true;
    return BZ_OK;
}

// One fused step on the active-node path: walls (applying the input's
// pending corrections), the sample set, its compact form and scatter list,
// the per-cell kernel, and the k_cell4 fallback that runs only when the step
// has more active nodes than the compact arrays hold.  The sample plan
// depends on the step counter only, so it runs on a side stream while the
// walls run (after everything before the step on s: the last step's kernel
// reads the plan's buffers), and the per-cell kernel waits for both.
// nostream: the relaxation alone (BZ_DO_COLLIDE), h~ = h; the walls still
// run so that the ghost values the kernel reads (times a zero Courant
// number) are those of the state.
// The plans of steps [n, n + K) built ahead into the handle's K slots on
// stream s, unless the slots already cover [n, n + cnt).  Never called while
// a stream is being captured (the step graphs hold only k_ahead_take).
bz_status ensure_plans(bz_handle *H, cudaStream_t s, int64_t n, int cnt)
{
    if (!H->lazy || H->ahead_K == 0) return BZ_OK;
    if (n >= H->ahead_lo && n + cnt <= H->ahead_hi) return BZ_OK;
    const bzk::AheadPlans &A = H->ahead;
    const int K = H->ahead_K;
    Geo gl = H->g;
    gl.swz = 0;
    ProfScope ps(H, 1, s);
    BZ_CUDA(cudaMemsetAsync(A.cnt, 0, sizeof(unsigned long long) * 2 * K, s));
    bzk::k_ahead_plan<<<dim3((A.nt + 63) / 64, K), 64, 0, s>>>(gl, A, n);
    BZ_LAUNCHED(H);
    bzk::k_ahead_scan<<<K, 1024, 0, s>>>(A, n);
    BZ_LAUNCHED(H);
    bzk::k_ahead_remap<<<dim3((A.nt + 255) / 256, K), 256, 0, s>>>(A, n);
    BZ_LAUNCHED(H);
    bzk::k_ahead_lscan<<<K, 1024, 0, s>>>(A, n);
    BZ_LAUNCHED(H);
    bzk::k_ahead_lfill<<<dim3((A.nt + 255) / 256, K), 256, 0, s>>>(A, n);
    BZ_LAUNCHED(H);
    if (H->lz_order_tpb > 0) {
        const int ch = H->ahead_chunk, nch = (H->lz_cmax + ch - 1) / ch, z0 = (int)(n % K);
        if (H->lz_G == 4)
            bzk::k_lz_order<8><<<dim3(bzk::kLzRoleT / 8, nch, K), 32, bzk::lz_order_smem(ch, 8), s>>>(
                bzk::kLzRoleT, H->lz_cmax, ch, A.meta, A.rec, K, z0, A.recn);
        else
            bzk::k_lz_order<16><<<dim3(bzk::kLzRoleT / 16, nch, K), 32, bzk::lz_order_smem(ch, 16), s>>>(
                bzk::kLzRoleT, H->lz_cmax, ch, A.meta, A.rec, K, z0, A.recn);
        BZ_LAUNCHED(H);
    }
    H->ahead_lo = n;
    H->ahead_hi = n + K;
    return BZ_OK;
}

// ahead: the step's plan is copied from the slots built ahead (ensure_plans
// covered it) instead of being built by the per-step chain.
bz_status launch_lazy(bz_handle *H, cudaStream_t s, bool advance_step = true, bool nostream = false,
                      bool ahead = false)
{
    const Geo &g = H->g;
    Geo gl = g;
    gl.swz = 0;
    const int in = H->cur, out = in ^ 1;
    float *hin = (float *)H->h[in];
    float *hout = (float *)H->h[out];
    BZ_CUDA(cudaEventRecord(H->lz_fork, s));
    BZ_CUDA(cudaStreamWaitEvent(H->lz_side, H->lz_fork, 0));
    const int pb = 256, pg = (g.nt + pb - 1) / pb;
    if (ahead) {
        ProfScope ps(H, 1, H->lz_side);
        bzk::k_ahead_take<<<H->nsm, 256, 0, H->lz_side>>>(H->ahead, H->d_step, H->lz_idx, H->lz_pa, H->lz_meta,
                                                           H->lz_mask, H->lz_wpre, H->lz_act, H->lz_rec,
                                                           H->lz_dest0, H->stats);
        BZ_LAUNCHED(H);
    } else {
        const cudaStream_t sp = H->lz_side;
        ProfScope ps(H, 1, sp);
        // 64-thread blocks spread the FP64 sampling over every SM.
        bzk::k_plan<float, int><<<(g.nt + 63) / 64, 64, 0, sp>>>(gl, H->d_step, H->lz_idx, H->lz_pa, nullptr,
                                                  H->stats);
        BZ_LAUNCHED(H);
        bzk::k_lz_mark<<<pg, pb, 0, sp>>>(g.nt, H->lz_idx, H->lz_flag);
        BZ_LAUNCHED(H);
        bzk::k_lz_scan<<<1, 1024, 0, sp>>>(g.nvt, H->lz_mcap, H->lz_flag, H->lz_cidx, H->lz_act,
                                          H->lz_mask, H->lz_wpre, H->lz_meta, H->stats);
        BZ_LAUNCHED(H);
        bzk::k_lz_remap<<<pg, pb, 0, sp>>>(g.nt, H->lz_idx, H->lz_cidx, H->lz_qc, H->lz_count);
        BZ_LAUNCHED(H);
        bzk::k_lz_lscan<<<1, 1024, 0, sp>>>(bzk::kLzRoleT, H->lz_G == 4 ? 4 : 3, H->lz_count,
                                           H->lz_cursor, H->lz_rowend,
                                           H->lz_meta, H->lz_rec, H->lz_dest0);
        BZ_LAUNCHED(H);
        bzk::k_lz_lfill<<<pg, pb, 0, sp>>>(g.nt, bzk::kLzRoleT, H->lz_G == 4 ? 4 : 3, H->lz_qc, H->lz_pa,
                                          H->lz_cursor, H->lz_rowend, H->lz_meta, H->lz_rec,
                                          H->lz_dest0);
        BZ_LAUNCHED(H);
        if (H->lz_order_tpb > 0) {
            // The walls start now, beside the order (one warp per SM, bound by
            // latency) rather than beside the bandwidth-hungry plan kernels.
            BZ_CUDA(cudaEventRecord(H->lz_mid, sp));
            const int nch = (H->lz_cmax + H->lz_chunk - 1) / H->lz_chunk;
            if (H->lz_G == 4)
                bzk::k_lz_order<8><<<dim3(bzk::kLzRoleT / 8, nch), 32, bzk::lz_order_smem(H->lz_chunk, 8), sp>>>(
                    bzk::kLzRoleT, H->lz_cmax, H->lz_chunk, H->lz_meta, H->lz_rec);
            else
                bzk::k_lz_order<16><<<dim3(bzk::kLzRoleT / 16, nch), 32, bzk::lz_order_smem(H->lz_chunk, 16), sp>>>(
                    bzk::kLzRoleT, H->lz_cmax, H->lz_chunk, H->lz_meta, H->lz_rec);
            BZ_LAUNCHED(H);
        }
    }
    BZ_CUDA(cudaEventRecord(H->lz_join, H->lz_side));
    if (!ahead && H->lz_order_tpb > 0) BZ_CUDA(cudaStreamWaitEvent(s, H->lz_mid, 0));
    {
        ProfScope ps(H, 0, s);
        bzk::k_walls<float><<<g.nfaces, bzk::kWallThreads, 0, s>>>(g, H->d_step, hin, (float *)H->ghost, H->nw,
                                                     nullptr, H->mu[in]);
        BZ_LAUNCHED(H);
    }
    BZ_CUDA(cudaStreamWaitEvent(s, H->lz_join, 0));
    {
        ProfScope ps(H, 2, s);
        bzk::LzArgs a{};
        a.hin = hin;
        a.mu_in = H->mu[in];
        a.ghost = (const float *)H->ghost;
        a.hout = hout;
        a.mu_out = H->mu[out];
        a.mom = H->mom;
        a.rec = H->lz_rec;
        a.dest0 = H->lz_dest0;
        a.meta = H->lz_meta;
        a.mask = H->lz_mask;
        a.wpre = H->lz_wpre;
        a.act = H->lz_act;
        a.mcap = H->lz_mcap;
        for (int k = 0; k < bzk::kLzX; ++k) a.e0[k] = H->lz_e0[k];
        a.clk = H->prof_clk;
        a.stats = H->stats;
        a.err = H->stats + 8;
        a.fb_count = H->sc_count;
        a.fb_n = g.nvt;
        // BZ_LAZY_TMA_TIMEOUT_TEST=1: CTA 0 expects 16 bytes more than its
        // first bulk copies bring, so its first wait runs out (tests of the
        // bounded waits; the step's result is then invalid).
        if (const char *tt = getenv("BZ_LAZY_TMA_TIMEOUT_TEST")) a.tx_excess = atoi(tt) != 0 ? 16 : 0;
        a.nostream = nostream ? 1 : 0;
        // Below 32^3 velocities the streaming of a group takes longer than
        // its collision terms: the collision warps start the increment sums.
        a.early_tail = g.nv < 32 ? 1 : 0;
        if (const char *et = getenv("BZ_LAZY_EARLY_TAIL")) a.early_tail = atoi(et) != 0 ? 1 : 0;
        if (H->lz_G == 4) launch_lz_kernel<4>(H, a, s);
        else launch_lz_kernel<2>(H, a, s);
        BZ_LAUNCHED(H);
    }
    {
        // Fallback (each launch returns at once unless the step overflowed);
        // timed with the per-step plan.
        ProfScope ps(H, 1, s);
        const ushort4 *pi = (const ushort4 *)H->pidx;
        auto *pa16 = (bzk::PlanA<float, uint16_t> *)H->pa;
        // (k_lz zeroed the scatter counts if the step overflowed.)
        bzk::k_lz_fb_plan<<<pg, pb, 0, s>>>(g.nt, g.nv, H->lz_meta, H->lz_idx, H->lz_pa,
                                            (ushort4 *)H->pidx, pa16, H->sc_count);
        BZ_LAUNCHED(H);
        bzk::k_scatter_scan<<<1, 1024, 0, s>>>(g.nvt, H->threads4, H->sc_count, H->sc_cursor,
                                               H->sc_meta, H->lz_meta);
        BZ_LAUNCHED(H);
        bzk::k_scatter_fill<<<pg, pb, 0, s>>>(g.nt, H->threads4, pi, H->sc_cursor, H->sc_meta,
                                              H->sc_ent, H->lz_meta);
        BZ_LAUNCHED(H);
        // The input is corrected in place and its pending corrections go;
        // the output's are cleared (k_cell4 writes corrected values).
        bzk::k_lz_materialize<<<std::min(g.nr, H->nsm * 8), 256, 0, s>>>(
            g, H->lz_meta, hin, H->mu[in], hin, H->mu[out], H->mu[in]);
        BZ_LAUNCHED(H);
        const int grid = nostream ? H->grid4c : H->grid4f;
#define BZ_C4G(F, M)                                                                              \
    bzk::k_cell4<F, M><<<grid, H->threads4, H->smem4, s>>>(g, H->map, hin, (const float *)H->ghost, \
                                                          pa16, H->sc_ent, H->sc_meta, hout, H->mom, \
                                                          H->stats, nullptr, H->lz_meta)
        if (H->maxt4 == 512) {
            if (nostream) BZ_C4G(false, 512); else BZ_C4G(true, 512);
        } else {
            if (nostream) BZ_C4G(false, 1024); else BZ_C4G(true, 1024);
        }
#undef BZ_C4G
        BZ_LAUNCHED(H);
    }
    if (!advance_step) return BZ_OK;           // a repeatable trial of the step
    H->cur = out;
    H->mom_valid = true;
    H->lazy_buf[out] = true;
    return advance(H, s);
}

template <typename R, typename I>
bz_status launch_step(bz_handle *H, cudaStream_t s, bool fused, bool do_stream, bool do_collide)
{
    using V4 = typename bzk::Idx4<I>::type;
    using PA = bzk::PlanA<R, I>;
    if constexpr (sizeof(R) == 4) {
        const bool ahead = H->ahead_K > 0;
        if (fused && H->lazy) return launch_lazy(H, s, true, false, ahead);
        // The relaxation alone on the active-node kernel (no streaming).
        if (!fused && do_collide && !do_stream && H->lazy) return launch_lazy(H, s, true, true, ahead);
    }
    // Every other path reads and writes corrected states.
    BZ_TRY(materialize_if_lazy(H, H->cur, s));
    BZ_TRY(drop_lazy(H, H->cur ^ 1, s));
    Geo &g = H->g;
    R *hin = (R *)H->h[H->cur];
    R *hout = (R *)H->h[H->cur ^ 1];
    if (do_stream || fused) {
        ProfScope ps(H, 0, s);
        bzk::k_walls<R><<<g.nfaces, bzk::kWallThreads, 0, s>>>(g, H->d_step, hin, (R *)H->ghost, H->nw, nullptr);
        BZ_LAUNCHED(H);
    }
    if ((do_collide || fused) && !H->per_cell) {
        ProfScope ps(H, 1, s);
        int pb = 256, pg = (g.nt + pb - 1) / pb;
        bzk::k_plan<R, I><<<pg, pb, 0, s>>>(g, H->d_step, (V4 *)H->pidx, (PA *)H->pa, nullptr, H->stats);
        BZ_LAUNCHED(H);
    }
    if (fused && launch_cell4(H, s, true, hin, hout)) {
        BZ_LAUNCHED(H);
        H->cur ^= 1;
        H->mom_valid = true;
        return advance(H, s);
    }
    if (fused) {
        ProfScope ps(H, 2, s);
        if (H->per_cell)
            bzk::k_cell<R, true, I, true><<<H->grid_cell_fused, H->threads, H->smem_cell, s>>>(
                g, hin, (const R *)H->ghost, (const V4 *)H->pidx, (const PA *)H->pa,
                (R *)H->gw_global, hout, H->mom, H->stats, H->gw_in_smem, H->d_step);
        else
            bzk::k_cell<R, true, I><<<H->grid_cell_fused, H->threads, H->smem_cell, s>>>(
                g, hin, (const R *)H->ghost, (const V4 *)H->pidx, (const PA *)H->pa,
                (R *)H->gw_global, hout, H->mom, H->stats, H->gw_in_smem);
        BZ_LAUNCHED(H);
        H->cur ^= 1;
        H->mom_valid = true;
        return advance(H, s);
    }
    if (do_stream) {
        R *dst = do_collide ? (R *)H->ht : hout;
        int grid = std::min(g.nr, H->nsm * 16);
        {
            ProfScope ps(H, 3, s);
            if constexpr (sizeof(R) == 4) {
                if (H->fast) {
                    const int Q = g.nv * g.nv / 4;
                    const int blk = Q * std::max(1, 512 / Q);
                    const int g4 = std::min(g.nr, H->nsm * std::max(1, 2048 / blk));
                    if (H->stretched)
                        bzk::k_stream4<true><<<g4, blk, 0, s>>>(g, (const float *)hin, (const float *)H->ghost,
                                                                (float *)dst);
                    else
                        bzk::k_stream4<false><<<g4, blk, 0, s>>>(g, (const float *)hin, (const float *)H->ghost,
                                                                 (float *)dst);
                } else {
                    bzk::k_stream<R><<<grid, 256, 0, s>>>(g, hin, (const R *)H->ghost, dst);
                }
            } else {
                bzk::k_stream<R><<<grid, 256, 0, s>>>(g, hin, (const R *)H->ghost, dst);
            }
            BZ_LAUNCHED(H);
        }
        if (!do_collide) {
            H->cur ^= 1;
            H->mom_valid = false;
            return BZ_OK;
        }
        hin = dst;
    }
    if (do_collide && launch_cell4(H, s, false, hin, hout)) {
        BZ_LAUNCHED(H);
        H->cur ^= 1;
        H->mom_valid = true;
        return advance(H, s);
    }
    if (do_collide) {
        ProfScope ps(H, 2, s);
        if (H->per_cell)
            bzk::k_cell<R, false, I, true><<<H->grid_cell, H->threads, H->smem_cell, s>>>(
                g, hin, (const R *)H->ghost, (const V4 *)H->pidx, (const PA *)H->pa,
                (R *)H->gw_global, hout, H->mom, H->stats, H->gw_in_smem, H->d_step);
        else
            bzk::k_cell<R, false, I><<<H->grid_cell, H->threads, H->smem_cell, s>>>(
                g, hin, (const R *)H->ghost, (const V4 *)H->pidx, (const PA *)H->pa,
                (R *)H->gw_global, hout, H->mom, H->stats, H->gw_in_smem);
        BZ_LAUNCHED(H);
        H->cur ^= 1;
        H->mom_valid = true;
        return advance(H, s);
    }
    return BZ_OK;
}

template <typename R, typename I, bool PC>
bz_status configure_kernels_pc(bz_handle *H, int *occ_f, int *occ_c)
{
    BZ_CUDA(bz_allow_max_smem(bzk::k_cell<R, true, I, PC>, H->smem_optin));
    BZ_CUDA(bz_allow_max_smem(bzk::k_cell<R, false, I, PC>, H->smem_optin));
    BZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_f, bzk::k_cell<R, true, I, PC>,
                                                          H->threads, H->smem_cell));
    BZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_c, bzk::k_cell<R, false, I, PC>,
                                                          H->threads, H->smem_cell));
    return BZ_OK;
}

template <typename R, typename I>
bz_status configure_kernels(bz_handle *H, int *occ_f, int *occ_c)
{
    return H->per_cell ? configure_kernels_pc<R, I, true>(H, occ_f, occ_c)
                       : configure_kernels_pc<R, I, false>(H, occ_f, occ_c);
}

template <typename R>
bz_status configure_cell_kernel(bz_handle *H)
{
    Geo &g = H->g;
    int n2 = g.nv * g.nv;
    H->threads = std::min(bzk::kMaxThreads, (n2 + 31) / 32 * 32);
    // Per-cell sample sets keep each sample's four node indices in shared memory.
    const size_t idxb = !H->per_cell ? 0 : H->idx16 ? sizeof(ushort4) : sizeof(int4);
    size_t with_gw = bzk::cell_smem_bytes<R>(g.nv, g.nvt, g.nt, true, idxb);
    size_t without = bzk::cell_smem_bytes<R>(g.nv, g.nvt, g.nt, false, idxb);
    if (without > (size_t)H->smem_optin)
        return fail(BZ_EUNSUPPORTED,
                    "velocity slab of %d nodes%s needs %zu bytes of shared memory; the device "
                    "offers %d per block", g.nvt,
                    H->per_cell ? " and the node indices of every per-cell sample" : "", without,
                    H->smem_optin);
    H->gw_in_smem = with_gw <= (size_t)H->smem_optin;
    H->smem_cell = H->gw_in_smem ? with_gw : without;
    int occ_f = 0, occ_c = 0;
    if (H->idx16) {
        BZ_TRY((configure_kernels<R, uint16_t>(H, &occ_f, &occ_c)));
    } else {
        BZ_TRY((configure_kernels<R, int>(H, &occ_f, &occ_c)));
    }
    if (occ_f < 1 || occ_c < 1)
        return fail(BZ_EUNSUPPORTED, "cell kernel cannot be resident (%d threads, %zu bytes)",
                    H->threads, H->smem_cell);
    H->grid_cell_fused = std::min(g.nr, H->nsm * occ_f);
    H->grid_cell = std::min(g.nr, H->nsm * occ_c);
    if (!H->gw_in_smem) {
        int grid = std::max(H->grid_cell, H->grid_cell_fused);
        BZ_TRY(dalloc(&H->gw_global, sizeof(R) * (size_t)g.nt * grid));
    }
    return BZ_OK;
}

void clear_events(bz_handle *H)
{
    for (auto &v : H->ev) {
        for (auto &p : v) {
            cudaEventDestroy(p.first);
            cudaEventDestroy(p.second);
        }
        v.clear();
    }
}

void release(bz_handle *H)
{
    clear_events(H);
    drop_graphs(H);
    if (H->cap_stream) cudaStreamDestroy(H->cap_stream);
    if (H->lz_side) cudaStreamDestroy(H->lz_side);
    if (H->lz_fork) cudaEventDestroy(H->lz_fork);
    if (H->lz_join) cudaEventDestroy(H->lz_join);
    if (H->lz_mid) cudaEventDestroy(H->lz_mid);
    void *ptrs[] = {H->d_step, H->sc_count, H->sc_cursor, H->sc_meta, H->sc_ent, H->prof_clk, H->h[0], H->h[1], H->ht, H->pidx, H->pa, H->ghost, H->nw, H->shear,
                    H->mom, H->gw_global, H->stats, H->flag, H->axv, H->axA, H->profile};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    void *st[] = {H->axe, H->axd, H->wlid, H->sx, H->sy};
    for (void *p : st)
        if (p) cudaFree(p);
    void *lz[] = {H->mu[0], H->mu[1], H->lz_idx, H->lz_pa, H->lz_qc, H->lz_flag, H->lz_cidx,
                  H->lz_act, H->lz_wpre, H->lz_meta, H->lz_count, H->lz_cursor, H->lz_rowend,
                  H->lz_dest0, H->lz_mask, H->lz_rec};
    for (void *p : lz)
        if (p) cudaFree(p);
    const bzk::AheadPlans &A = H->ahead;
    void *ah[] = {A.idx, A.pa, A.qc, A.flag, A.cidx, A.act, A.mask, A.wpre, A.meta, A.count, A.cursor,
                  A.rowend, A.dest0, A.rec, A.cnt};
    for (void *p : ah)
        if (p) cudaFree(p);
    bz_adj_release(&H->adj);
}

}  // namespace

// The discretisation of a problem statement (Sec. 3, Sec. 5.1): grids, time
// step, collision prefactor, eps, wall constants and the equilibrium Gram
// matrix.  walls may be NULL (lid at rest; eps must then be given).
void bz_discretise(const bz_space *space, const bz_vel *vel, const bz_walls *walls,
                   const bz_params *params, bzk::Geo &g, bz_grid_tables &tb)
{
    const int N = vel->nv;
    g.nx = space->nx;
    g.ny = space->ny;
    g.nv = N;
    g.nvt = N * N * N;
    g.nr = g.nx * g.ny;
    g.nfaces = 2 * g.nx + 2 * g.ny;
    g.nt = (int)params->n_pairs;
    g.vmax = vel->vmax;
    g.dv = (2.0 * vel->vmax) / (double)N;
    g.dx = (1.0 / space->kn) / (double)g.nx;
    g.dy = (1.0 / space->kn) / (double)g.ny;
    const double cfl = params->cfl > 0.0 ? params->cfl : 0.5;
    // Grids (Sec. 3, Sec. 5.1), uniform or stretched.
    const bool sv = vel->rv > 0.0 && vel->rv < 1.0;
    std::vector<double> &edges = tb.edges, &axv = tb.axv, &axw = tb.axw, &axA = tb.axA;
    edges.assign(N + 1, 0.0);
    axv.assign(N, 0.0);
    axw.assign(N, 0.0);
    if (sv) {
        // Half-axis widths d0, d0 q, d0 q^2, ... (q = 1/rv) from the origin
        // outward summing to vmax; edges mirrored about 0.
        const int m = N / 2;
        const double q = 1.0 / vel->rv;
        const double d0 = g.vmax * (q - 1.0) / (std::pow(q, (double)m) - 1.0);
        for (int k = 0; k <= N; ++k) {
            const int i = k >= m ? k - m : m - k;
            const double e = d0 * (std::pow(q, (double)i) - 1.0) / (q - 1.0);
            edges[k] = k >= m ? e : -e;
        }
        for (int j = 0; j < N; ++j) {
            axv[j] = 0.5 * (edges[j] + edges[j + 1]);
            axw[j] = edges[j + 1] - edges[j];
        }
    } else {
        for (int j = 0; j < N; ++j) {
            axv[j] = -g.vmax + ((double)j + 0.5) * g.dv;
            axw[j] = g.dv;
        }
    }
    // Spatial widths: shrinking by r per cell toward the refined end(s).
    auto widths = [](int n, bool both_ends, double r, double L) {
        std::vector<double> w(n, L / n);
        if (!(r > 0.0 && r < 1.0)) return w;
        auto dist = [&](int k) { return both_ends ? std::min(k, n - 1 - k) : n - 1 - k; };
        double sum = 0.0;
        for (int k = 0; k < n; ++k) sum += std::pow(1.0 / r, (double)dist(k));
        for (int k = 0; k < n; ++k) w[k] = L * std::pow(1.0 / r, (double)dist(k)) / sum;
        return w;
    };
    tb.cdx = widths(g.nx, true, space->rx, 1.0 / space->kn);
    tb.cdy = widths(g.ny, false, space->ry, 1.0 / space->kn);
    double hmin = tb.cdx[0];
    for (double w : tb.cdx) hmin = std::min(hmin, w);
    for (double w : tb.cdy) hmin = std::min(hmin, w);
    const double vtop = axv[N - 1];
    g.dt = cfl * hmin / vtop;
    const double kcoll =
        params->kcoll > 0.0 ? params->kcoll : 5.0 * 1.016034 / 16.0 * std::sqrt(2.0 / M_PI);
    g.cw = M_PI * kcoll * g.dt / (double)g.nt;
    const double lu0 = walls ? walls->lid_u0 : 0.0, lamp = walls ? walls->lid_amp : 0.0;
    g.eps = params->eps > 0.0 ? params->eps
                              : lid_eps(lu0, lamp, walls ? walls->lid_profile : nullptr, g.nx);
    g.seed = params->seed;
    g.instance = params->instance;
    g.lid_u0 = lu0;
    g.lid_amp = lamp;
    g.lid_period = walls ? walls->lid_period : 0.0;
    g.strip = g.nx >= 16 ? 8 : g.nx;
    g.redraw_cap = -1;
    g.epsf = (float)g.eps;
    g.ryf = (float)(g.dx / g.dy);
    g.vmaxf = (float)g.vmax;
    g.idvf = (float)(1.0 / g.dv);
    g.cwf = (float)g.cw;
    // Per-axis weight factors (w_j = A_x A_y A_z) and the wall flux constants.
    axA.assign(N, 0.0);
    for (int j = 0; j < N; ++j)
        axA[j] = axw[j] * (1.0 / std::sqrt(M_PI)) * std::exp(-axv[j] * axv[j]);
    double hn = 0.0, zsum = 0.0;
    for (int j = 0; j < N; ++j) {
        zsum += axA[j];
        if (axv[j] > 0.0) hn += axv[j] * axA[j];
    }
    g.hn = hn;
    g.zsum = zsum;
    g.cout = hn * zsum * zsum;
    // Gram matrix of the equilibrium, sum_j w_j psi_a psi_b.
    for (int a = 0; a < 25; ++a) g.G0[a] = 0.0;
    for (int jx = 0; jx < N; ++jx)
        for (int jy = 0; jy < N; ++jy)
            for (int jz = 0; jz < N; ++jz) {
                double w = axA[jx] * axA[jy] * axA[jz];
                double p[5] = {1.0, axv[jx], axv[jy], axv[jz],
                               axv[jx] * axv[jx] + axv[jy] * axv[jy] + axv[jz] * axv[jz]};
                for (int a = 0; a < 5; ++a)
                    for (int b = 0; b < 5; ++b) g.G0[a * 5 + b] += w * p[a] * p[b];
            }
    for (int a = 0; a < 25; ++a) g.G0f[a] = (float)g.G0[a];
}

extern "C" {

const char *bz_last_error(void) { return g_last_error.c_str(); }

const char *bz_version(void) { return "bz 0.1 (sm_103a)"; }

bz_status bz_create(const bz_space *space, const bz_vel *vel, const bz_walls *walls,
                    const bz_params *params, bz_handle **out)
{
    g_last_error.clear();
    if (!out) return fail(BZ_EINVAL, "out is NULL");
    *out = nullptr;
    if (!space || !vel || !walls || !params) return fail(BZ_EINVAL, "NULL argument");
    if (space->nx < 1 || space->ny < 1) return fail(BZ_EINVAL, "nx, ny must be >= 1");
    if ((int64_t)space->nx * space->ny > (1 << 30)) return fail(BZ_EINVAL, "too many cells");
    if (!(space->kn > 0.0) || !std::isfinite(space->kn)) return fail(BZ_EINVAL, "kn must be > 0");
    if (vel->nv < 2 || vel->nv > bzk::kMaxN)
        return fail(BZ_EINVAL, "nv must be in [2, %d]", bzk::kMaxN);
    if (!(vel->vmax > 0.0) || !std::isfinite(vel->vmax)) return fail(BZ_EINVAL, "vmax must be > 0");
    for (double r : {vel->rv, space->rx, space->ry})
        if (!(r >= 0.0) || !(r <= 1.0)) return fail(BZ_EINVAL, "stretching ratios must be in [0, 1]");
    if (vel->rv > 0.0 && vel->rv < 1.0 && vel->nv % 2 != 0)
        return fail(BZ_EINVAL, "a stretched velocity grid needs an even nv");
    if (params->n_pairs < 1 || params->n_pairs > 0x7FFFFFFF)
        return fail(BZ_EINVAL, "n_pairs must be in [1, 2^31-1]");
    if (params->dtype != BZ_F32 && params->dtype != BZ_F64)
        return fail(BZ_EINVAL, "dtype must be BZ_F32 or BZ_F64");
    if (params->sample_mode != BZ_SHARED && params->sample_mode != BZ_PER_CELL)
        return fail(BZ_EINVAL, "unknown sample_mode");
    if (!(params->cfl >= 0.0 && params->cfl <= 1.0)) return fail(BZ_EINVAL, "cfl must be in [0, 1]");
    if (!(params->eps >= 0.0) || !std::isfinite(params->eps)) return fail(BZ_EINVAL, "eps must be >= 0");
    if (!(params->kcoll >= 0.0) || !std::isfinite(params->kcoll))
        return fail(BZ_EINVAL, "kcoll must be >= 0");
    if (!std::isfinite(walls->lid_u0) || !std::isfinite(walls->lid_amp) ||
        !(walls->lid_period >= 0.0) || !std::isfinite(walls->lid_period))
        return fail(BZ_EINVAL, "invalid lid motion");
    if (walls->lid_profile)
        for (int i = 0; i < space->nx; ++i)
            if (!std::isfinite(walls->lid_profile[i])) return fail(BZ_EINVAL, "lid_profile[%d]", i);
    if (fault_injected("alloc"))
        return fail(BZ_ENOMEM, "device allocation failed (BZ_FAULT=alloc)");

    bz_handle *H = new bz_handle();
    auto bail = [&](bz_status st) {
        release(H);
        delete H;
        return st;
    };
    Geo &g = H->g;
    const int N = vel->nv;
    bz_grid_tables tb;
    bz_discretise(space, vel, walls, params, g, tb);
    if (const char *fb = getenv("BZ_SOLVE_FALLBACK")) g.solve_fb = atoi(fb) != 0 ? 1 : 0;
    if (const char *rc = getenv("BZ_REDRAW_CAP")) g.redraw_cap = atoi(rc) >= 0 ? atoi(rc) : -1;
    const bool sv = vel->rv > 0.0 && vel->rv < 1.0;
    const bool sxg = space->rx > 0.0 && space->rx < 1.0, syg = space->ry > 0.0 && space->ry < 1.0;
    H->stretched = sv || sxg || syg;
    H->dtype = params->dtype;
    H->esz = params->dtype == BZ_F64 ? 8 : 4;
    H->per_cell = params->sample_mode == BZ_PER_CELL;
    const std::vector<double> &edges = tb.edges, &axv = tb.axv, &axw = tb.axw, &axA = tb.axA;
    const std::vector<double> &cdx = tb.cdx, &cdy = tb.cdy;

    cudaError_t e = cudaGetDevice(&H->dev);
    if (e != cudaSuccess) {
        fail(BZ_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
        return bail(BZ_ECUDA);
    }
    cudaDeviceGetAttribute(&H->nsm, cudaDevAttrMultiProcessorCount, H->dev);
    cudaDeviceGetAttribute(&H->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, H->dev);

    bz_status st = BZ_OK;
    const size_t nodes = (size_t)g.nr * g.nvt;
#define BZ_STEP(x)                   \
    do {                             \
        st = (x);                    \
        if (st != BZ_OK) return bail(st); \
    } while (0)
    BZ_STEP(dalloc(&H->h[0], nodes * H->esz));
    BZ_STEP(dalloc(&H->h[1], nodes * H->esz));
    H->idx16 = g.nvt < 65535;
    BZ_STEP(dalloc(&H->pidx, (H->idx16 ? sizeof(ushort4) : sizeof(int4)) * (size_t)g.nt));
    BZ_STEP(dalloc(&H->pa, 16 * (size_t)g.nt));
    BZ_STEP(dalloc(&H->ghost, H->esz * (size_t)g.nfaces * N));
    BZ_STEP(dalloc(&H->nw, sizeof(double) * g.nfaces));
    BZ_STEP(dalloc(&H->shear, sizeof(double) * (g.nx + 1)));
    BZ_STEP(dalloc(&H->mom, sizeof(double) * 11 * (size_t)g.nr));
    BZ_STEP(dalloc(&H->stats, sizeof(unsigned long long) * 9));
    BZ_STEP(dalloc(&H->flag, sizeof(int)));
    BZ_STEP(dalloc(&H->axv, sizeof(double) * N));
    BZ_STEP(dalloc(&H->axA, sizeof(double) * N));
    BZ_STEP(dalloc(&H->profile, sizeof(double) * g.nx));
    BZ_STEP(dalloc(&H->d_step, sizeof(int64_t)));
    if (H->dtype == BZ_F64)
        BZ_STEP(configure_cell_kernel<double>(H));
    else
        BZ_STEP(configure_cell_kernel<float>(H));
    BZ_STEP(configure_cell4(H));
#undef BZ_STEP
    if (H->stretched) {
        std::vector<double> fx(g.nx), fy(g.ny);
        std::vector<double> wl(g.nx);
        for (int i = 0; i < g.nx; ++i) {
            fx[i] = g.dx / cdx[i];
            wl[i] = cdx[i] * space->kn;
        }
        for (int i = 0; i < g.ny; ++i) fy[i] = g.dx / cdy[i];
        st = dalloc(&H->axe, sizeof(double) * (N + 1));
        if (st == BZ_OK) st = dalloc(&H->axd, sizeof(double) * N);
        if (st == BZ_OK) st = dalloc(&H->sx, sizeof(double) * g.nx);
        if (st == BZ_OK) st = dalloc(&H->sy, sizeof(double) * g.ny);
        if (st == BZ_OK) st = dalloc(&H->wlid, sizeof(double) * g.nx);
        if (st != BZ_OK) return bail(st);
        e = cudaMemcpy(H->axe, edges.data(), sizeof(double) * (N + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(H->axd, axw.data(), sizeof(double) * N, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(H->sx, fx.data(), sizeof(double) * g.nx, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(H->sy, fy.data(), sizeof(double) * g.ny, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(H->wlid, wl.data(), sizeof(double) * g.nx, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            fail(BZ_ECUDA, "grid table upload failed: %s", cudaGetErrorString(e));
            return bail(BZ_ECUDA);
        }
        if (sv) {
            g.axe = H->axe;
            g.axd = H->axd;
        }
        g.sx = H->sx;
        g.sy = H->sy;
        g.wlid = H->wlid;
    }
    e = cudaMemcpy(H->axv, axv.data(), sizeof(double) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(H->axA, axA.data(), sizeof(double) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && walls->lid_profile) {
        H->host_profile.assign(walls->lid_profile, walls->lid_profile + g.nx);
        e = cudaMemcpy(H->profile, walls->lid_profile, sizeof(double) * g.nx, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(H->h[0], 0, nodes * H->esz);
    if (e == cudaSuccess) e = cudaMemset(H->h[1], 0, nodes * H->esz);
    if (e == cudaSuccess) e = cudaMemset(H->stats, 0, sizeof(unsigned long long) * 9);
    if (e == cudaSuccess) e = cudaMemset(H->d_step, 0, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        fail(BZ_ECUDA, "initialisation failed: %s", cudaGetErrorString(e));
        return bail(BZ_ECUDA);
    }
    g.axv = H->axv;
    g.axA = H->axA;
    g.lid_profile = walls->lid_profile ? H->profile : nullptr;
    st = configure_lazy(H);
    if (st != BZ_OK) return bail(st);
    *out = H;
    return BZ_OK;
}

bz_status bz_destroy(bz_handle *H)
{
    if (!H) return BZ_OK;
    cudaDeviceSynchronize();
    release(H);
    delete H;
    return BZ_OK;
}

namespace {

bz_status one_step(bz_handle *H, cudaStream_t s, bool fused, bool ds, bool dc)
{
    if (H->dtype == BZ_F64)
        return H->idx16 ? launch_step<double, uint16_t>(H, s, fused, ds, dc)
                        : launch_step<double, int>(H, s, fused, ds, dc);
    return H->idx16 ? launch_step<float, uint16_t>(H, s, fused, ds, dc)
                    : launch_step<float, int>(H, s, fused, ds, dc);
}

bool graphs_enabled()
{
    const char *e = getenv("BZ_GRAPH");
    return !(e && strcmp(e, "0") == 0);
}

// Capture two fused steps (state buffer cur -> other -> cur) into a CUDA graph.
// The kernels read the step number from device memory and k_advance moves it
// on, so the graph can be replayed any number of times.
bz_status capture_pair(bz_handle *H)
{
    const int cur0 = H->cur;
    const int64_t step0 = H->step;
    const long long l0 = H->launches;
    const bool mv0 = H->mom_valid;
    const bool lz0[2] = {H->lazy_buf[0], H->lazy_buf[1]};
    // With profiling on, the timed launches' events become event record
    // nodes of the graph (recorded as external events while capturing).
    H->capturing = H->prof;
    H->cap_ev.clear();
    BZ_CUDA(cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal));
    bz_status st = one_step(H, H->cap_stream, true, false, false);
    if (st == BZ_OK) st = one_step(H, H->cap_stream, true, false, false);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(H->cap_stream, &graph);
    H->capturing = false;
    for (auto &c : H->cap_ev) {
        H->gplace.push_back(c.second.first);
        H->gplace.push_back(c.second.second);
    }
    H->graph_launches = H->launches - l0;
    H->cur = cur0;
    H->step = step0;
    H->launches = l0;
    H->mom_valid = mv0;
    H->lazy_buf[0] = lz0[0];
    H->lazy_buf[1] = lz0[1];
    if (st != BZ_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail(BZ_ECUDA, "step capture failed: %s", cudaGetErrorString(e));
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(BZ_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    H->graph[cur0] = ex;
    if (H->cap_ev.empty()) {
        cudaGraphDestroy(graph);
        return BZ_OK;
    }
    // The event record nodes of the timed launches, by the events they
    // were captured with.  The graph stays alive: its nodes name them.
    size_t nn = 0;
    BZ_CUDA(cudaGraphGetNodes(graph, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    BZ_CUDA(cudaGraphGetNodes(graph, nodes.data(), &nn));
    std::vector<std::pair<cudaEvent_t, cudaGraphNode_t>> rec;
    for (cudaGraphNode_t n : nodes) {
        cudaGraphNodeType t;
        BZ_CUDA(cudaGraphNodeGetType(n, &t));
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        BZ_CUDA(cudaGraphEventRecordNodeGetEvent(n, &ev));
        rec.push_back({ev, n});
    }
    auto node_of = [&](cudaEvent_t ev) -> cudaGraphNode_t {
        for (auto &r : rec)
            if (r.first == ev) return r.second;
        return nullptr;
    };
    for (auto &c : H->cap_ev) {
        cudaGraphNode_t na = node_of(c.second.first), nb = node_of(c.second.second);
        if (!na || !nb) {
            H->gprof[cur0].clear();
            cudaGraphDestroy(graph);
            return fail(BZ_ECUDA, "profiled step capture: an event record node is missing");
        }
        H->gprof[cur0].push_back({c.first, na, nb});
    }
    if (H->gtmpl[cur0]) cudaGraphDestroy(H->gtmpl[cur0]);
    H->gtmpl[cur0] = graph;
    return BZ_OK;
}

// Fresh events for the timed launches of the next replay of graph p (a
// replay records into the events its record nodes hold at launch time).
bz_status arm_profiled_graph(bz_handle *H, int p)
{
    for (auto &n : H->gprof[p]) {
        cudaEvent_t a = nullptr, b = nullptr;
        BZ_CUDA(cudaEventCreate(&a));
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return fail(BZ_ECUDA, "cudaEventCreate failed");
        }
        H->ev[n.k].push_back({a, b});
        BZ_CUDA(cudaGraphExecEventRecordNodeSetEvent(H->graph[p], n.a, a));
        BZ_CUDA(cudaGraphExecEventRecordNodeSetEvent(H->graph[p], n.b, b));
    }
    return BZ_OK;
}

}  // namespace

bz_status bz_step_ex(bz_handle *H, int32_t nsteps, uint32_t flags, void *stream)
{
    if (!H) return fail(BZ_EINVAL, "handle is NULL");
    if (nsteps < 0) return fail(BZ_EINVAL, "nsteps must be >= 0");
    if (flags & ~(uint32_t)(BZ_DO_STREAM | BZ_DO_COLLIDE | BZ_SPLIT))
        return fail(BZ_EINVAL, "unknown flags 0x%x", flags);
    if (fault_injected("launch")) return fail(BZ_ECUDA, "kernel launch failed (BZ_FAULT=launch)");
    cudaStream_t s = (cudaStream_t)stream;
    bool fused = flags == 0;
    bool ds = (flags & BZ_DO_STREAM) || (flags & BZ_SPLIT);
    bool dc = (flags & BZ_DO_COLLIDE) || (flags & BZ_SPLIT);
    if (ds && dc && !H->ht) BZ_TRY(dalloc(&H->ht, H->esz * (size_t)H->g.nr * H->g.nvt));
    int32_t n = 0;
    if (fused && nsteps >= 2 && graphs_enabled()) {
        // The captured steps read the buffers as they are now: bring the
        // pair into the state the steps leave it in before capturing.
        if (!H->lazy) {
            BZ_TRY(materialize_if_lazy(H, H->cur, s));
            BZ_TRY(drop_lazy(H, H->cur ^ 1, s));
        }
        if (!H->graph[H->cur]) BZ_TRY(capture_pair(H));
        for (; n + 1 < nsteps; n += 2) {
            BZ_TRY(ensure_plans(H, s, H->step, 2));
            if (H->prof) BZ_TRY(arm_profiled_graph(H, H->cur));
            BZ_CUDA(cudaGraphLaunch(H->graph[H->cur], s));
            H->step += 2;
            H->launches += H->graph_launches;
            H->mom_valid = true;
            if (H->lazy) H->lazy_buf[0] = H->lazy_buf[1] = true;
        }
    }
    const bool planned = fused || (dc && !ds);   // the steps that run the active-node kernel
    for (; n < nsteps; ++n) {
        if (planned) BZ_TRY(ensure_plans(H, s, H->step, 1));
        BZ_TRY(one_step(H, s, fused, ds, dc));
    }
    return BZ_OK;
}

bz_status bz_step(bz_handle *H, int32_t nsteps, void *stream)
{
    return bz_step_ex(H, nsteps, 0u, stream);
}

bz_status bz_moments(bz_handle *H, double *out, void *stream)
{
    if (!H || !out) return fail(BZ_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const Geo &g = H->g;
    if (!H->mom_valid) {
        BZ_TRY(materialize_if_lazy(H, H->cur, s));
        int grid = std::min(g.nr, H->nsm * 8);
        if (H->dtype == BZ_F64)
            bzk::k_moments<double><<<grid, 256, 0, s>>>(g, (const double *)H->h[H->cur], H->mom);
        else
            bzk::k_moments<float><<<grid, 256, 0, s>>>(g, (const float *)H->h[H->cur], H->mom);
        BZ_LAUNCHED(H);
        H->mom_valid = true;
    }
    size_t n = (size_t)g.nr * 11;
    BZ_CUDA(cudaMemsetAsync(H->flag, 0, sizeof(int), s));
    bzk::k_nonfinite<<<std::max(1, std::min(H->nsm, (int)((n + 255) / 256))), 256, 0, s>>>(
        H->mom, (int64_t)n, H->flag);
    BZ_LAUNCHED(H);
    BZ_CUDA(cudaMemcpyAsync(out, H->mom, sizeof(double) * n, cudaMemcpyDefault, s));
    int flag = 0;
    BZ_CUDA(cudaMemcpyAsync(&flag, H->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    BZ_CUDA(cudaStreamSynchronize(s));
    if (flag) return fail(BZ_ENONFINITE, "non-finite macroscopic quantity");
    return BZ_OK;
}

bz_status bz_lid_shear(bz_handle *H, double *out, void *stream)
{
    if (!H || !out) return fail(BZ_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const Geo &g = H->g;
    if (H->dtype == BZ_F64)
        bzk::k_walls<double><<<g.nfaces, bzk::kWallThreads, 0, s>>>(g, H->d_step, (const double *)H->h[H->cur],
                                                      (double *)H->ghost, H->nw, H->shear);
    else
        bzk::k_walls<float><<<g.nfaces, bzk::kWallThreads, 0, s>>>(g, H->d_step, (const float *)H->h[H->cur],
                                                     (float *)H->ghost, H->nw, H->shear,
                                                     H->lazy ? H->mu[H->cur] : nullptr);
    BZ_LAUNCHED(H);
    double *tmp = H->mom;  // reuse: nr*11 >= nx+1 always (ny >= 1)
    if ((size_t)g.nr * 11 < (size_t)g.nx + 1) return fail(BZ_EINVAL, "internal size");
    bzk::k_shear_mean<<<1, 256, 0, s>>>(H->shear, g.nx, g.wlid, tmp);
    BZ_LAUNCHED(H);
    H->mom_valid = false;
    BZ_CUDA(cudaMemcpyAsync(out, tmp, sizeof(double) * (g.nx + 1), cudaMemcpyDefault, s));
    return BZ_OK;
}

bz_status bz_get_state(bz_handle *H, void *dst, int64_t *step, void *stream)
{
    if (!H || !dst) return fail(BZ_EINVAL, "NULL argument");
    BZ_TRY(materialize_if_lazy(H, H->cur, (cudaStream_t)stream));
    BZ_CUDA(cudaMemcpyAsync(dst, H->h[H->cur], H->esz * (size_t)H->g.nr * H->g.nvt,
                            cudaMemcpyDefault, (cudaStream_t)stream));
    if (step) *step = H->step;
    return BZ_OK;
}

bz_status bz_set_state(bz_handle *H, const void *src, int64_t step, void *stream)
{
    if (!H || !src) return fail(BZ_EINVAL, "NULL argument");
    if (step < 0) return fail(BZ_EINVAL, "step must be >= 0");
    BZ_TRY(drop_lazy(H, H->cur, (cudaStream_t)stream));
    BZ_CUDA(cudaMemcpyAsync(H->h[H->cur], src, H->esz * (size_t)H->g.nr * H->g.nvt,
                            cudaMemcpyDefault, (cudaStream_t)stream));
    BZ_CUDA(cudaMemcpyAsync(H->d_step, &step, sizeof(int64_t), cudaMemcpyHostToDevice,
                            (cudaStream_t)stream));
    BZ_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    H->step = step;
    H->mom_valid = false;
    return BZ_OK;
}

bz_status bz_set_lid(bz_handle *H, double lid_u0, double lid_amp, double lid_period,
                     const double *lid_profile)
{
    if (!H) return fail(BZ_EINVAL, "handle is NULL");
    if (!std::isfinite(lid_u0) || !std::isfinite(lid_amp) || !(lid_period >= 0.0) ||
        !std::isfinite(lid_period))
        return fail(BZ_EINVAL, "invalid lid motion");
    Geo &g = H->g;
    if (lid_profile) {
        for (int i = 0; i < g.nx; ++i)
            if (!std::isfinite(lid_profile[i])) return fail(BZ_EINVAL, "lid_profile[%d]", i);
        // Ordered after earlier work on the legacy stream semantics of cudaMemcpy.
        BZ_CUDA(cudaMemcpy(H->profile, lid_profile, sizeof(double) * g.nx, cudaMemcpyHostToDevice));
        g.lid_profile = H->profile;
    } else {
        g.lid_profile = nullptr;
    }
    g.lid_u0 = lid_u0;
    g.lid_amp = lid_amp;
    g.lid_period = lid_period;
    drop_graphs(H);   // the captured launches hold the old wall parameters
    return BZ_OK;
}

bz_status bz_get_info(const bz_handle *H, bz_info *o)
{
    if (!H || !o) return fail(BZ_EINVAL, "NULL argument");
    const Geo &g = H->g;
    o->dt = g.dt;
    o->dx = g.dx;
    o->dy = g.dy;
    o->dv = g.dv;
    o->eps = g.eps;
    o->kcoll = g.cw * g.nt / (M_PI * g.dt);
    o->nodes = (int64_t)g.nr * g.nvt;
    o->state_bytes = o->nodes * (int64_t)H->esz;
    o->step = H->step;
    o->nr = g.nr;
    o->nvt = g.nvt;
    o->dtype = H->dtype;
    o->threads_per_cell = H->lazy ? H->lz_T : H->fast ? H->threads4 : H->threads;
    o->smem_bytes = (int32_t)(H->lazy ? H->lz_smem : H->fast ? H->smem4 : H->smem_cell);
    o->kernel_variant = H->lazy ? 2 : H->fast ? 1 : 0;
    o->plan_batch = H->lazy ? H->ahead_K : 0;
    o->plan_end = H->lazy && H->ahead_K > 0 ? H->ahead_hi : 0;
    return BZ_OK;
}

bz_status bz_stats(bz_handle *H, int64_t out[8])
{
    if (!H || !out) return fail(BZ_EINVAL, "NULL argument");
    unsigned long long d[9];
    BZ_CUDA(cudaDeviceSynchronize());
    BZ_CUDA(cudaMemcpy(d, H->stats, sizeof(d), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 8; ++i) out[i] = (int64_t)d[i];
    out[0] = H->step;
    out[4] = H->launches;
    out[7] = H->lz_mcap;
    if (d[8]) {
        // Reported once: the flag is cleared for the steps that follow.
        BZ_CUDA(cudaMemset(H->stats + 8, 0, sizeof(unsigned long long)));
        return fail(BZ_ETIMEOUT, "a bounded device wait of the active-node kernel gave up");
    }
    return BZ_OK;
}

bz_status bz_sample_plan(bz_handle *H, int64_t step, int32_t *idx, double *W, void *stream)
{
    if (!H || !idx || !W) return fail(BZ_EINVAL, "NULL argument");
    if (step < 0) return fail(BZ_EINVAL, "step must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const Geo &g = H->g;
    int4 *di = nullptr;
    double *dw = nullptr;
    int64_t *dstep = nullptr;
    BZ_TRY(dalloc(&di, sizeof(int4) * (size_t)g.nt));
    bz_status st = dalloc(&dw, sizeof(double) * (size_t)g.nt);
    if (st == BZ_OK) st = dalloc(&dstep, sizeof(int64_t));
    if (st != BZ_OK) {
        cudaFree(di);
        cudaFree(dw);
        return st;
    }
    if (cudaMemcpy(dstep, &step, sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(di);
        cudaFree(dw);
        cudaFree(dstep);
        return fail(BZ_ECUDA, "step upload failed");
    }
    int pb = 256, pg = (g.nt + pb - 1) / pb;
    Geo gl = g;
    gl.swz = 0;                       // logical node order for the caller
    if (H->dtype == BZ_F64)
        bzk::k_plan<double, int><<<pg, pb, 0, s>>>(gl, dstep, di, (bzk::PlanA<double, int> *)nullptr, dw, nullptr);
    else
        bzk::k_plan<float, int><<<pg, pb, 0, s>>>(gl, dstep, di, (bzk::PlanA<float, int> *)nullptr, dw, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(idx, di, sizeof(int4) * (size_t)g.nt, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(W, dw, sizeof(double) * (size_t)g.nt, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(di);
    cudaFree(dw);
    cudaFree(dstep);
    if (e != cudaSuccess) return fail(BZ_ECUDA, "sample plan failed: %s", cudaGetErrorString(e));
    H->launches++;
    return BZ_OK;
}

bz_status bz_sample_plan_cell(bz_handle *H, int64_t step, int32_t cell, int32_t *idx, double *W,
                              void *stream)
{
    if (!H || !idx || !W) return fail(BZ_EINVAL, "NULL argument");
    if (step < 0) return fail(BZ_EINVAL, "step must be >= 0");
    if (cell < 0 || cell >= H->g.nr) return fail(BZ_EINVAL, "cell %d outside [0, %d)", cell, H->g.nr);
    cudaStream_t s = (cudaStream_t)stream;
    const Geo &g = H->g;
    int4 *di = nullptr;
    double *dw = nullptr;
    BZ_TRY(dalloc(&di, sizeof(int4) * (size_t)g.nt));
    bz_status st = dalloc(&dw, sizeof(double) * (size_t)g.nt);
    if (st != BZ_OK) {
        cudaFree(di);
        return st;
    }
    const int pb = 256, pg = (g.nt + pb - 1) / pb;
    if (H->dtype == BZ_F64)
        bzk::k_plan_cell<double><<<pg, pb, 0, s>>>(g, step, (uint32_t)cell, di, dw);
    else
        bzk::k_plan_cell<float><<<pg, pb, 0, s>>>(g, step, (uint32_t)cell, di, dw);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(idx, di, sizeof(int4) * (size_t)g.nt, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(W, dw, sizeof(double) * (size_t)g.nt, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(di);
    cudaFree(dw);
    if (e != cudaSuccess) return fail(BZ_ECUDA, "per-cell sample plan failed: %s", cudaGetErrorString(e));
    H->launches++;
    return BZ_OK;
}

bz_status bz_profile(bz_handle *H, int32_t enable)
{
    if (!H) return fail(BZ_EINVAL, "handle is NULL");
    H->prof = enable != 0;
    drop_graphs(H);
    // The active-node path captures its profiled two-step graph now, so
    // that a timed region that starts next does not hold the capture.
    if (enable == 1 && H->lazy && graphs_enabled()) BZ_TRY(capture_pair(H));
    if (enable >= 2 && !H->prof_clk) {
        BZ_TRY(dalloc(&H->prof_clk, sizeof(long long) * bzk::kClkCells * bzk::kClkPhases));
        BZ_CUDA(cudaMemset(H->prof_clk, 0, sizeof(long long) * bzk::kClkCells * bzk::kClkPhases));
    } else if (enable < 2 && H->prof_clk) {
        cudaDeviceSynchronize();
        cudaFree(H->prof_clk);
        H->prof_clk = nullptr;
    }
    return BZ_OK;
}

bz_status bz_phase_clocks(bz_handle *H, int64_t *out, int32_t n)
{
    if (!H || !out || n < bzk::kClkCells * bzk::kClkPhases) return fail(BZ_EINVAL, "invalid argument");
    if (!H->prof_clk) return fail(BZ_ESTATE, "phase trace not enabled (bz_profile(h, 2))");
    BZ_CUDA(cudaDeviceSynchronize());
    BZ_CUDA(cudaMemcpy(out, H->prof_clk, sizeof(long long) * bzk::kClkCells * bzk::kClkPhases,
                       cudaMemcpyDeviceToHost));
    return BZ_OK;
}

bz_status bz_profile_read(bz_handle *H, double ms[4], int64_t launches[4])
{
    if (!H || !ms || !launches) return fail(BZ_EINVAL, "NULL argument");
    for (int k = 0; k < 4; ++k) {
        ms[k] = 0.0;
        launches[k] = (int64_t)H->ev[k].size();
        for (auto &p : H->ev[k]) {
            BZ_CUDA(cudaEventSynchronize(p.second));
            float t = 0.f;
            BZ_CUDA(cudaEventElapsedTime(&t, p.first, p.second));
            ms[k] += t;
        }
    }
    clear_events(H);
    return BZ_OK;
}

bz_status bz_adjoint_step(bz_handle *H, int64_t step, const void *h_n, const void *lam_in,
                          void *lam_out, double *grad_lid, double wD, void *stream)
{
    if (!H || !h_n || !lam_in || !lam_out) return fail(BZ_EINVAL, "NULL argument");
    if (step < 0) return fail(BZ_EINVAL, "step must be >= 0");
    if (H->per_cell)
        return fail(BZ_EUNSUPPORTED, "the adjoint is implemented for the shared sample set only");
    if (H->stretched) return fail(BZ_EUNSUPPORTED, "the adjoint is implemented for uniform grids only");
    if (!std::isfinite(wD)) return fail(BZ_EINVAL, "wD must be finite");
    const size_t bytes = H->esz * (size_t)H->g.nr * H->g.nvt;
    const char *a = (const char *)h_n, *b = (const char *)lam_out;
    if (a < b + bytes && b < a + bytes) return fail(BZ_EINVAL, "lam_out overlaps h_n");
    g_last_error.clear();
    bz_status st = bz_adj_prepare(&H->adj, H->g, H->dtype, H->nsm, H->smem_optin);
    if (st != BZ_OK) return st;
    return bz_adj_launch(&H->adj, H->g, H->dtype, step, h_n, lam_in, lam_out, grad_lid, wD,
                         H->stats, (cudaStream_t)stream, &H->launches);
}

bz_status bz_philox(uint32_t k0, uint32_t k1, const uint32_t *ctr, int64_t n, uint32_t *out)
{
    if (!ctr || !out || n < 0) return fail(BZ_EINVAL, "invalid argument");
    if (n == 0) return BZ_OK;
    uint4 *dc = nullptr, *dout = nullptr;
    BZ_TRY(dalloc(&dc, sizeof(uint4) * (size_t)n));
    bz_status st = dalloc(&dout, sizeof(uint4) * (size_t)n);
    if (st != BZ_OK) {
        cudaFree(dc);
        return st;
    }
    cudaError_t e = cudaMemcpy(dc, ctr, sizeof(uint4) * (size_t)n, cudaMemcpyDefault);
    if (e == cudaSuccess) {
        bzk::k_philox<<<(unsigned)((n + 255) / 256), 256>>>(make_uint2(k0, k1), dc, dout, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(uint4) * (size_t)n, cudaMemcpyDefault);
    cudaFree(dc);
    cudaFree(dout);
    if (e != cudaSuccess) return fail(BZ_ECUDA, "philox failed: %s", cudaGetErrorString(e));
    return BZ_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------
struct bz_batch {
    int n = 0;
    std::vector<bz_handle *> inst;
    std::vector<bzk::BInst> hinst;
    bzk::BInst *d_inst = nullptr;
    int *d_cell_pre = nullptr, *d_face_pre = nullptr, *d_samp_pre = nullptr;
    int tot_cells = 0, tot_faces = 0, tot_samples = 0;
    int nsm = 0;
    int maxt = 1024, grid = 0, strip = 8;
    size_t smem = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    std::vector<int64_t> step;
    // Fan-out mode: every instance's own step (the active-node kernels) on
    // `branches` forked streams, the whole step captured as one multi-branch
    // graph; one graph per parity pattern of the instances' steps.
    int mode = 0;                           // 0 persistent kernels, 1 fan-out, 2 persistent active-node
    int branches = 1;
    bool fan_ok = false;                    // every instance runs the active-node path
    std::vector<cudaStream_t> br;
    std::vector<cudaEvent_t> ev;            // fork + one join event per branch
    std::vector<int> owner;                 // branch of each instance
    cudaGraphExec_t fgraph[2] = {nullptr, nullptr};
    std::vector<int> fkey[2];
    // Persistent active-node mode: every instance's active-node step, one
    // launch per kernel class (bz_batch.cuh, kbl_*), the per-cell kernel as
    // persistent CTAs over segments of the instances' cell groups.
    bool lz_ok = false;
    bool lz_ahead = false;                  // every instance builds its plans ahead: copy them
    bzk::LzInst *d_lzinst = nullptr;
    int4 *d_segs = nullptr;
    int *d_next = nullptr;                  // one claim counter per velocity grid
    int nseg = 0;
    size_t lz_smem = 0;
    struct LzClass { int nv, seg0, nseg; size_t smem; };
    std::vector<LzClass> lz_classes;        // the segments of each velocity grid
    cudaStream_t lz_side = nullptr;         // the sample plans run here, beside the walls
    cudaEvent_t lz_fork = nullptr, lz_join = nullptr;
    // The velocity grids' kernels after the first run on streams of their own,
    // so that each starts on the SMs the previous one leaves.
    std::vector<cudaStream_t> lz_cls_s;
    std::vector<cudaEvent_t> lz_cls_done;
    cudaEvent_t lz_go = nullptr;
    cudaGraphExec_t graph2 = nullptr;
};

namespace {

bzk::Map4 map_for(int N, int maxt)
{
    const int Q = N * N / 4;
    int K = 1;
    for (int k = 1; k <= N; ++k)
        if (N % k == 0 && Q * k <= maxt) K = k;
    return bzk::Map4{Q, K, N / K};
}

void batch_free(bz_batch *B)
{
    if (B->graph) cudaGraphExecDestroy(B->graph);
    if (B->graph2) cudaGraphExecDestroy(B->graph2);
    void *lzp[] = {B->d_lzinst, B->d_segs, B->d_next};
    for (void *p : lzp)
        if (p) cudaFree(p);
    if (B->lz_side) cudaStreamDestroy(B->lz_side);
    for (cudaStream_t x : B->lz_cls_s) cudaStreamDestroy(x);
    for (cudaEvent_t x : B->lz_cls_done) cudaEventDestroy(x);
    if (B->lz_go) cudaEventDestroy(B->lz_go);
    if (B->lz_fork) cudaEventDestroy(B->lz_fork);
    if (B->lz_join) cudaEventDestroy(B->lz_join);
    for (auto &g : B->fgraph)
        if (g) cudaGraphExecDestroy(g);
    for (cudaStream_t st : B->br) cudaStreamDestroy(st);
    for (cudaEvent_t e : B->ev) cudaEventDestroy(e);
    if (B->cap) cudaStreamDestroy(B->cap);
    void *ptrs[] = {B->d_inst, B->d_cell_pre, B->d_face_pre, B->d_samp_pre};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (bz_handle *h : B->inst) bz_destroy(h);
}

template <int M>
bz_status batch_occupancy(bz_batch *B, int *occ)
{
    int dev = 0, optin = 0;
    BZ_CUDA(cudaGetDevice(&dev));
    BZ_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    BZ_CUDA(bz_allow_max_smem(bzk::kb_cell4<M>, optin));
    BZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, bzk::kb_cell4<M>, M, B->smem));
    return BZ_OK;
}

// Apply a schedule: strip width into every instance's geometry, block size.
bz_status batch_apply(bz_batch *B, int maxt, int ctas_per_sm, int strip)
{
    int occ = 0;
    if (maxt == 512) BZ_TRY(batch_occupancy<512>(B, &occ));
    else BZ_TRY(batch_occupancy<1024>(B, &occ));
    if (occ < 1) return fail(BZ_EUNSUPPORTED, "batched cell kernel cannot be resident");
    B->maxt = maxt;
    B->grid = std::min(B->tot_cells, B->nsm * std::min(occ, ctas_per_sm));
    B->strip = strip;
    for (int i = 0; i < B->n; ++i) {
        B->hinst[i].g.strip = std::min(strip, B->hinst[i].g.nx);
    }
    BZ_CUDA(cudaMemcpy(B->d_inst, B->hinst.data(), sizeof(bzk::BInst) * B->n,
                       cudaMemcpyHostToDevice));
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    return BZ_OK;
}

// One step of every instance; advance = false recomputes the current step.
constexpr int kMaxBranches = 8;

void drop_fan_graphs(bz_batch *B)
{
    for (int k = 0; k < 2; ++k) {
        if (B->fgraph[k]) cudaGraphExecDestroy(B->fgraph[k]);
        B->fgraph[k] = nullptr;
        B->fkey[k].clear();
    }
}

// Instances go to the branch with the least work so far (largest first).
void assign_branches(bz_batch *B, int nb)
{
    std::vector<int> order(B->n);
    for (int i = 0; i < B->n; ++i) order[i] = i;
    auto work = [&](int i) { return (double)B->inst[i]->g.nr * B->inst[i]->g.nvt; };
    std::sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
    std::vector<double> load(nb, 0.0);
    B->owner.assign(B->n, 0);
    for (int i : order) {
        int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        B->owner[i] = k;
        load[k] += work(i);
    }
    B->branches = nb;
}

// The instances' states for the persistent kernels: corrected, no pending
// corrections (leaving fan-out mode), or fresh zero corrections (entering it).
bz_status batch_set_mode(bz_batch *B, int mode, cudaStream_t s)
{
    if (mode == B->mode) return BZ_OK;
    for (int i = 0; i < B->n; ++i) {
        bz_handle *h = B->inst[i];
        const size_t mb = sizeof(float) * 8 * (size_t)h->g.nr;
        if (B->mode != 0) {       // leaving a mode whose states carry pending corrections
            const int b = (int)(B->step[i] & 1);
            bzk::k_lz_materialize<<<std::min(h->g.nr, h->nsm * 8), 256, 0, s>>>(
                h->g, nullptr, (const float *)h->h[b], h->mu[b], (float *)h->h[b], nullptr);
            BZ_CUDA(cudaGetLastError());
        }
        BZ_CUDA(cudaMemsetAsync(h->mu[0], 0, mb, s));
        BZ_CUDA(cudaMemsetAsync(h->mu[1], 0, mb, s));
        h->lazy_buf[0] = h->lazy_buf[1] = false;
    }
    B->mode = mode;
    return BZ_OK;
}

// Fan-out mode keeps states with pending corrections: apply them in place
// (the value is unchanged) before instance i's state is read.
bz_status batch_correct_in_place(bz_batch *B, int i, cudaStream_t s)
{
    if (B->mode == 0) return BZ_OK;
    bz_handle *h = B->inst[i];
    const int b = (int)(B->step[i] & 1);
    bzk::k_lz_materialize<<<std::min(h->g.nr, h->nsm * 8), 256, 0, s>>>(
        h->g, nullptr, (const float *)h->h[b], h->mu[b], (float *)h->h[b], nullptr);
    BZ_CUDA(cudaGetLastError());
    BZ_CUDA(cudaMemsetAsync(h->mu[b], 0, sizeof(float) * 8 * (size_t)h->g.nr, s));
    return BZ_OK;
}

// One fan-out step: fork to the branches, each instance's active-node step
// on its branch (advance: the step counter moves on; else a repeatable trial),
// join back to s.
bz_status fan_launch(bz_batch *B, cudaStream_t s, bool advance_step)
{
    const int nb = B->branches;
    BZ_CUDA(cudaEventRecord(B->ev[0], s));
    for (int k = 0; k < nb; ++k) BZ_CUDA(cudaStreamWaitEvent(B->br[k], B->ev[0], 0));
    for (int i = 0; i < B->n; ++i) {
        bz_handle *h = B->inst[i];
        h->cur = (int)(B->step[i] & 1);
        h->step = B->step[i];
        BZ_TRY(launch_lazy(h, B->br[B->owner[i]], advance_step, false, h->ahead_K > 0));
    }
    for (int k = 0; k < nb; ++k) {
        BZ_CUDA(cudaEventRecord(B->ev[1 + k], B->br[k]));
        BZ_CUDA(cudaStreamWaitEvent(s, B->ev[1 + k], 0));
    }
    return BZ_OK;
}

// The plans of the instances' current steps built ahead where their slots do
// not cover them yet (the instances step together, so they all need a batch
// at the same steps): each instance's batch on its branch, forked from and
// joined back to s.  Never called while a stream is being captured.
bz_status fan_ensure(bz_batch *B, cudaStream_t s)
{
    bool need = false;
    for (int i = 0; i < B->n && !need; ++i) {
        const bz_handle *h = B->inst[i];
        need = h->lazy && h->ahead_K > 0 && !(B->step[i] >= h->ahead_lo && B->step[i] + 1 <= h->ahead_hi);
    }
    if (!need) return BZ_OK;
    const int nb = B->branches;
    BZ_CUDA(cudaEventRecord(B->ev[0], s));
    for (int k = 0; k < nb; ++k) BZ_CUDA(cudaStreamWaitEvent(B->br[k], B->ev[0], 0));
    for (int i = 0; i < B->n; ++i) BZ_TRY(ensure_plans(B->inst[i], B->br[B->owner[i]], B->step[i], 1));
    for (int k = 0; k < nb; ++k) {
        BZ_CUDA(cudaEventRecord(B->ev[1 + k], B->br[k]));
        BZ_CUDA(cudaStreamWaitEvent(s, B->ev[1 + k], 0));
    }
    return BZ_OK;
}

// Graph of one fan-out step for the instances' current step parities.
bz_status fan_graph(bz_batch *B, cudaGraphExec_t *out)
{
    std::vector<int> key(B->n);
    for (int i = 0; i < B->n; ++i) key[i] = (int)(B->step[i] & 1);
    for (int k = 0; k < 2; ++k)
        if (B->fgraph[k] && B->fkey[k] == key) {
            *out = B->fgraph[k];
            return BZ_OK;
        }
    std::vector<int> cur0(B->n);
    std::vector<int64_t> st0(B->n);
    std::vector<long long> l0(B->n);
    for (int i = 0; i < B->n; ++i) {
        cur0[i] = B->inst[i]->cur;
        st0[i] = B->inst[i]->step;
        l0[i] = B->inst[i]->launches;
    }
    BZ_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
    bz_status st = fan_launch(B, B->cap, true);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(B->cap, &graph);
    for (int i = 0; i < B->n; ++i) {           // capturing ran no step
        B->inst[i]->cur = cur0[i];
        B->inst[i]->step = st0[i];
        B->inst[i]->launches = l0[i];
    }
    if (st != BZ_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail(BZ_ECUDA, "batch capture failed: %s", cudaGetErrorString(e));
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(BZ_ECUDA, "batch graph: %s", cudaGetErrorString(e));
    const int slot = B->fgraph[0] ? (B->fgraph[1] ? 0 : 1) : 0;
    if (B->fgraph[slot]) cudaGraphExecDestroy(B->fgraph[slot]);
    B->fgraph[slot] = ex;
    B->fkey[slot] = key;
    *out = ex;
    return BZ_OK;
}

bz_status batch_launch(bz_batch *B, cudaStream_t s, bool advance)
{
    const int pb = 256;
    bzk::kb_walls<<<B->tot_faces, bzk::kWallThreads, 0, s>>>(B->d_inst, B->d_face_pre, B->n);
    bzk::kb_plan<<<(B->tot_samples + pb - 1) / pb, pb, 0, s>>>(B->d_inst, B->d_samp_pre, B->n);
    bzk::kb_scatter_scan<<<B->n, 1024, 0, s>>>(B->d_inst, B->maxt);
    bzk::kb_scatter_fill<<<(B->tot_samples + pb - 1) / pb, pb, 0, s>>>(B->d_inst, B->d_samp_pre,
                                                                        B->n, B->maxt);
    if (B->maxt == 512)
        bzk::kb_cell4<512><<<B->grid, 512, B->smem, s>>>(B->d_inst, B->d_cell_pre, B->n);
    else
        bzk::kb_cell4<1024><<<B->grid, 1024, B->smem, s>>>(B->d_inst, B->d_cell_pre, B->n);
    if (advance) bzk::kb_advance<<<(B->n + 127) / 128, 128, 0, s>>>(B->d_inst, B->n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BZ_ECUDA, "batch launch failed: %s", cudaGetErrorString(e));
    return BZ_OK;
}

}  // namespace

extern "C" {

// One step of every instance in the persistent active-node mode (advance =
// false: a repeatable recomputation of the current step).
bz_status lz_batch_launch(bz_batch *B, cudaStream_t s, bool advance)
{
    const int pb = 256, sg = (B->tot_samples + pb - 1) / pb;
    // The sample plans depend on the step counters only: they run on a side
    // stream beside the walls (after everything before the step on s).
    BZ_CUDA(cudaEventRecord(B->lz_fork, s));
    BZ_CUDA(cudaStreamWaitEvent(B->lz_side, B->lz_fork, 0));
    const cudaStream_t sp = B->lz_side;
    if (B->lz_ahead) {
        // Each instance's plan copied from its slots (the batches are built
        // ahead by the caller of this launch, outside any capture).
        bzk::kbl_take<<<dim3(8, B->n), 256, 0, sp>>>(B->d_lzinst);
    } else {
        bzk::kbl_plan<<<sg, pb, 0, sp>>>(B->d_lzinst, B->d_samp_pre, B->n);
        bzk::kbl_scan<<<B->n, 1024, 0, sp>>>(B->d_lzinst);
        bzk::kbl_remap<<<sg, pb, 0, sp>>>(B->d_lzinst, B->d_samp_pre, B->n);
        bzk::kbl_lscan<<<B->n, 1024, 0, sp>>>(B->d_lzinst);
        bzk::kbl_lfill<<<sg, pb, 0, sp>>>(B->d_lzinst, B->d_samp_pre, B->n);
    }
    BZ_CUDA(cudaEventRecord(B->lz_join, sp));
    bzk::kbl_walls<<<B->tot_faces, bzk::kWallThreads, 0, s>>>(B->d_lzinst, B->d_face_pre, B->n);
    BZ_CUDA(cudaMemsetAsync(B->d_next, 0, sizeof(int) * B->lz_classes.size(), s));
    BZ_CUDA(cudaStreamWaitEvent(s, B->lz_join, 0));
    const size_t nc = B->lz_classes.size();
    if (nc > 1) BZ_CUDA(cudaEventRecord(B->lz_go, s));
    for (size_t k = 0; k < nc; ++k) {
        const auto &c = B->lz_classes[k];
        const int4 *sg4 = B->d_segs + c.seg0;
        int *nx = B->d_next + k;
        const cudaStream_t sk = k == 0 ? s : B->lz_cls_s[k - 1];
        if (k > 0) BZ_CUDA(cudaStreamWaitEvent(sk, B->lz_go, 0));
        switch (c.nv) {
        case 24: bzk::kbl_lz<24><<<B->nsm, bzk::kLzThreads, c.smem, sk>>>(B->d_lzinst, sg4, c.nseg, nx); break;
        case 20: bzk::kbl_lz<20><<<B->nsm, bzk::kLzThreads, c.smem, sk>>>(B->d_lzinst, sg4, c.nseg, nx); break;
        case 16: bzk::kbl_lz<16><<<B->nsm, bzk::kLzThreads, c.smem, sk>>>(B->d_lzinst, sg4, c.nseg, nx); break;
        default: bzk::kbl_lz<0><<<B->nsm, bzk::kLzThreads, c.smem, sk>>>(B->d_lzinst, sg4, c.nseg, nx); break;
        }
        if (k > 0) BZ_CUDA(cudaEventRecord(B->lz_cls_done[k - 1], sk));
    }
    for (size_t k = 1; k < nc; ++k) BZ_CUDA(cudaStreamWaitEvent(s, B->lz_cls_done[k - 1], 0));
    // The 4-node-vector fallback of instances that overflowed (no work otherwise).
    bzk::kbl_fb_plan<<<sg, pb, 0, s>>>(B->d_lzinst, B->d_samp_pre, B->n);
    bzk::kbl_fb_scan<<<B->n, 1024, 0, s>>>(B->d_lzinst, 512);
    bzk::kbl_fb_fill<<<sg, pb, 0, s>>>(B->d_lzinst, B->d_samp_pre, B->n, 512);
    bzk::kbl_fb_materialize<<<std::min(B->tot_cells, B->nsm * 8), 256, 0, s>>>(B->d_lzinst, B->d_cell_pre,
                                                                              B->n);
    bzk::kbl_fb_cell4<<<B->nsm, 512, B->smem, s>>>(B->d_lzinst, B->d_cell_pre, B->n);
    if (advance) bzk::kbl_advance<<<(B->n + 127) / 128, 128, 0, s>>>(B->d_lzinst, B->n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BZ_ECUDA, "batch launch failed: %s", cudaGetErrorString(e));
    return BZ_OK;
}

// Set-up of the persistent active-node mode (lz_ok stays false when an
// instance does not run the active-node kernel with groups of four cells).
bz_status lz_batch_prepare(bz_batch *B)
{
    B->lz_ok = false;
    for (bz_handle *h : B->inst)
        if (!h->lazy || h->lz_G != 4) return BZ_OK;
    const int n = B->n;
    std::vector<bzk::LzInst> li(n);
    size_t smem = 0;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) {
        bz_handle *h = B->inst[i];
        bzk::LzInst &b = li[i];
        b.g = h->g;
        b.step = h->d_step;
        for (int p = 0; p < 2; ++p) {
            b.h[p] = (float *)h->h[p];
            b.mu[p] = h->mu[p];
        }
        b.ghost = (float *)h->ghost;
        b.nw = h->nw;
        b.idx = h->lz_idx;
        b.pa = h->lz_pa;
        b.qc = h->lz_qc;
        b.flag = h->lz_flag;
        b.cidx = h->lz_cidx;
        b.count = h->lz_count;
        b.cursor = h->lz_cursor;
        b.rowend = h->lz_rowend;
        b.map = map_for(h->g.nv, 512);
        b.pidx16 = (ushort4 *)h->pidx;
        b.pa16 = (bzk::PlanA<float, uint16_t> *)h->pa;
        b.sc_count = h->sc_count;
        b.sc_cursor = h->sc_cursor;
        b.sc_meta = h->sc_meta;
        b.sc_ent = h->sc_ent;
        b.ahead = h->ahead;
        if (h->ahead_K == 0) b.ahead.K = 0;
        for (int p = 0; p < 2; ++p) {
            bzk::LzArgs &a = b.a[p];
            a = bzk::LzArgs{};
            a.hin = b.h[p];
            a.mu_in = b.mu[p];
            a.ghost = b.ghost;
            a.hout = b.h[p ^ 1];
            a.mu_out = b.mu[p ^ 1];
            a.mom = h->mom;
            a.rec = h->lz_rec;
            a.dest0 = h->lz_dest0;
            a.meta = h->lz_meta;
            a.mask = h->lz_mask;
            a.wpre = h->lz_wpre;
            a.act = h->lz_act;
            a.mcap = h->lz_mcap;
            for (int k = 0; k < bzk::kLzX; ++k) a.e0[k] = h->lz_e0[k];
            a.stats = h->stats;
            a.early_tail = h->g.nv < 32 ? 1 : 0;
        }
        smem = std::max(smem, (size_t)bzk::lz_offsets(h->g.nvt, h->lz_mcap, 4).end);
        order[i] = i;
    }
    // Segments of about 32 groups: R strided lanes r, r + R, ... of each
    // instance's groups, the instances with the largest velocity grids (the
    // costliest groups) first.
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return B->inst[x]->g.nv > B->inst[y]->g.nv;
    });
    std::vector<int4> segs;
    B->lz_classes.clear();
    for (int i : order) {
        const int nv = B->inst[i]->g.nv;
        const int key = nv == 24 || nv == 20 || nv == 16 ? nv : 0;
        if (B->lz_classes.empty() || B->lz_classes.back().nv != key)
            B->lz_classes.push_back({key, (int)segs.size(), 0, 0});
        auto &c = B->lz_classes.back();
        c.smem = std::max(c.smem, (size_t)bzk::lz_offsets(B->inst[i]->g.nvt, B->inst[i]->lz_mcap, 4).end);
        const int ng = (B->inst[i]->g.nr + 3) / 4, R = std::max(1, (ng + 31) / 32);
        for (int r = 0; r < R && r < ng; ++r) segs.push_back(make_int4(i, r, (ng - 1 - r) / R + 1, R));
        c.nseg = (int)segs.size() - c.seg0;
    }
    bz_handle *h0 = B->inst[0];
    BZ_CUDA(bz_allow_max_smem(bzk::kbl_lz<24>, h0->smem_optin));
    BZ_CUDA(bz_allow_max_smem(bzk::kbl_lz<20>, h0->smem_optin));
    BZ_CUDA(bz_allow_max_smem(bzk::kbl_lz<16>, h0->smem_optin));
    BZ_CUDA(bz_allow_max_smem(bzk::kbl_lz<0>, h0->smem_optin));
    BZ_CUDA(bz_allow_max_smem(bzk::kbl_fb_cell4, h0->smem_optin));
    int occ = 0, occ4 = 0;
    BZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bzk::kbl_lz<0>, bzk::kLzThreads, smem));
    BZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ4, bzk::kbl_fb_cell4, 512, B->smem));
    if (occ < 1 || occ4 < 1) return BZ_OK;
    BZ_TRY(dalloc(&B->d_lzinst, sizeof(bzk::LzInst) * n));
    BZ_TRY(dalloc(&B->d_segs, sizeof(int4) * segs.size()));
    BZ_TRY(dalloc(&B->d_next, sizeof(int) * B->lz_classes.size()));
    BZ_CUDA(cudaMemcpy(B->d_lzinst, li.data(), sizeof(bzk::LzInst) * n, cudaMemcpyHostToDevice));
    BZ_CUDA(cudaMemcpy(B->d_segs, segs.data(), sizeof(int4) * segs.size(), cudaMemcpyHostToDevice));
    {
        int least = 0, greatest = 0;
        BZ_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        BZ_CUDA(cudaStreamCreateWithPriority(&B->lz_side, cudaStreamNonBlocking, greatest));
        BZ_CUDA(cudaEventCreateWithFlags(&B->lz_fork, cudaEventDisableTiming));
        BZ_CUDA(cudaEventCreateWithFlags(&B->lz_join, cudaEventDisableTiming));
        BZ_CUDA(cudaEventCreateWithFlags(&B->lz_go, cudaEventDisableTiming));
        for (size_t k = 1; k < B->lz_classes.size(); ++k) {
            cudaStream_t x = nullptr;
            cudaEvent_t e = nullptr;
            BZ_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
            B->lz_cls_s.push_back(x);
            BZ_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            B->lz_cls_done.push_back(e);
        }
    }
    B->nseg = (int)segs.size();
    B->lz_smem = smem;
    B->lz_ok = true;
    // With every instance's plans built ahead (the default) the step copies
    // them (BZ_BATCH_LZ_AHEAD=0: every step builds them in the step).
    B->lz_ahead = true;
    for (bz_handle *h : B->inst) B->lz_ahead = B->lz_ahead && h->ahead_K > 0;
    if (const char *e = getenv("BZ_BATCH_LZ_AHEAD")) B->lz_ahead = B->lz_ahead && atoi(e) != 0;
    return BZ_OK;
}

bz_status bz_batch_create(int32_t n, const bz_space *spaces, const bz_vel *vels,
                          const bz_walls *walls, const bz_params *params, bz_batch **out)
{
    g_last_error.clear();
    if (!out) return fail(BZ_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 4096) return fail(BZ_EINVAL, "n must be in [1, 4096]");
    if (!spaces || !vels || !walls || !params) return fail(BZ_EINVAL, "NULL argument");
    for (int i = 0; i < n; ++i) {
        if (params[i].dtype != BZ_F32) return fail(BZ_EUNSUPPORTED, "instance %d: batches are FP32", i);
        if (params[i].sample_mode != BZ_SHARED)
            return fail(BZ_EUNSUPPORTED, "instance %d: batches use the shared sample set", i);
        if ((vels[i].rv > 0.0 && vels[i].rv < 1.0) || (spaces[i].rx > 0.0 && spaces[i].rx < 1.0) ||
            (spaces[i].ry > 0.0 && spaces[i].ry < 1.0))
            return fail(BZ_EUNSUPPORTED, "instance %d: batches use uniform grids", i);
        if (vels[i].nv % 4 != 0 || vels[i].nv < 12)
            return fail(BZ_EUNSUPPORTED, "instance %d: nv must be a multiple of 4, >= 12", i);
        if (params[i].n_pairs > 32768)
            return fail(BZ_EUNSUPPORTED, "instance %d: at most 32768 samples per step", i);
    }
    bz_batch *B = new bz_batch();
    auto bail = [&](bz_status st) {
        std::string msg = g_last_error;
        batch_free(B);
        delete B;
        g_last_error = msg;
        return st;
    };
    B->n = n;
    size_t smem = 0;
    std::vector<int> cpre(n + 1, 0), fpre(n + 1, 0), spre(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        bz_handle *h = nullptr;
        bz_status st = bz_create(spaces + i, vels + i, walls + i, params + i, &h);
        if (st != BZ_OK) return bail(st);
        B->inst.push_back(h);
        if (!h->fast) {
            fail(BZ_EUNSUPPORTED, "instance %d does not fit the FP32 per-cell kernel", i);
            return bail(BZ_EUNSUPPORTED);
        }
        bzk::BInst b{};
        b.g = h->g;
        b.map[0] = map_for(h->g.nv, 512);
        b.map[1] = map_for(h->g.nv, 1024);
        b.h[0] = (float *)h->h[0];
        b.h[1] = (float *)h->h[1];
        b.ghost = (float *)h->ghost;
        b.nw = h->nw;
        b.pidx = (ushort4 *)h->pidx;
        b.pa = (bzk::PlanA<float, uint16_t> *)h->pa;
        b.sc_count = h->sc_count;
        b.sc_cursor = h->sc_cursor;
        b.sc_meta = h->sc_meta;
        b.sc_ent = h->sc_ent;
        b.mom = h->mom;
        b.step = h->d_step;
        B->hinst.push_back(b);
        cpre[i + 1] = cpre[i] + h->g.nr;
        fpre[i + 1] = fpre[i] + h->g.nfaces;
        spre[i + 1] = spre[i] + h->g.nt;
        smem = std::max(smem, bzk::cell4_smem_bytes(h->g.nv, h->g.nvt, h->g.nt));
        if (cudaMemset(h->sc_count, 0, sizeof(int) * h->g.nvt) != cudaSuccess) {
            fail(BZ_ECUDA, "memset failed");
            return bail(BZ_ECUDA);
        }
    }
    B->tot_cells = cpre[n];
    B->tot_faces = fpre[n];
    B->tot_samples = spre[n];
    B->nsm = B->inst[0]->nsm;
    B->smem = smem;
    B->step.assign(n, 0);
    bz_status st = dalloc(&B->d_inst, sizeof(bzk::BInst) * n);
    if (st == BZ_OK) st = dalloc(&B->d_cell_pre, sizeof(int) * (n + 1));
    if (st == BZ_OK) st = dalloc(&B->d_face_pre, sizeof(int) * (n + 1));
    if (st == BZ_OK) st = dalloc(&B->d_samp_pre, sizeof(int) * (n + 1));
    if (st != BZ_OK) return bail(st);
    cudaError_t e = cudaMemcpy(B->d_cell_pre, cpre.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_face_pre, fpre.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_samp_pre, spre.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        fail(BZ_ECUDA, "batch set-up failed: %s", cudaGetErrorString(e));
        return bail(BZ_ECUDA);
    }
    // Default schedule: two 512-thread CTAs per SM when they fit, else one of 1024.
    int occ512 = 0;
    st = batch_occupancy<512>(B, &occ512);
    if (st == BZ_OK) st = occ512 >= 2 ? batch_apply(B, 512, 2, 8) : batch_apply(B, 1024, 1, 8);
    if (st != BZ_OK) return bail(st);
    // Fan-out mode: branch streams and their fork / join events.
    B->fan_ok = true;
    for (bz_handle *h : B->inst) B->fan_ok = B->fan_ok && h->lazy;
    B->br.assign(kMaxBranches, nullptr);
    B->ev.assign(kMaxBranches + 1, nullptr);
    for (auto &st2 : B->br)
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking);
    for (auto &ev : B->ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        fail(BZ_ECUDA, "batch set-up failed: %s", cudaGetErrorString(e));
        return bail(BZ_ECUDA);
    }
    assign_branches(B, 4);
    st = lz_batch_prepare(B);
    if (st != BZ_OK) return bail(st);
    if (const char *m = getenv("BZ_BATCH_MODE")) {
        const int want = strcmp(m, "fanout") == 0 && B->fan_ok ? 1 : (strcmp(m, "lz") == 0 && B->lz_ok ? 2 : 0);
        if (want) {
            st = batch_set_mode(B, want, nullptr);
            if (st == BZ_OK) st = cudaDeviceSynchronize() == cudaSuccess ? BZ_OK : BZ_ECUDA;
            if (st != BZ_OK) return bail(st);
        }
    }
    *out = B;
    return BZ_OK;
}

bz_status bz_batch_destroy(bz_batch *B)
{
    if (!B) return BZ_OK;
    cudaDeviceSynchronize();
    batch_free(B);
    delete B;
    return BZ_OK;
}

bz_status bz_batch_step(bz_batch *B, int32_t nsteps, void *stream)
{
    if (!B) return fail(BZ_EINVAL, "batch is NULL");
    if (nsteps < 0) return fail(BZ_EINVAL, "nsteps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (B->mode == 2) {
        if (nsteps > 0 && graphs_enabled() && !B->graph2) {
            BZ_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
            bz_status st = lz_batch_launch(B, B->cap, true);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(B->cap, &graph);
            if (st != BZ_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (e != cudaSuccess) return fail(BZ_ECUDA, "batch capture failed: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&B->graph2, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return fail(BZ_ECUDA, "batch graph: %s", cudaGetErrorString(e));
        }
        for (int32_t k = 0; k < nsteps; ++k) {
            if (B->lz_ahead) BZ_TRY(fan_ensure(B, s));
            if (B->graph2 && graphs_enabled()) BZ_CUDA(cudaGraphLaunch(B->graph2, s));
            else BZ_TRY(lz_batch_launch(B, s, true));
            for (auto &v : B->step) v += 1;
        }
        for (int i = 0; i < B->n; ++i) {
            bz_handle *h = B->inst[i];
            h->step = B->step[i];
            h->cur = (int)(h->step & 1);
            if (nsteps > 0) {
                h->lazy_buf[h->cur] = true;
                h->mom_valid = true;
            }
        }
        return BZ_OK;
    }
    if (B->mode == 1) {
        for (int32_t k = 0; k < nsteps; ++k) {
            BZ_TRY(fan_ensure(B, s));
            if (graphs_enabled()) {
                cudaGraphExec_t ex = nullptr;
                BZ_TRY(fan_graph(B, &ex));
                BZ_CUDA(cudaGraphLaunch(ex, s));
                for (int i = 0; i < B->n; ++i) {
                    bz_handle *h = B->inst[i];
                    h->launches += 14;
                    h->step = B->step[i] + 1;
                    h->cur = (int)(h->step & 1);
                    h->lazy_buf[h->cur] = true;
                    h->mom_valid = true;
                }
            } else {
                BZ_TRY(fan_launch(B, s, true));
            }
            for (auto &v : B->step) v += 1;
        }
        return BZ_OK;
    }
    if (nsteps > 0 && graphs_enabled()) {
        if (!B->graph) {
            BZ_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
            bz_status st = batch_launch(B, B->cap, true);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(B->cap, &graph);
            if (st != BZ_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (e != cudaSuccess) return fail(BZ_ECUDA, "batch capture failed: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&B->graph, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return fail(BZ_ECUDA, "batch graph: %s", cudaGetErrorString(e));
        }
        for (int32_t k = 0; k < nsteps; ++k) BZ_CUDA(cudaGraphLaunch(B->graph, s));
    } else {
        for (int32_t k = 0; k < nsteps; ++k) BZ_TRY(batch_launch(B, s, true));
    }
    for (auto &v : B->step) v += nsteps;
    return BZ_OK;
}

bz_status bz_batch_set_state(bz_batch *B, int32_t i, const void *src, int64_t step, void *stream)
{
    if (!B || i < 0 || i >= B->n || !src || step < 0) return fail(BZ_EINVAL, "invalid argument");
    bz_handle *h = B->inst[i];
    cudaStream_t s = (cudaStream_t)stream;
    BZ_CUDA(cudaMemcpyAsync(h->h[step & 1], src, h->esz * (size_t)h->g.nr * h->g.nvt,
                            cudaMemcpyDefault, s));
    if (h->mu[step & 1])                       // a new state has no pending corrections
        BZ_CUDA(cudaMemsetAsync(h->mu[step & 1], 0, sizeof(float) * 8 * (size_t)h->g.nr, s));
    BZ_CUDA(cudaMemcpyAsync(h->d_step, &step, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    BZ_CUDA(cudaStreamSynchronize(s));
    B->step[i] = step;
    return BZ_OK;
}

bz_status bz_batch_get_state(bz_batch *B, int32_t i, void *dst, int64_t *step, void *stream)
{
    if (!B || i < 0 || i >= B->n || !dst) return fail(BZ_EINVAL, "invalid argument");
    bz_handle *h = B->inst[i];
    BZ_TRY(batch_correct_in_place(B, i, (cudaStream_t)stream));
    BZ_CUDA(cudaMemcpyAsync(dst, h->h[B->step[i] & 1], h->esz * (size_t)h->g.nr * h->g.nvt,
                            cudaMemcpyDefault, (cudaStream_t)stream));
    if (step) *step = B->step[i];
    return BZ_OK;
}

bz_status bz_batch_moments(bz_batch *B, int32_t i, double *out, void *stream)
{
    if (!B || i < 0 || i >= B->n || !out) return fail(BZ_EINVAL, "invalid argument");
    bz_handle *h = B->inst[i];
    cudaStream_t s = (cudaStream_t)stream;
    const Geo &g = h->g;
    BZ_TRY(batch_correct_in_place(B, i, s));
    bzk::k_moments<float><<<std::min(g.nr, h->nsm * 8), 256, 0, s>>>(
        g, (const float *)h->h[B->step[i] & 1], h->mom);
    BZ_CUDA(cudaGetLastError());
    BZ_CUDA(cudaMemcpyAsync(out, h->mom, sizeof(double) * 11 * (size_t)g.nr, cudaMemcpyDefault, s));
    BZ_CUDA(cudaStreamSynchronize(s));
    return BZ_OK;
}

bz_status bz_batch_tune(bz_batch *B, int32_t trial_steps, void *stream, int32_t *choice,
                        double *ms, int32_t *ncand)
{
    if (!B || trial_steps < 1) return fail(BZ_EINVAL, "invalid argument");
    cudaStream_t s = (cudaStream_t)stream;
    // Candidates: the persistent kernels (threads per CTA, CTAs per SM, strip
    // width), then fan-out graphs of the instances' own steps (branches).
    struct Cand { int mode, maxt, cps, strip, branches; };
    std::vector<Cand> cands;
    for (int maxt : {512, 1024})
        for (int cps : {1, 2})
            for (int strip : {4, 8, 16}) {
                if (maxt == 1024 && cps == 2) continue;   // 64 registers x 2048 threads do not fit
                cands.push_back({0, maxt, cps, strip, 0});
            }
    if (B->fan_ok)
        for (int nb : {1, 2, 4, 8}) cands.push_back({1, 0, 0, 0, nb});
    if (B->lz_ok) cands.push_back({2, 0, 0, 0, 0});
    cudaEvent_t e0, e1;
    BZ_CUDA(cudaEventCreate(&e0));
    BZ_CUDA(cudaEventCreate(&e1));
    int best = -1;
    double best_ms = 1e300;
    for (size_t c = 0; c < cands.size(); ++c) {
        const Cand &k = cands[c];
        double t = -1.0;
        if (k.mode == 0) {
            if (batch_set_mode(B, 0, s) == BZ_OK &&
                batch_apply(B, k.maxt, k.cps, k.strip) == BZ_OK && batch_launch(B, s, false) == BZ_OK) {
                cudaEventRecord(e0, s);
                bool ok = true;
                for (int r = 0; r < trial_steps && ok; ++r) ok = batch_launch(B, s, false) == BZ_OK;
                cudaEventRecord(e1, s);
                float f = 0.f;
                if (ok && cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&f, e0, e1) == cudaSuccess)
                    t = f / trial_steps;
            }
        } else if (k.mode == 2) {
            if (batch_set_mode(B, 2, s) == BZ_OK && (!B->lz_ahead || fan_ensure(B, s) == BZ_OK) &&
                lz_batch_launch(B, s, false) == BZ_OK) {
                cudaEventRecord(e0, s);
                bool ok = true;
                for (int r = 0; r < trial_steps && ok; ++r) ok = lz_batch_launch(B, s, false) == BZ_OK;
                cudaEventRecord(e1, s);
                float f = 0.f;
                if (ok && cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&f, e0, e1) == cudaSuccess)
                    t = f / trial_steps;
            }
        } else if (batch_set_mode(B, 1, s) == BZ_OK) {
            // A graph of one repeatable (non-advancing) fan-out step.
            assign_branches(B, k.branches);
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t ex = nullptr;
            std::vector<long long> l0(B->n);
            for (int i = 0; i < B->n; ++i) l0[i] = B->inst[i]->launches;
            bool ok = fan_ensure(B, s) == BZ_OK &&
                      cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            bz_status st = ok ? fan_launch(B, B->cap, false) : BZ_ECUDA;
            ok = cudaStreamEndCapture(B->cap, &graph) == cudaSuccess && ok && st == BZ_OK;
            for (int i = 0; i < B->n; ++i) B->inst[i]->launches = l0[i];
            ok = ok && cudaGraphInstantiate(&ex, graph, 0) == cudaSuccess;
            if (graph) cudaGraphDestroy(graph);
            if (ok && cudaGraphLaunch(ex, s) == cudaSuccess) {
                cudaEventRecord(e0, s);
                for (int r = 0; r < trial_steps && ok; ++r) ok = cudaGraphLaunch(ex, s) == cudaSuccess;
                cudaEventRecord(e1, s);
                float f = 0.f;
                if (ok && cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&f, e0, e1) == cudaSuccess)
                    t = f / trial_steps;
            }
            if (ex) cudaGraphExecDestroy(ex);
        }
        if (ms && c < 16) ms[c] = t;
        if (t > 0.0 && t < best_ms) {
            best_ms = t;
            best = (int)c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ncand) *ncand = (int32_t)cands.size();
    if (best < 0) return fail(BZ_ECUDA, "no schedule could be timed");
    const Cand &k = cands[best];
    BZ_TRY(batch_set_mode(B, k.mode, s));
    if (k.mode == 0) {
        BZ_TRY(batch_apply(B, k.maxt, k.cps, k.strip));
    } else if (k.mode == 1) {
        assign_branches(B, k.branches);
        drop_fan_graphs(B);
    }
    if (choice) *choice = best;
    return BZ_OK;
}

bz_status bz_batch_schedule(const bz_batch *B, int32_t out[4])
{
    if (!B || !out) return fail(BZ_EINVAL, "invalid argument");
    out[0] = B->maxt;
    out[1] = B->grid;
    out[2] = B->strip;
    out[3] = B->mode == 1 ? B->branches : (B->mode == 2 ? -1 : 0);
    return BZ_OK;
}

}  // extern "C"
