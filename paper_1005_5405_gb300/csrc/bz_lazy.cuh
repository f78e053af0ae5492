// bz_lazy.cuh -- FP32 step on the active velocity nodes, correction deferred.
//
// Same mathematics as k_cell4 (Eqs. streaming2D, monteCarloInt,
// collision_step, rinorm_a, correzione, densita..sforzi), organised around two
// facts:
//
// * The Monte Carlo terms of a step touch only the nodes that one of its
//   shared samples maps to (v, v1, v*, v1*): for Maxwellian draws a small
//   fraction of the grid (about 7% of 32^3 at 2x10^4 samples).  Every other
//   node keeps h_c = h~.  The per-step plan lists those "active" nodes once
//   (compact index m), and the collision terms of every cell work on arrays
//   of M entries instead of the whole velocity slab.
// * The correction h^{n+1} = h_c + (1 + eps h_c)(mu . psi) needs mu, which
//   needs the moments of every node.  Instead of holding the whole slab until
//   mu is known, the step stores h_c and the cell's mu; whoever reads the
//   state next (the next step's streaming, the walls, a state copy) applies
//   the correction on the fly.  The state is therefore the pair (h_c, mu);
//   mu = 0 is an ordinary state.
//
// Without the slab a CTA needs two compact arrays, so two CTAs share an SM
// and each works on G cells at once: the G values of a node are adjacent, so
// one vector access serves all G cells and every collision term is decoded
// once per G cells.
//
// The collision terms are applied as a pull: the plan sorts the terms
// (destination, sample, sign) by destination and gives each thread a run of
// them; a term carries the byte offsets of the sample's two pre-collision
// nodes and its signed weight, so the thread recomputes the sample's product
// from h~ and sums a destination's terms in registers.  Floating-point
// arithmetic on node pairs uses the packed FP32x2 instructions.
//
// The conserved-moment sums of N_c and the output moments come from 26
// monomial sums (degree <= 4) of N = w h~ over all nodes, taken while
// streaming, plus the same sums of the collision increment over the active
// nodes.  If a step has more active nodes than the kernel's arrays hold
// (mcap), the kernel returns at once and the k_cell4 path computes the step.
#pragma once

#include "bz_cell4.cuh"

#include <type_traits>

namespace bzk {

constexpr int kLzMono = 26;        // monomial sums per cell
constexpr int kLzX = 30;           // with v^2, v_x v^2, v_y v^2, v_z v^2
constexpr int kLzRoleT = 256;      // threads of each role: streaming, collision
constexpr int kLzThreads = 2 * kLzRoleT;
constexpr int kLzRoleWarps = kLzRoleT / 32;
constexpr int kLzMaxG = 4;         // cells per CTA group
constexpr int kLzMaxN = 32;        // velocity nodes per axis (N^2 / 4 <= kLzRoleT)
constexpr int kLzStages = 5;       // streaming stages staged per thread
constexpr unsigned long long kLzWaitNs = 1000000000ull;   // an mbarrier wait gives up after 1 s

// meta layout: [0] M, [1] overflow (M > mcap), [2] E (terms of the step),
// [3] C (terms per thread).
constexpr int kLzMetaSize = 4;

// Planes per streaming stage: the largest divisor K of N/2 with K N^2/4 <=
// kLzRoleT (one node quad per streaming thread; stages never straddle jx =
// N/2, so the upwind x source is the same cell for the whole stage).  0:
// unsupported.
__host__ __device__ constexpr int lz_planes4(int N)
{
    int K = 0;
    for (int k = 1; k <= N / 2; ++k)
        if ((N / 2) % k == 0 && k * (N * N / 4) <= kLzRoleT) K = k;
    return K;
}

// ---------------------------------------------------------------------
// Per-step plan (once per step; every cell shares it)
// ---------------------------------------------------------------------

// Marks every node a sample of the step maps to.
static __global__ void k_lz_mark(int nt, const int4 *__restrict__ idx, int *__restrict__ flag)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nt) return;
    const int4 q = idx[l];
    if (q.x >= 0) flag[q.x] = 1;
    if (q.y >= 0) flag[q.y] = 1;
    if (q.z >= 0) flag[q.z] = 1;
    if (q.w >= 0) flag[q.w] = 1;
}

// Compact numbering of the marked nodes (ascending node order), one CTA of
// 1024 threads: cidx[j] = m, act[m] = j, the bit mask of marked nodes and, per
// 32-node word, the compact index of its first marked node.  Clears the flags.
// Each warp forms 32 mask words from coalesced flag loads (one ballot per
// word), lane k keeping word k; warp and block scans of the word counts
// give the compact indices.
// stats (nullable): [5] counts steps whose active set exceeded mcap.
__device__ __forceinline__ void lz_scan_block(int nvt, int mcap, int *__restrict__ flag, int *__restrict__ cidx,
                                              int *__restrict__ act, uint32_t *__restrict__ mask,
                                              int *__restrict__ wpre, int *__restrict__ meta,
                                              unsigned long long *__restrict__ stats)
{
    __shared__ int wsum[32];
    __shared__ int btot;
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5, nw = nvt / 32;
    int carry = 0;
    for (int b0 = 0; b0 < nw; b0 += 1024) {
        const int base = b0 + wp * 32;                // this warp's 32 words
        uint32_t bits = 0;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const int w = base + k;
            const bool set = w < nw && flag[w * 32 + lane] != 0;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, set);
            if (lane == k) bits = bal;
        }
        const int w = base + lane, cnt = __popc(bits);
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) wsum[wp] = inc;
        __syncthreads();
        if (wp == 0) {
            const int x0 = wsum[lane];
            int x = x0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= o) x += v;
            }
            wsum[lane] = x - x0;
            if (lane == 31) btot = x;
        }
        __syncthreads();
        int run = carry + wsum[wp] + inc - cnt;
        carry += btot;
        __syncthreads();                              // wsum and btot are reused
        if (w < nw) {
            mask[w] = bits;
            wpre[w] = run;
            for (uint32_t bb = bits; bb; bb &= bb - 1) {
                const int j = w * 32 + __ffs(bb) - 1;
                cidx[j] = run;
                act[run] = j;
                flag[j] = 0;
                ++run;
            }
        }
    }
    if (t == 0) {
        meta[0] = carry;
        meta[1] = carry > mcap ? 1 : 0;
        if (stats) {
            if (carry > mcap) atomicAdd(stats + 5, 1ull);
            stats[6] = (unsigned long long)carry;
        }
    }
}
static __global__ void __launch_bounds__(1024) k_lz_scan(int nvt, int mcap, int *__restrict__ flag,
                                                 int *__restrict__ cidx, int *__restrict__ act,
                                                 uint32_t *__restrict__ mask, int *__restrict__ wpre,
                                                 int *__restrict__ meta,
                                                 unsigned long long *__restrict__ stats = nullptr)
{
    lz_scan_block(nvt, mcap, flag, cidx, act, mask, wpre, meta, stats);
}

// Compact node indices (a, b, a*, b*) of every sample, and the number of
// terms per destination.
__device__ __forceinline__ void lz_remap_one(int l, const int4 *__restrict__ idx, const int *__restrict__ cidx,
                                             ushort4 *__restrict__ qc, int *__restrict__ count)
{
    const int4 q = idx[l];
    const int d[4] = {q.x >= 0 ? cidx[q.x] : -1, q.y >= 0 ? cidx[q.y] : -1,
                      q.z >= 0 ? cidx[q.z] : -1, q.w >= 0 ? cidx[q.w] : -1};
    qc[l] = Idx4<uint16_t>::make(d);
#pragma unroll
    for (int r = 0; r < 4; ++r)
        if (d[r] >= 0) atomicAdd(count + d[r], 1);
}
static __global__ void k_lz_remap(int nt, const int4 *__restrict__ idx, const int *__restrict__ cidx,
                           ushort4 *__restrict__ qc, int *__restrict__ count)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < nt) lz_remap_one(l, idx, cidx, qc, count);
}

// Exclusive scan of the term counts over the M destinations (cursor = first
// position of each destination's terms in the sorted order, rowend = one past
// its last), the number of terms E and the run length C of each of the
// kernel's T threads; clears the counts.  A destination without terms gets
// one term of weight 0 (at the zero entry M, entries of 1 << osh bytes), so
// that every destination has a row and a run steps to the next destination
// at each row end.  One CTA of 1024 threads.
__device__ __forceinline__ void lz_lscan_block(int T, int osh, int *__restrict__ count, int *__restrict__ cursor,
                                               int *__restrict__ rowend, int *__restrict__ meta,
                                               uint2 *__restrict__ rec, int *__restrict__ dest0)
{
    __shared__ int part[1024];
    const int t = threadIdx.x, M = meta[0], per = (M + 1023) / 1024;
    const int b = min(M, t * per), e = min(M, b + per);
    int s = 0;
    for (int i = b; i < e; ++i) s += max(count[i], 1);
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    // Runs of C terms, C a multiple of 8; the positions past the last term
    // hold zero records (weight 0, no destination change) and every run
    // starts at the zero entry M until k_lz_lfill names its first term.
    const int E = part[1023], C = ((E + T - 1) / T + 7) / 8 * 8;
    for (int p = E + t; p < C * T; p += 1024) {
        const int tt = p / C, i = p - tt * C;
        rec[(int64_t)i * T + tt] = make_uint2(0u, 0u);
    }
    for (int tt = t; tt < T; tt += 1024) dest0[tt] = M;
    __syncthreads();
    const uint32_t zo = (uint32_t)M << osh;
    int run = part[t] - s;
    for (int i = b; i < e; ++i) {
        cursor[i] = run;
        if (count[i] == 0) {
            const int tt = run / C, j = run - tt * C;
            rec[(int64_t)j * T + tt] = make_uint2(zo | (zo << 16) | 1u, 0u);
            if (j == 0) dest0[tt] = i;
            ++run;
        }
        run += count[i];
        rowend[i] = run;
        count[i] = 0;
    }
    if (t == 1023) {
        meta[2] = E;
        meta[3] = C;
    }
}
static __global__ void __launch_bounds__(1024) k_lz_lscan(int T, int osh, int *__restrict__ count,
                                                         int *__restrict__ cursor,
                                                         int *__restrict__ rowend,
                                                         int *__restrict__ meta, uint2 *__restrict__ rec,
                                                         int *__restrict__ dest0)
{
    lz_lscan_block(T, osh, count, cursor, rowend, meta, rec, dest0);
}

// The term records, sorted by destination: position p of the sorted order
// goes to thread p / C, slot i = p mod C, stored at rec[i T + p / C] so that
// the threads' i-th records are adjacent.  A record is
//   x = a_off | b_off << 16 | last,   y = +-W (bits of the float),
// with a_off, b_off the byte offsets of the sample's pre-collision nodes in
// the kernel's compact array (entries of 1 << osh bytes; a node outside the
// grid points to the zero entry M), last set on the final term of a
// destination, and the sign negative for the loss terms (the destination is
// a or b).  dest0[tt] is the destination of thread tt's first term.
// Nothing is written when the step overflowed (the kernel does not run then).
template <typename PA>
__device__ __forceinline__ void lz_lfill_one(int l, int T, int osh, const ushort4 *__restrict__ qc,
                                             const PA *__restrict__ pa, int *__restrict__ cursor,
                                             const int *__restrict__ rowend, const int *__restrict__ meta,
                                             uint2 *__restrict__ rec, int *__restrict__ dest0)
{
    if (meta[1]) return;
    const int M = meta[0], C = meta[3];
    const ushort4 q = qc[l];
    const int d[4] = {idx_of(q.x), idx_of(q.y), idx_of(q.z), idx_of(q.w)};
    const uint32_t ao = (uint32_t)(d[0] >= 0 ? d[0] : M) << osh;
    const uint32_t bo = (uint32_t)(d[1] >= 0 ? d[1] : M) << osh;
    const uint32_t x = ao | (bo << 16);
    const float W = pa[l].W;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (d[r] < 0) continue;
        const int pos = atomicAdd(cursor + d[r], 1);
        const int tt = pos / C, i = pos - tt * C;
        const uint32_t last = pos == rowend[d[r]] - 1 ? 1u : 0u;
        rec[(int64_t)i * T + tt] = make_uint2(x | last, __float_as_uint(r < 2 ? -W : W));
        if (i == 0) dest0[tt] = d[r];
    }
}
template <typename PA>
__global__ void k_lz_lfill(int nt, int T, int osh, const ushort4 *__restrict__ qc,
                           const PA *__restrict__ pa, int *__restrict__ cursor,
                           const int *__restrict__ rowend, const int *__restrict__ meta,
                           uint2 *__restrict__ rec, int *__restrict__ dest0)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < nt) lz_lfill_one(l, T, osh, qc, pa, cursor, rowend, meta, rec, dest0);
}

// Bank-aware order of the term records.  A collision thread reads the two
// operands of its term with two 16-byte (G = 4) or 8-byte (G = 2) shared
// loads.  The loads of a warp are served NB = 8 (or 16) lanes at a time, one
// wavefront per distinct entry in the busiest of the NB bank groups (entry
// index mod NB), so the NB runs that one phase reads together are ordered
// jointly.  Terms move only inside their destination segment of a run, and
// the two operands of a term may be swapped (the product is symmetric).
// Position by position, the runs choose in order of how few choices they
// have left (the one with the fewest remaining terms in its segment first;
// padding, which reads entry 0, before all): each takes the remaining term
// of its segment, and the operand order, whose first and second operands
// meet the fewest bank groups already holding another entry at that
// position.  A run decides position p once it has decided p - 1 and every
// run before it at p has decided p.  The positions are cut into chunks
// ordered independently (a segment that crosses a chunk's end is cut
// there).  One warp per phase group and chunk: NB runs x 32 / NB lanes that
// scan a run's choices.  Nothing happens if a run is longer than cmax.
// Several plans at once: blockIdx.z selects plan slot (z0 + blockIdx.z) mod
// zK, whose meta and records lie kLzMetaSize ints and rec_stride records
// after those of slot 0.
constexpr int kLzOrderWin = 64;     // positions whose taken entries are held at a time

__host__ __device__ inline size_t lz_order_smem(int chunk, int nb)
{
    // records (rows padded to an odd length), taken entries of a window of
    // positions, segment ends, run order masks, decided masks of the window,
    // padding masks
    const size_t m = nb == 8 ? 1 : 2;
    return (size_t)nb * (chunk + 1) * sizeof(uint2) + (size_t)kLzOrderWin * nb * sizeof(uint32_t) +
           (size_t)chunk * nb * (sizeof(uint16_t) + m) + (size_t)kLzOrderWin * m + (size_t)chunk * m + 32;
}

template <int NB>
__global__ void __launch_bounds__(32) k_lz_order(int T, int cmax, int chunk, const int *__restrict__ meta,
                                                 uint2 *__restrict__ rec, int zK = 1, int z0 = 0,
                                                 int64_t rec_stride = 0)
{
    {
        const int zs = (z0 + (int)blockIdx.z) % zK;
        meta += zs * kLzMetaSize;
        rec += zs * rec_stride;
    }
    static_assert(NB == 8 || NB == 16, "phase width");
    constexpr int H = 32 / NB;                       // lanes per run
    constexpr int OSH = NB == 8 ? 4 : 3;             // log2 of the entry size
    constexpr int W = kLzOrderWin;
    constexpr uint16_t kNone = 0xFFFF;
    using Mask = typename std::conditional<NB == 8, uint8_t, uint16_t>::type;
    extern __shared__ __align__(16) unsigned char osm[];
    const int lane = threadIdx.x, l = lane / H, h = lane - l * H;
    const unsigned rmask = ((1u << H) - 1u) << (l * H);   // the lanes of this run
    const int tt = blockIdx.x * NB + l;
    const int C = meta[3], c0 = blockIdx.y * chunk;
    if (C > cmax || meta[1] || blockIdx.x * NB + NB > T || c0 >= C) return;
    const int L = min(chunk, C - c0), SP = chunk + 1;
    uint2 *b = reinterpret_cast<uint2 *>(osm);                   // [NB][SP] working copies of the runs
    uint32_t *u = reinterpret_cast<uint32_t *>(b + NB * SP);     // [W][NB] entries taken: first | second << 16
    uint16_t *seg = reinterpret_cast<uint16_t *>(u + W * NB);    // [NB][chunk] segment end | last << 15
    Mask *bm = reinterpret_cast<Mask *>(seg + NB * chunk);       // [NB][chunk] runs that choose before this one
    Mask *dec = bm + NB * chunk;                                // [W] runs that have decided p
    Mask *pad = dec + W;                                        // [chunk] runs that are padding at p
    // Positions p live in slot p mod W of u and dec while some run has not
    // decided them; a run decides p only while p < (the smallest undecided
    // position) + W, which delays some decisions but changes none.
#pragma unroll 4
    for (int i = lane; i < NB * L; i += 32) {       // the NB runs of a position are adjacent in rec
        const int p = i / NB, r = i - p * NB;
        b[r * SP + p] = rec[(int64_t)(c0 + p) * T + blockIdx.x * NB + r];
    }
    __syncwarp();
    // Segments: up to a destination's last term or the chunk's end, before
    // the padding (zero records).
    if (h == 0) {
        const uint2 *br = b + l * SP;
        uint16_t *se = seg + l * chunk;
        int i = 0;
        while (i < L && !(br[i].x == 0u && br[i].y == 0u)) {
            int e = i;                                // the segment's last position (< L)
            while (e + 1 < L && !(br[e].x & 1u) && !(br[e + 1].x == 0u && br[e + 1].y == 0u)) ++e;
            const uint16_t v = (uint16_t)(e | (br[e].x & 1u) << 15);
            for (int p = i; p <= e; ++p) se[p] = v;
            i = e + 1;
        }
        for (int p = i; p < L; ++p) se[p] = kNone;
    }
    __syncwarp();
    // Per position: the order of the runs (remaining choices, then run
    // index); padding is decided from the start and reads entry 0.
    for (int p = lane; p < L; p += 32) {
        int sz[NB];
        Mask d = 0;
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            const uint16_t v = seg[r * chunk + p];
            sz[r] = v == kNone ? 0 : (v & 0x7FFF) - p + 1;
            if (v == kNone) d |= (Mask)(1u << r);
        }
        pad[p] = d;
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            Mask m = 0;
#pragma unroll
            for (int r2 = 0; r2 < NB; ++r2)
                if (sz[r2] < sz[r] || (sz[r2] == sz[r] && r2 < r)) m |= (Mask)(1u << r2);
            bm[r * chunk + p] = m;
        }
    }
    __syncwarp();
    // The first window: nothing taken, padding decided (its reads are entry 0).
    int wend = min(W, L);                             // positions below this hold their slot
    for (int i = lane; i < wend * NB; i += 32) {
        const int q = i / NB, g = i - q * NB;
        u[i] = g == 0 && pad[q] ? 0u : 0xFFFFFFFFu;
    }
    for (int q = lane; q < wend; q += 32) dec[q] = pad[q];
    __syncwarp();
    uint2 *bl = b + l * SP;
    const uint16_t *sl = seg + l * chunk;
    const Mask *bml = bm + l * chunk;
    int p = 0;                                        // this run's next position in the chunk
    uint16_t sv = L > 0 ? sl[0] : kNone;              // its segment: end | last << 15, kNone: padding
    // Every step some run is ready (the first, at the smallest undecided
    // position, in that position's order; that position lies in the window),
    // so NB * L steps always suffice.
    for (int step = 0; step < NB * L; ++step) {
        const bool active = p < L && sv != kNone;
        if (!__any_sync(0xFFFFFFFFu, active)) break;
        // The smallest undecided position; positions up to it + W get slots.
        const int pmin = (int)__reduce_min_sync(0xFFFFFFFFu, (unsigned)(active ? p : L));
        const int wnew = min(pmin + W, L);
        if (wnew > wend) {
            // (positions below wnew - W are behind every run: not set up)
            const int w0 = max(wend, wnew - W);
            for (int i = lane; i < (wnew - w0) * NB; i += 32) {
                const int q = w0 + i / NB, g = i % NB;
                u[(q & (W - 1)) * NB + g] = g == 0 && pad[q] ? 0u : 0xFFFFFFFFu;
            }
            for (int q = w0 + lane; q < wnew; q += 32) dec[q & (W - 1)] = pad[q];
            wend = wnew;
            __syncwarp();
        }
        bool ready = false;
        Mask dp = 0;
        if (active && p < wend) {
            const Mask need = bml[p];
            dp = dec[p & (W - 1)];
            ready = (Mask)(dp & need) == need;
        }
        __syncwarp();                                 // the reads above precede this step's writes
        uint32_t best = 0xFFFFFFFFu;                  // cost << 24 | swap << 23 | position
        const int s1 = sv & 0x7FFF;
        const uint32_t *row = u + (p & (W - 1)) * NB; // entries taken at p, by group
        if (ready) {
            // Passes of 4 H candidates; the run's lanes take the same passes.
            for (int jb = p; jb <= s1; jb += 4 * H) {
                const int j0 = jb + h;
                uint32_t xs[4], wa[4], wb[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) xs[k] = j0 + k * H <= s1 ? bl[j0 + k * H].x : 0u;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    wa[k] = row[(xs[k] >> OSH) & (NB - 1)];
                    wb[k] = row[(xs[k] >> (16 + OSH)) & (NB - 1)];
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int j = j0 + k * H;
                    if (j > s1) break;
                    const uint32_t ea = (xs[k] & 0xFFFCu) >> OSH, eb = xs[k] >> (16 + OSH);
                    const uint32_t a1 = wa[k] & 0xFFFFu, a2 = wa[k] >> 16, b1 = wb[k] & 0xFFFFu, b2 = wb[k] >> 16;
                    const uint32_t cn = (a1 != kNone && a1 != ea) + (b2 != kNone && b2 != eb);
                    const uint32_t cs = (b1 != kNone && b1 != eb) + (a2 != kNone && a2 != ea);
                    const uint32_t key = cs < cn ? (cs << 24 | 1u << 23 | (uint32_t)j) : (cn << 24 | (uint32_t)j);
                    best = min(best, key);
                }
                // A candidate with no conflict and no swap beats every later
                // one (the key then orders by position): the scan stops.
#pragma unroll
                for (int o = 1; o < H; o <<= 1) best = min(best, __shfl_xor_sync(rmask, best, o));
                if (best < (1u << 23)) break;
            }
        }
#pragma unroll
        for (int o = 1; o < H; o <<= 1) best = min(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
        if (ready && h == 0) {
            const int j = (int)(best & 0xFFFFu);
            uint2 r = bl[j];
            const uint2 front = bl[p];
            r.x &= ~1u;
            if (best >> 23 & 1u) r.x = (r.x >> 16) | ((r.x & 0xFFFCu) << 16);
            if (p == s1) r.x |= (uint32_t)(sv >> 15);
            rec[(int64_t)(c0 + p) * T + tt] = r;
            bl[j] = front;                            // the front term fills the hole
            const uint32_t e1 = (r.x & 0xFFFCu) >> OSH, e2 = r.x >> (16 + OSH);
            const uint32_t g1 = e1 & (NB - 1), g2 = e2 & (NB - 1);
            uint32_t v1 = row[g1];
            if ((v1 & 0xFFFFu) == kNone) v1 = (v1 & 0xFFFF0000u) | e1;
            uint32_t v2 = g2 == g1 ? v1 : row[g2];
            if ((v2 >> 16) == kNone) v2 = (v2 & 0xFFFFu) | e2 << 16;
            uint32_t *roww = u + (p & (W - 1)) * NB;
            roww[g1] = g2 == g1 ? v2 : v1;
            if (g2 != g1) roww[g2] = v2;
            dec[p & (W - 1)] = (Mask)(dp | (1u << l));
        }
        __syncwarp();
        if (ready) {
            ++p;
            if (p > s1) sv = p < L ? sl[p] : kNone;
        }
    }
    // Positions left undecided (none when the loop ran out normally) keep
    // their remaining terms, with the destination bit at the segment end.
    if (h == 0)
        for (; p < L && sl[p] != kNone; ++p) {
            uint2 r = bl[p];
            r.x &= ~1u;
            if (p == (sl[p] & 0x7FFF)) r.x |= (uint32_t)(sl[p] >> 15);
            rec[(int64_t)(c0 + p) * T + tt] = r;
        }
}

// ---------------------------------------------------------------------
// Fallback when a step has more active nodes than mcap: the k_cell4 plan is
// derived from the logical one, the input is corrected in place and mu_out
// is cleared (k_cell4 writes corrected states).  All return at once otherwise.
// ---------------------------------------------------------------------
__device__ __forceinline__ void lz_fb_plan_one(int l, int N, const int4 *__restrict__ idx,
                                               const PlanA<float, int> *__restrict__ pa,
                                               ushort4 *__restrict__ pidx16, PlanA<float, uint16_t> *__restrict__ pa16,
                                               int *__restrict__ count)
{
    const int4 q = idx[l];
    int o[4] = {q.x, q.y, q.z, q.w};
    const int nq = N / 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int j = o[k];
        if (j < 0) continue;
        const int jx = j / (N * N), jz = j % N, row = j - jz;
        int r = jz / 4 + jx % nq;
        if (r >= nq) r -= nq;
        o[k] = row + 4 * r + (jz & 3);
    }
    const ushort4 u = Idx4<uint16_t>::make(o);
    pidx16[l] = u;
    pa16[l] = make_plan_a<float, uint16_t>(o[0], o[1], (double)pa[l].W);
    if (u.x != 0xFFFF) atomicAdd(count + u.x, 1);
    if (u.y != 0xFFFF) atomicAdd(count + u.y, 1);
    if (u.z != 0xFFFF) atomicAdd(count + u.z, 1);
    if (u.w != 0xFFFF) atomicAdd(count + u.w, 1);
}
static __global__ void k_lz_fb_plan(int nt, int N, const int *__restrict__ meta,
                             const int4 *__restrict__ idx, const PlanA<float, int> *__restrict__ pa,
                             ushort4 *__restrict__ pidx16, PlanA<float, uint16_t> *__restrict__ pa16,
                             int *__restrict__ count)
{
    if (!meta[1]) return;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < nt) lz_fb_plan_one(l, N, idx, pa, pidx16, pa16, count);
}

// The correction of a stored node value: h = h_c + (1 + eps h_c) kappa.
__device__ __forceinline__ float lz_corr(float hc, float kappa, float eps)
{
    return fmaf(eps * hc, kappa, hc + kappa);
}

// h <- h_c + (1 + eps h_c)(mu_c . psi_j) for every node (in place allowed:
// hout may be hin, so neither is restrict-qualified); mu_zero (nullable) is
// then cleared, and mu_used (nullable; may be mu) gets each cell's
// corrections cleared once they are read.  When skip_unless (nullable)
// points to 0, does nothing.  One CTA per cell at a time; float4 over jz.
static __global__ void k_lz_materialize(Geo g, const int *__restrict__ skip_unless,
                                 const float *hin, const float *mu, float *hout,
                                 float *__restrict__ mu_zero, float *mu_used = nullptr)
{
    if (skip_unless && !skip_unless[1]) return;
    __shared__ float sv[kMaxN];
    __shared__ float smu[8];
    const int N = g.nv, nq = N / 4, Q = N * N / 4;
    for (int i = threadIdx.x; i < N; i += blockDim.x) sv[i] = (float)g.axv[i];
    const float eps = g.epsf;
    const int64_t plane = g.nvt / 4;
    for (int c = blockIdx.x; c < g.nr; c += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < 8) smu[threadIdx.x] = mu[(int64_t)c * 8 + threadIdx.x];
        __syncthreads();
        if (mu_used && threadIdx.x < 8) mu_used[(int64_t)c * 8 + threadIdx.x] = 0.f;
        const float4 *src = reinterpret_cast<const float4 *>(hin) + (int64_t)c * plane;
        float4 *dst = reinterpret_cast<float4 *>(hout) + (int64_t)c * plane;
        for (int o = threadIdx.x; o < (int)plane; o += blockDim.x) {
            const int jx = o / Q, q = o % Q, jy = q / nq, jz = 4 * (q % nq);
            const float vx = sv[jx], vy = sv[jy];
            const float base = smu[0] + smu[1] * vx + smu[2] * vy + smu[4] * (vx * vx + vy * vy);
            float4 h = src[o];
            float *hp = &h.x;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float vz = sv[jz + i];
                hp[i] = lz_corr(hp[i], base + smu[3] * vz + smu[4] * vz * vz, eps);
            }
            dst[o] = h;
        }
    }
    if (mu_zero) {
        const int64_t n = (int64_t)g.nr * 8;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x)
            mu_zero[i] = 0.f;
    }
}

// ---------------------------------------------------------------------
// Packed FP32x2 arithmetic (each component rounds like fmaf / __fadd_rn).
// ---------------------------------------------------------------------
__device__ __forceinline__ float2 lz_add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 lz_mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 lz_fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lz_dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 lz_lo(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 lz_hi(float4 a) { return make_float2(a.z, a.w); }

// Values of a node in the G cells of a group (adjacent in shared memory).
template <int G> struct LzVec;
template <> struct LzVec<2> { using T = float2; };
template <> struct LzVec<4> { using T = float4; };

__device__ __forceinline__ float2 lz_zero2() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ void lz_set_zero(float2 &a) { a = lz_zero2(); }
__device__ __forceinline__ void lz_set_zero(float4 &a) { a = make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void lz_atomic_add(float2 *p, float2 v)
{
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}
__device__ __forceinline__ void lz_atomic_add(float4 *p, float4 v)
{
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
    atomicAdd(&p->z, v.z);
    atomicAdd(&p->w, v.w);
}

// ---------------------------------------------------------------------
// Per-thread asynchronous copies global -> shared (cp.async), completed by
// the issuing thread's cp.async.wait_group: each thread prefetches the source
// values of its own nodes several streaming stages ahead, with no register
// cost and no synchronisation with other threads.
// ---------------------------------------------------------------------
__device__ __forceinline__ uint32_t lz_saddr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void lz_cp16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(lz_saddr(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void lz_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void lz_cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void lz_cp_wait_stage()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(kLzStages - 1) : "memory");
}

// Bulk copies global -> shared through the tensor-memory-access unit
// (cp.async.bulk, completion counted in bytes on an mbarrier) and the
// mbarrier operations of the streaming ring.  Every wait is bounded: each
// poll returns within the hardware's own suspend limit, and after kLzWaitNs
// of the global timer the wait gives up and returns false.
__device__ __forceinline__ void lz_mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void lz_mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void lz_mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void lz_mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool lz_mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long lz_now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool lz_mbar_wait(uint32_t bar, uint32_t parity)
{
    if (lz_mbar_try(bar, parity)) return true;
    const unsigned long long t0 = lz_now_ns();
    while (!lz_mbar_try(bar, parity))
        if (lz_now_ns() - t0 > kLzWaitNs) return false;
    return true;
}
// A bounded wait that is skipped once any wait of the CTA has given up (the
// CTA then finishes without waiting and reports the error).
__device__ __forceinline__ void lz_ring_wait(uint32_t bar, uint32_t parity, int &err)
{
    volatile int *e = &err;
    if (*e == 0 && !lz_mbar_wait(bar, parity)) *e = 1;
}
__device__ __forceinline__ void lz_bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Orders this thread's generic-proxy shared-memory writes before later
// bulk copies (async proxy) into the same bytes.
__device__ __forceinline__ void lz_fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Everything the kernel needs besides the geometry (by value).
struct LzArgs {
    const float *hin, *mu_in, *ghost;
    float *hout, *mu_out;
    double *mom;
    const uint2 *rec;       // term records (k_lz_lfill)
    const int *dest0;       // first destination of each thread's run
    const int *meta;
    const uint32_t *mask;
    const int *wpre, *act;
    int mcap;
    float e0[kLzX];         // sum_j w_j X_k(v_j) of the 30 monomials
    long long *clk;         // nullable: phase trace of CTA 0 (kClkCells groups x kClkPhases)
    unsigned long long *stats;  // nullable: [3] counts correction solves that fell back
    int nostream;           // 1: h~ = h (no free streaming; the relaxation alone)
    int early_tail;         // 1: the collision warps start the increment sums at once
    unsigned long long *err;    // nullable: set to 1 when a bounded mbarrier wait gave up
    int tx_excess;          // bulk-copy ring, CTA 0's first stage: bytes expected beyond
                            // those copied (a wait that runs out, for tests; normally 0)
    int *fb_count;          // nullable: counts of the fallback's scatter list, zeroed
    int fb_n;               // (fb_n ints) when the step overflowed, before the fallback
};

// Shared memory.  A fixed-layout head (compile-time offsets): warp partial
// sums, per-axis tables, the groups' cells and the correction tables of the
// cells the streaming reads.  Then two compact arrays of h~ (G values per
// active node plus a zero entry; the streaming warps fill one while the
// collision warps use the other), the compact array of collision
// increments, the per-thread staging slots of the streaming prefetch
// (kLzStages stages x {own, x source, y source} x streaming threads, 16 bytes
// each), the active-node bit mask, its word prefixes and the node list.
struct alignas(128) LzHead {
    float fpart[3][kLzMaxG][kLzRoleWarps][32];   // warp partials of the F sums, per group (it mod 3)
    float dpart[2][kLzMaxG][kLzRoleWarps][32];   // warp partials of the D sums, per group (it mod 2)
    float4 ta[kLzMaxN];                          // -ax, -ax, A, A
    float4 tv12[kLzMaxN];                        // v, v, v^2, v^2
    float4 tv34[kLzMaxN];                        // v^3, v^3, v^4, v^4
    float v[kLzMaxN], A[kLzMaxN], IA[kLzMaxN], cuy[kLzMaxN];
    float4 tcx[kLzMaxG][kLzMaxN];                // ca of the own and the upwind x cell, duplicated
    float2 tcy[kLzMaxG][2][kLzMaxN];             // ca of the cell below (0) and above (1), duplicated
    float mus[kLzMaxG][5][8];                    // mu of own, right, left, below, above (0 outside)
    int4 cell[2][kLzMaxG];                       // c, ix, iy of a group's cells (c < 0: none), per buffer
    int tail_next;                               // next chunk of the increment sums to claim
    int tma_err;                                 // a bounded wait of the bulk-copy ring gave up
    unsigned long long bar_full[kLzStages];      // bulk-copy ring: stage landed (transaction bytes)
    unsigned long long bar_empty[kLzStages];     // bulk-copy ring: stage read by the streaming warps
};
constexpr uint32_t kLzAOff = (sizeof(LzHead) + 15) & ~(size_t)15;

struct LzOff {
    uint32_t abytes, a1, bc, ring, mask, wpre, act, end;
};
__host__ __device__ inline LzOff lz_offsets(int nvt, int mcap, int G)
{
    LzOff o;
    o.abytes = (uint32_t)(((sizeof(float) * (size_t)G * (mcap + 1)) + 127) & ~(size_t)127);
    size_t off = kLzAOff + o.abytes;
    o.a1 = (uint32_t)off; off += o.abytes;
    o.bc = (uint32_t)off; off += o.abytes;
    o.ring = (uint32_t)off; off += (size_t)kLzStages * 3 * kLzRoleT * sizeof(float4);
    o.mask = (uint32_t)off; off += sizeof(uint32_t) * (nvt / 32);
    o.wpre = (uint32_t)off; off += sizeof(uint16_t) * (nvt / 32);
    o.act = (uint32_t)off; off += sizeof(uint16_t) * (size_t)mcap;
    o.end = (uint32_t)((off + 15) & ~(size_t)15);
    return o;
}

// Monomial index of psi_a * phi_b in the 30-entry sum vector X (psi = 1,
// v_x, v_y, v_z, v^2; phi = 1, v_x, v_y, v_z, v_x^2, v_y^2, v_z^2, v_x v_y,
// v_x v_z, v_y v_z).  X order: 0 1; 1-3 v_x, v_y, v_z; 4-6 v_x^2, v_y^2,
// v_z^2; 7-9 v_x v_y, v_x v_z, v_y v_z; 10-12 v_x^3, v_y^3, v_z^3; 13 v_x^2 v_y;
// 14 v_x^2 v_z; 15 v_x v_y^2; 16 v_y^2 v_z; 17 v_x v_z^2; 18 v_y v_z^2;
// 19 v_x v_y v_z; 20-22 v_x^2 v^2, v_y^2 v^2, v_z^2 v^2; 23-25 v_x v_y v^2,
// v_x v_z v^2, v_y v_z v^2; 26 v^2; 27-29 v_x v^2, v_y v^2, v_z v^2.
__host__ __device__ constexpr int lz_psiphi(int a, int b)
{
    constexpr unsigned char t[5][10] = {
        {0, 1, 2, 3, 4, 5, 6, 7, 8, 9},
        {1, 4, 7, 8, 10, 15, 17, 13, 14, 19},
        {2, 7, 5, 9, 13, 11, 18, 15, 19, 16},
        {3, 8, 9, 6, 14, 16, 12, 19, 17, 18},
        {26, 27, 28, 29, 20, 21, 22, 23, 24, 25}};
    return t[a][b];
}

// The 26 monomial sums of sum_nodes n(v) from per-thread power sums over jx
// (s[p] = sum n v_x^p) at fixed v_y = y, v_z = z.
__device__ __forceinline__ void lz_mono_from_powers(const float (&s)[5], float y, float z,
                                                    float (&M)[32])
{
    const float y2 = y * y, z2 = z * z, q = y2 + z2, yz = y * z;
    M[0] += s[0];
    M[1] += s[1];
    M[2] += y * s[0];
    M[3] += z * s[0];
    M[4] += s[2];
    M[5] += y2 * s[0];
    M[6] += z2 * s[0];
    M[7] += y * s[1];
    M[8] += z * s[1];
    M[9] += yz * s[0];
    M[10] += s[3];
    M[11] += y2 * y * s[0];
    M[12] += z2 * z * s[0];
    M[13] += y * s[2];
    M[14] += z * s[2];
    M[15] += y2 * s[1];
    M[16] += y2 * z * s[0];
    M[17] += z2 * s[1];
    M[18] += y * z2 * s[0];
    M[19] += yz * s[1];
    const float t2 = s[2] + q * s[0];
    M[20] += s[4] + q * s[2];
    M[21] += y2 * t2;
    M[22] += z2 * t2;
    M[23] += y * (s[3] + q * s[1]);
    M[24] += z * (s[3] + q * s[1]);
    M[25] += yz * t2;
}

// The same sums for one node value d at velocity (x, y, z).
__device__ __forceinline__ void lz_mono_node(float d, float x, float y, float z, float (&M)[32])
{
    const float x2 = x * x;
    const float s[5] = {d, d * x, d * x2, d * x2 * x, d * x2 * x2};
    lz_mono_from_powers(s, y, z, M);
}

// Sum of 32 values over a warp, left with lane l holding the total of value l
// (recursive halving: 31 shuffles instead of 32 x 5).
__device__ __forceinline__ float lz_warp_reduce_scatter(float (&v)[32])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? v[i] : v[i + o];
            const float keep = up ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, o);
        }
    }
    return v[0];
}

// X (30) from the 26 sums.
__device__ __forceinline__ void lz_extend(const float *T, float *X)
{
#pragma unroll
    for (int k = 0; k < kLzMono; ++k) X[k] = T[k];
    X[26] = T[4] + T[5] + T[6];
    X[27] = T[10] + T[15] + T[17];
    X[28] = T[13] + T[11] + T[18];
    X[29] = T[14] + T[16] + T[12];
}

// Correction and output moments of one cell from the sums T (of the
// post-collision N_c = N + dN) and D (of the collision increment dN): mu to
// mu_out, moments to mom.  Called by all 32 lanes of a warp (the lanes share
// the residual of the solve); lane 0 stores.
__device__ __forceinline__ void lz_finish(const Geo &g, const LzArgs &a, int c, const float *T,
                                       const float *D, int *fallback)
{
    const int lane = threadIdx.x & 31;
    float X[kLzX];
    lz_extend(T, X);
    // Eqs. rinorm_a, correzione: G mu = -D with G from the sums of N_c and
    // D the conserved moments of the increment (1, v, v^2).
    float P[19];
    for (int k = 0; k < 10; ++k) P[k] = X[k];
    P[10] = X[27];
    P[11] = X[28];
    P[12] = X[29];
    P[13] = X[20] + X[21] + X[22];
    P[14] = D[0];
    P[15] = D[1];
    P[16] = D[2];
    P[17] = D[3];
    P[18] = D[4] + D[5] + D[6];
    float mu[5];
    if (!correction_spd(g, P, mu, lane)) {
        double Pd[19], m8[5];
        for (int k = 0; k < 19; ++k) Pd[k] = (double)P[k];
        int f2 = 0;
        correction_solve<float>(g, Pd, m8, &f2);
        if (lane == 0) ++*fallback;
        for (int k = 0; k < 5; ++k) mu[k] = (float)m8[k];
    }
    if (lane != 0) return;
    float *mo = a.mu_out + (int64_t)c * 8;
    for (int k = 0; k < 5; ++k) mo[k] = mu[k];
    // Moments of h^{n+1}: sum w h phi = sum N_c phi + sum_a mu_a (E0 + eps sum N_c psi_a phi).
    const float eps = g.epsf;
    float m10[10];
#pragma unroll
    for (int b = 0; b < 10; ++b) {
        float s = X[b];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int x = lz_psiphi(k, b);
            s += mu[k] * (a.e0[x] + eps * X[x]);
        }
        m10[b] = s;
    }
    if (a.mom) finalize_moments_f(m10, eps, a.mom + (int64_t)c * 11);
}

// The (v_y, v_z) part of a cell's pending correction at a thread's four
// nodes (jy, 4 qz .. 4 qz + 3): mu_y v_y + mu_z v_z + mu_4 (v_y^2 + v_z^2), as
// two node pairs.
__device__ __forceinline__ void lz_bd(const float *mu, const float *v, int jy, int qz, float2 (&bd)[2])
{
    const float vy = v[jy];
    float b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float vz = v[4 * qz + i];
        b[i] = mu[2] * vy + mu[3] * vz + mu[4] * (vy * vy + vz * vz);
    }
    bd[0] = make_float2(b[0], b[1]);
    bd[1] = make_float2(b[2], b[3]);
}

// lz_mono_from_powers for two cells at once (s and M hold one value per
// cell; y and z are the node's, shared by both).
__device__ __forceinline__ void lz_mono_from_powers2(const float2 (&s)[5], float y, float z,
                                                     float2 (&M)[32])
{
    const float y2 = y * y, z2 = z * z, q = y2 + z2, yz = y * z;
    const float2 Y = lz_dup(y), Z = lz_dup(z), Y2 = lz_dup(y2), Z2 = lz_dup(z2), YZ = lz_dup(yz);
    M[0] = lz_add2(M[0], s[0]);
    M[1] = lz_add2(M[1], s[1]);
    M[2] = lz_fma2(Y, s[0], M[2]);
    M[3] = lz_fma2(Z, s[0], M[3]);
    M[4] = lz_add2(M[4], s[2]);
    M[5] = lz_fma2(Y2, s[0], M[5]);
    M[6] = lz_fma2(Z2, s[0], M[6]);
    M[7] = lz_fma2(Y, s[1], M[7]);
    M[8] = lz_fma2(Z, s[1], M[8]);
    M[9] = lz_fma2(YZ, s[0], M[9]);
    M[10] = lz_add2(M[10], s[3]);
    M[11] = lz_fma2(lz_dup(y2 * y), s[0], M[11]);
    M[12] = lz_fma2(lz_dup(z2 * z), s[0], M[12]);
    M[13] = lz_fma2(Y, s[2], M[13]);
    M[14] = lz_fma2(Z, s[2], M[14]);
    M[15] = lz_fma2(Y2, s[1], M[15]);
    M[16] = lz_fma2(lz_dup(y2 * z), s[0], M[16]);
    M[17] = lz_fma2(Z2, s[1], M[17]);
    M[18] = lz_fma2(lz_dup(y * z2), s[0], M[18]);
    M[19] = lz_fma2(YZ, s[1], M[19]);
    const float2 Q = lz_dup(q);
    const float2 t2 = lz_fma2(Q, s[0], s[2]), t3 = lz_fma2(Q, s[1], s[3]);
    M[20] = lz_add2(M[20], lz_fma2(Q, s[2], s[4]));
    M[21] = lz_fma2(Y2, t2, M[21]);
    M[22] = lz_fma2(Z2, t2, M[22]);
    M[23] = lz_fma2(Y, t3, M[23]);
    M[24] = lz_fma2(Z, t3, M[24]);
    M[25] = lz_fma2(YZ, t2, M[25]);
}

// lz_warp_reduce_scatter for two cells at once.
__device__ __forceinline__ float2 lz_warp_reduce_scatter2(float2 (&v)[32])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float2 send = up ? v[i] : v[i + o];
            const float2 keep = up ? v[i + o] : v[i];
            v[i] = make_float2(keep.x + __shfl_xor_sync(0xFFFFFFFFu, send.x, o),
                               keep.y + __shfl_xor_sync(0xFFFFFFFFu, send.y, o));
        }
    }
    return v[0];
}

// Shared-memory accesses by 32-bit shared address.
__device__ __forceinline__ void lz_cp16s(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void lz_sts4(uint32_t dst, float v)
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %1, %1, %1};" ::"r"(dst), "f"(v) : "memory");
}
__device__ __forceinline__ float4 lz_lds4(uint32_t src)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(src)
                 : "memory");
    return v;
}

// A streaming thread's constant geometry.
struct LzQuad {
    int S, J, Jh, P4, pl, N, jy;
    bool yup, streams;
    int64_t pbytes;             // bytes per cell (N^3 floats)
    int sbytes;                 // bytes per stage of a cell (S float4)
    uint32_t ring0, ring_end;   // shared addresses: this thread's slots of ring slot 0; ring end
};
constexpr uint32_t kLzSrcStride = kLzRoleT * 16;          // between the three sources of a stage
constexpr uint32_t kLzSlotStride = 3 * kLzSrcStride;      // between stage slots

// Prefetch position of a thread: cell pk of the group, stage pst of that
// cell, the shared address of the slots it fills next, and what the cell's
// sources are (cells, or a wall's ghost values).
struct LzPf {
    int pk, pst;
    int sidx;                // ring slot index of the next stage (bulk-copy ring)
    uint32_t slot;
    const char *own;         // this thread's quad of stage pst of cell pk
    int64_t yoff;            // byte offset of the y source cell
    float gxr, gxl;          // ghost values of the right and left walls (cells at a wall)
    const float *gy;         // ghost values of the bottom or top wall, by jx (cells at a wall)
    bool xin_r, xin_l, yin;  // the right, left and y sources are cells
};

__device__ __forceinline__ void lz_pf_cell(LzPf &p, const LzQuad &q, const Geo &g, const LzArgs &a,
                                           const int4 *cells, const char *hin_t)
{
    const int4 ce = cells[p.pk];
    p.own = hin_t + (int64_t)ce.x * q.pbytes;
    p.xin_r = ce.y < g.nx - 1;
    p.xin_l = ce.y > 0;
    p.yin = q.yup ? ce.z > 0 : ce.z < g.ny - 1;
    p.yoff = q.yup ? -(int64_t)g.nx * q.pbytes : (int64_t)g.nx * q.pbytes;
    p.gxr = p.xin_r ? 0.f : __ldg(a.ghost + (g.ny + ce.z) * q.N + q.jy);
    p.gxl = p.xin_l ? 0.f : __ldg(a.ghost + ce.z * q.N + q.jy);
    p.gy = a.ghost + (q.yup ? 2 * g.ny + ce.y : 2 * g.ny + g.nx + ce.y) * q.N + q.pl;
}

// Stages this thread's own, x-source and y-source quads of the next stage
// (a wall's ghost value where the source lies outside the cavity) and
// commits one group of copies (an empty one past the group's last stage).
__device__ __forceinline__ void lz_prefetch(LzPf &p, const LzQuad &q, const Geo &g, const LzArgs &a,
                                            const int4 *cells, const char *hin_t, int ncell)
{
    if (q.streams && p.pk < ncell) {
        if (p.pst == 0) lz_pf_cell(p, q, g, a, cells, hin_t);
        lz_cp16s(p.slot, p.own);
        // x source: the right cell while v_x < 0 (the first half of the
        // stages), the left cell after.
        if (p.pst < q.Jh) {
            if (p.xin_r) lz_cp16s(p.slot + kLzSrcStride, p.own + q.pbytes);
            else lz_sts4(p.slot + kLzSrcStride, p.gxr);
        } else {
            if (p.xin_l) lz_cp16s(p.slot + kLzSrcStride, p.own - q.pbytes);
            else lz_sts4(p.slot + kLzSrcStride, p.gxl);
        }
        if (p.yin) lz_cp16s(p.slot + 2 * kLzSrcStride, p.own + p.yoff);
        else lz_sts4(p.slot + 2 * kLzSrcStride, __ldg(p.gy + p.pst * q.P4));
        p.own += q.sbytes;
    }
    lz_cp_commit();
    p.slot += kLzSlotStride;
    if (p.slot == q.ring_end) p.slot = q.ring0;
    if (++p.pst == q.J) {
        p.pst = 0;
        ++p.pk;
    }
}

// The producer's view of the bulk-copy ring: per slot (one bit each),
// whether a stage was issued into it whose reading has not been awaited yet,
// the parity of the next phase of its empty barrier, and the parity of its
// issue count.
struct LzTmaProd {
    uint32_t pending, epar, ipar;
};

// The same step with bulk copies: thread 0 of the role issues the stage's
// runs once every streaming warp has read the slot's previous stage.  The
// own and the x-source runs are S float4 each, contiguous in global memory
// and in the slot (a stage never straddles jx = N/2).  The y source differs
// within a plane: its rows jy < N/2 (v_y < 0) come from the cell above and
// its rows jy >= N/2 from the cell below, so each of the stage's P4 planes
// takes two half-plane copies.  Each thread still writes its wall ghost
// values into its own bytes of the slot (no copy where the source lies
// outside the cavity).
__device__ __forceinline__ void lz_prefetch_tma(LzPf &p, const LzQuad &q, const Geo &g, const LzArgs &a,
                                                const int4 *cells, const char *hin_t, int ncell, LzHead &H,
                                                LzTmaProd &pr)
{
    if (p.pk < ncell) {
        if (p.pst == 0) lz_pf_cell(p, q, g, a, cells, hin_t);
        const bool left = p.pst >= q.Jh;
        const bool xin = left ? p.xin_l : p.xin_r;
        if (q.streams) {
            if (!xin) lz_sts4(p.slot + kLzSrcStride, left ? p.gxl : p.gxr);
            if (!p.yin) lz_sts4(p.slot + 2 * kLzSrcStride, __ldg(p.gy + p.pst * q.P4));
        }
        // After a wait gave up, nothing more is issued (the waits are skipped).
        if (threadIdx.x == 0 && *(volatile int *)&H.tma_err == 0) {
            const int s = p.sidx;
            const uint32_t full = lz_saddr(&H.bar_full[s]);
            if (pr.pending >> s & 1u) {
                lz_ring_wait(lz_saddr(&H.bar_empty[s]), pr.epar >> s & 1u, H.tma_err);
                pr.epar ^= 1u << s;
            }
            const uint32_t extra = (blockIdx.x == 0 && pr.ipar == 0u && pr.pending == 0u) ? (uint32_t)a.tx_excess : 0u;
            pr.pending |= 1u << s;
            pr.ipar ^= 1u << s;
            const uint32_t sb = (uint32_t)q.sbytes;
            const uint32_t hb = (uint32_t)(q.N * q.N) * 2u;          // half a plane (N^2/2 floats)
            const int4 ce = cells[p.pk];
            const bool above = ce.z < g.ny - 1, below = ce.z > 0;
            const uint32_t ybytes = (uint32_t)q.P4 * hb * ((above ? 1u : 0u) + (below ? 1u : 0u));
            lz_mbar_expect_tx(full, sb * (1u + (xin ? 1u : 0u)) + ybytes + extra);
            lz_bulk_g2s(p.slot, p.own, sb, full);
            if (xin) lz_bulk_g2s(p.slot + kLzSrcStride, left ? p.own - q.pbytes : p.own + q.pbytes, sb, full);
            const int64_t ystep = (int64_t)g.nx * q.pbytes;
            for (int pl = 0; pl < q.P4; ++pl) {
                const uint32_t o = (uint32_t)pl * 2u * hb;
                if (above) lz_bulk_g2s(p.slot + 2 * kLzSrcStride + o, p.own + ystep + o, hb, full);
                if (below) lz_bulk_g2s(p.slot + 2 * kLzSrcStride + o + hb, p.own - ystep + o + hb, hb, full);
            }
        }
        p.own += q.sbytes;
    }
    p.slot += kLzSlotStride;
    if (++p.sidx == kLzStages) {
        p.sidx = 0;
        p.slot = q.ring0;
    }
    if (++p.pst == q.J) {
        p.pst = 0;
        ++p.pk;
    }
}

// Per-cell state of a thread's streaming: the (v_y, v_z) parts of the
// sources' pending corrections and the power sums over jx of N = w h~ /
// (A_y A_z) for the quad's two node pairs.
struct LzAcc {
    float2 bdo[2], bdx[2], bdy[2];
    float2 s0[2], s1[2], s2[2], s3[2], s4[2];
};

// One streaming stage of one cell (Eq. streaming2D with the deferred
// correction applied to its sources): h~ to dst, the power sums, and the
// active nodes of the quad to the compact array (component k of G).  SX:
// stretched cells, the x Courant numbers times the cell's factor fx2.
template <int G, bool SX>
__device__ __forceinline__ void lz_stream_stage(uint32_t sl, int jx, int j0, int k, const LzHead &H,
                                                const float4 *tcx, const float2 *tcy, LzAcc &c,
                                                float4 *dst, const uint32_t *smask, const uint16_t *swpre,
                                                float *Af, float2 eps2, float2 one2, float2 nay2, float2 fx2)
{
    const float4 h0 = lz_lds4(sl), hx = lz_lds4(sl + kLzSrcStride), hy = lz_lds4(sl + 2 * kLzSrcStride);
    const float4 cx4 = tcx[jx];
    const float2 cy2 = tcy[jx];
    const float4 ta = H.ta[jx];
    const float2 nax2 = SX ? lz_mul2(lz_lo(ta), fx2) : lz_lo(ta), A2 = lz_hi(ta);
    const float4 v12 = H.tv12[jx], v34 = H.tv34[jx];
    const float2 h0p[2] = {lz_lo(h0), lz_hi(h0)}, hxp[2] = {lz_lo(hx), lz_hi(hx)},
                 hyp[2] = {lz_lo(hy), lz_hi(hy)};
    float2 ht[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        // u = h_c + (1 + eps h_c) kappa of each source, as h_c (1 + eps kappa) + kappa.
        const float2 ko = lz_add2(lz_lo(cx4), c.bdo[p]);
        const float2 u0 = lz_fma2(h0p[p], lz_fma2(eps2, ko, one2), ko);
        const float2 kx = lz_add2(lz_hi(cx4), c.bdx[p]);
        const float2 ux = lz_fma2(hxp[p], lz_fma2(eps2, kx, one2), kx);
        const float2 ky = lz_add2(cy2, c.bdy[p]);
        const float2 uy = lz_fma2(hyp[p], lz_fma2(eps2, ky, one2), ky);
        // Eq. streaming2D: u0 - ax (u0 - ux) - ay (u0 - uy).
        const float2 mux = make_float2(-ux.x, -ux.y), muy = make_float2(-uy.x, -uy.y);
        float2 h = lz_fma2(nax2, lz_add2(u0, mux), u0);
        h = lz_fma2(nay2, lz_add2(u0, muy), h);
        ht[p] = h;
        const float2 n = lz_mul2(h, A2);
        c.s0[p] = lz_add2(c.s0[p], n);
        c.s1[p] = lz_fma2(n, lz_lo(v12), c.s1[p]);
        c.s2[p] = lz_fma2(n, lz_hi(v12), c.s2[p]);
        c.s3[p] = lz_fma2(n, lz_lo(v34), c.s3[p]);
        c.s4[p] = lz_fma2(n, lz_hi(v34), c.s4[p]);
    }
    *dst = make_float4(ht[0].x, ht[0].y, ht[1].x, ht[1].y);
    // Active nodes of the quad (nodes j0 .. j0 + 3) go to the compact array.
    const uint32_t mw = smask[j0 >> 5];
    const int sh = j0 & 31;
    const uint32_t bits = (mw >> sh) & 15u;
    if (bits) {
        int mi = swpre[j0 >> 5] + __popc(mw & ((1u << sh) - 1u));
        const float hv[4] = {ht[0].x, ht[0].y, ht[1].x, ht[1].y};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (bits >> i & 1u) Af[(mi++) * G + k] = hv[i];
    }
}

// g = ha + hb + eps ha hb per cell, as ha + hb (1 + eps ha), and acc += w g
// (Eq. monteCarloInt: the sample's product, signed and weighted for its
// destination).
__device__ __forceinline__ void lz_term(float2 ha, float2 hb, float2 eps2, float2 w2, float2 &acc)
{
    const float2 g = lz_fma2(hb, lz_fma2(eps2, ha, lz_dup(1.f)), ha);
    acc = lz_fma2(w2, g, acc);
}
__device__ __forceinline__ void lz_term(float4 ha, float4 hb, float2 eps2, float2 w2, float4 &acc)
{
    float2 lo = lz_lo(acc), hi = lz_hi(acc);
    lz_term(lz_lo(ha), lz_lo(hb), eps2, w2, lo);
    lz_term(lz_hi(ha), lz_hi(hb), eps2, w2, hi);
    acc = make_float4(lo.x, lo.y, hi.x, hi.y);
}

// The state of a thread's run: the sum of its current destination, which is
// stored when the destination's last term has passed (atomically for the
// thread's first destination and its unfinished last one, which neighbouring
// runs may share).
template <typename V> struct LzRun {
    V acc;
    int dest;
    bool first;
};

template <typename V>
__device__ __forceinline__ void lz_apply(V ha, V hb, uint2 r, float2 eps2, LzRun<V> &st, V *Bv)
{
    lz_term(ha, hb, eps2, lz_dup(__uint_as_float(r.y)), st.acc);
    if (r.x & 1u) {
        if (st.first) lz_atomic_add(Bv + st.dest, st.acc);
        else Bv[st.dest] = st.acc;
        st.first = false;
        ++st.dest;
        lz_set_zero(st.acc);
    }
}

// Applies 8 records (the operands of two terms are read before either of
// them can store a destination's sum).
template <typename V, uint32_t AMASK>
__device__ __forceinline__ void lz_apply8(const uint2 (&r)[8], const char *Ab, float2 eps2, LzRun<V> &st,
                                          V *Bv)
{
#pragma unroll
    for (int h = 0; h < 8; h += 2) {
        const V ha0 = *reinterpret_cast<const V *>(Ab + (r[h].x & AMASK));
        const V hb0 = *reinterpret_cast<const V *>(Ab + (r[h].x >> 16));
        const V ha1 = *reinterpret_cast<const V *>(Ab + (r[h + 1].x & AMASK));
        const V hb1 = *reinterpret_cast<const V *>(Ab + (r[h + 1].x >> 16));
        lz_apply(ha0, hb0, r[h], eps2, st, Bv);
        lz_apply(ha1, hb1, r[h + 1], eps2, st, Bv);
    }
}

// Barrier among the 256 threads of one role (named barrier 1: streaming,
// 2: collision; 0 is __syncthreads).
__device__ __forceinline__ void lz_role_bar(int id)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kLzRoleT) : "memory");
}
// Named barrier 3 over all threads: the collision role arrives without
// waiting once its terms are complete; the streaming role waits for that.
__device__ __forceinline__ void lz_terms_done_arrive()
{
    asm volatile("bar.arrive 3, %0;" ::"n"(kLzThreads) : "memory");
}
__device__ __forceinline__ void lz_terms_done_wait()
{
    asm volatile("bar.sync 3, %0;" ::"n"(kLzThreads) : "memory");
}
constexpr int kLzTailChunk = 256;  // active nodes per claimed chunk of the increment sums

// One CTA of 512 threads per SM, two roles working on consecutive groups of
// G cells: warps 0-7 stream group i (Eq. streaming2D, the power sums, the
// active nodes to one compact array) and then solve the correction and the
// moments of group i - 2, while warps 8-15 apply the collision terms, their
// sums and the write-back of group i - 1 from the other compact array.
// Streaming is bound by HBM and the collision terms by shared memory, so
// the two overlap.
//
// NV: the velocity axis length as a compile-time constant (0: read g.nv at
// run time).  SX: stretched cells (per-column and per-row Courant factors
// g.sx, g.sy).  Streaming thread t < S = K N^2/4 owns node quad q = t mod
// (N^2/4) (four consecutive jz at one (jx, jy)) of jx-plane t div (N^2/4) of
// every stage; a stage covers K planes and a cell J = N / K stages.
//
// TMA: the streaming sources arrive by bulk copies (cp.async.bulk) that
// thread 0 of the role issues into a ring of kLzStages slots, with a full
// and an empty mbarrier per slot, instead of per-thread cp.async.
//
// lz_run runs the pipeline of one CTA over the groups grp0, grp0 + gstride,
// ... (nmine of them) of one problem; the kernel k_lz gives CTA b the groups
// b, b + gridDim.x, ...
template <int G, int NV, bool SX, bool TMA = false>
__device__ __forceinline__ void lz_run(const Geo &g, const LzArgs &a, char *smem_raw, int grp0, int gstride,
                                       int nmine)
{
    using V = typename LzVec<G>::T;
    if (a.meta[1]) {                              // too many active nodes: k_cell4 runs
        if (a.fb_count)
            for (int i = (int)(blockIdx.x * blockDim.x + threadIdx.x); i < a.fb_n; i += gridDim.x * blockDim.x)
                a.fb_count[i] = 0;
        return;
    }
    const int N = NV ? NV : g.nv;
    const int N2 = N * N, nvt = N2 * N, t = threadIdx.x;
    const int Qd = N2 / 4, nq = N / 4, P4 = lz_planes4(N), J = N / P4, Jh = J / 2;
    const int S = P4 * Qd;                        // float4 per stage (the threads that stream)
    const int half = N / 2;
    const int64_t plane4 = nvt / 4;               // float4 per cell
    LzHead &H = *reinterpret_cast<LzHead *>(smem_raw);
    const int M = a.meta[0];
    const LzOff so = lz_offsets(nvt, a.mcap, G);
    float4 *ring = reinterpret_cast<float4 *>(smem_raw + so.ring);
    V *Bv = reinterpret_cast<V *>(smem_raw + so.bc);
    float *Bf = reinterpret_cast<float *>(smem_raw + so.bc);
    uint32_t *smask = reinterpret_cast<uint32_t *>(smem_raw + so.mask);
    uint16_t *swpre = reinterpret_cast<uint16_t *>(smem_raw + so.wpre);
    uint16_t *sact = reinterpret_cast<uint16_t *>(smem_raw + so.act);
    const float eps = g.epsf;
    const float2 eps2 = lz_dup(eps), one2 = lz_dup(1.f);
    const int lane = t & 31, warp = t >> 5;
    const bool streamer = t < kLzRoleT;

    // ---- tables (once per launch) ----------------------------------------
    for (int i = t; i < N; i += kLzThreads) {
        const double v = g.axv[i], A = g.axA[i];
        // Courant numbers 0 without streaming: h~ is then exactly the
        // corrected input (every source term is multiplied by zero).
        const float nax = a.nostream ? 0.f : -(float)fabs(v * g.dt / g.dx), fA = (float)A, fv = (float)v;
        H.v[i] = fv;
        H.A[i] = fA;
        H.IA[i] = (float)(1.0 / A);
        H.cuy[i] = a.nostream ? 0.f : (float)fabs(v * g.dt / (SX ? g.dx : g.dy));
        H.ta[i] = make_float4(nax, nax, fA, fA);
        const float v2 = (float)(v * v), v3 = (float)(v * v * v), v4 = (float)(v * v * v * v);
        H.tv12[i] = make_float4(fv, fv, v2, v2);
        H.tv34[i] = make_float4(v3, v3, v4, v4);
    }
    for (int w = t; w < nvt / 32; w += kLzThreads) {
        smask[w] = a.mask[w];
        swpre[w] = (uint16_t)a.wpre[w];
    }
    for (int m = t; m < M; m += kLzThreads) sact[m] = (uint16_t)a.act[m];
    for (int i = t; i < 2 * kLzMaxG * kLzRoleWarps * 32; i += kLzThreads) (&H.dpart[0][0][0][0])[i] = 0.f;
    if (TMA && t == 0) {
        for (int s = 0; s < kLzStages; ++s) {
            lz_mbar_init(lz_saddr(&H.bar_full[s]), 1);
            lz_mbar_init(lz_saddr(&H.bar_empty[s]), kLzRoleWarps);
        }
        H.tma_err = 0;
        lz_mbar_init_fence();
    }
    __syncthreads();

    // A streaming thread's quad.
    const bool streams = t < S;
    const int pl = streams ? t / Qd : 0, q = streams ? t - pl * Qd : 0;
    const int jy = q / nq, qz = q - jy * nq;
    const bool yup = jy >= half;                  // v_y > 0: the y source is below
    const float2 nay2 = lz_dup(-H.cuy[jy]);
    const float4 *hin4 = reinterpret_cast<const float4 *>(a.hin);
    float4 *hout4 = reinterpret_cast<float4 *>(a.hout);
    int fallback = 0;
    LzTmaProd prod{0u, 0u, 0u};                   // thread 0: the bulk-copy ring's producer state
    uint32_t fpar = 0u;                           // parity of each slot's next full phase

    // Iteration it: the streaming warps take this CTA's group it, the
    // collision warps its group it - 1.
    for (int it = 0; it <= nmine + 1; ++it) {
        const bool clk = a.clk && grp0 == 0 && it < kClkCells;
        if (clk && t == 0) a.clk[it * kClkPhases + 0] = clock64();
        if (streamer) {
            if (it < nmine) {
                const int grp = grp0 + it * gstride, buf = it & 1;
                float *Af = reinterpret_cast<float *>(smem_raw + kLzAOff + buf * so.abytes);
                if (t < G) {
                    const int kc = grp * G + t;
                    const int c = kc < g.nr ? cell_of(g, kc) : -1;
                    H.cell[buf][t] = make_int4(c, c >= 0 ? c % g.nx : 0, c >= 0 ? c / g.nx : 0, 0);
                }
                lz_role_bar(1);
                int ncell = 0;
#pragma unroll
                for (int k = 0; k < G; ++k) ncell += H.cell[buf][k].x >= 0 ? 1 : 0;
                // mu of the five cells each cell's streaming reads (0 outside the cavity).
                for (int i = t; i < G * 40; i += kLzRoleT) {
                    const int k = i / 40, r = i - k * 40, s5 = r / 8, m = r - s5 * 8;
                    const int4 ce = H.cell[buf][k];
                    int cs = ce.x;
                    bool ok = ce.x >= 0 && m < 5;
                    if (s5 == 1) { ok = ok && ce.y < g.nx - 1; cs = ce.x + 1; }
                    if (s5 == 2) { ok = ok && ce.y > 0; cs = ce.x - 1; }
                    if (s5 == 3) { ok = ok && ce.z > 0; cs = ce.x - g.nx; }
                    if (s5 == 4) { ok = ok && ce.z < g.ny - 1; cs = ce.x + g.nx; }
                    H.mus[k][s5][m] = ok ? a.mu_in[(int64_t)cs * 8 + m] : 0.f;
                }
                // kLzStages - 1 stages in flight ahead of the one being used.
                const uint32_t ring0 = lz_saddr(ring) + t * 16;
                const LzQuad qd{S, J, Jh, P4, pl, N, jy, yup, streams, (int64_t)nvt * 4, S * 16, ring0,
                                ring0 + kLzStages * kLzSlotStride};
                const char *hin_t = reinterpret_cast<const char *>(hin4 + t);
                LzPf pf{};
                pf.slot = ring0;
                const int4 *cells = H.cell[buf];
#pragma unroll
                for (int kk = 0; kk < kLzStages - 1; ++kk) {
                    if (TMA) lz_prefetch_tma(pf, qd, g, a, cells, hin_t, ncell, H, prod);
                    else lz_prefetch(pf, qd, g, a, cells, hin_t, ncell);
                }
                lz_role_bar(1);
                // Correction tables of the group's cells: ca(jx) = mu_0 + mu_x
                // v_x + mu_4 v_x^2 of the own cell, the upwind x cell (right for
                // jx < N/2, left otherwise), and the cells below and above.
                for (int i = t; i < G * N; i += kLzRoleT) {
                    const int k = i / N, jx = i - k * N;
                    const float vx = H.v[jx];
                    float ca[5];
#pragma unroll
                    for (int s5 = 0; s5 < 5; ++s5) {
                        const float *m = H.mus[k][s5];
                        ca[s5] = m[0] + m[1] * vx + m[4] * vx * vx;
                    }
                    const float cx = jx < half ? ca[1] : ca[2];
                    H.tcx[k][jx] = make_float4(ca[0], ca[0], cx, cx);
                    H.tcy[k][0][jx] = lz_dup(ca[3]);
                    H.tcy[k][1][jx] = lz_dup(ca[4]);
                }
                lz_role_bar(1);

                // ---- streaming with the deferred correction applied to its sources
                uint32_t cslot = ring0;           // slots of the stage being used
                int cidx = 0;                     // and their index
#pragma unroll 1
                for (int k = 0; k < ncell; ++k) {
                    // A cell at a wall had ghost values written into its slots
                    // by the threads (generic proxy) before later bulk copies.
                    const int4 cek = cells[k];
                    const bool wallk = TMA && (cek.y == 0 || cek.y == g.nx - 1 || cek.z == 0 || cek.z == g.ny - 1);
                    LzAcc ac;
#pragma unroll
                    for (int p = 0; p < 2; ++p)
                        ac.s0[p] = ac.s1[p] = ac.s2[p] = ac.s3[p] = ac.s4[p] = lz_zero2();
                    lz_bd(H.mus[k][0], H.v, jy, qz, ac.bdo);
                    lz_bd(H.mus[k][1], H.v, jy, qz, ac.bdx);
                    lz_bd(H.mus[k][yup ? 3 : 4], H.v, jy, qz, ac.bdy);
                    const float4 *tcx = H.tcx[k];
                    const float2 *tcy = H.tcy[k][yup ? 0 : 1];
                    float4 *dst = hout4 + (int64_t)cells[k].x * plane4 + t;
                    // Courant factors of this cell on stretched grids.
                    float2 fx2 = one2, nay2k = nay2;
                    if (SX) {
                        fx2 = lz_dup((float)g.sx[cells[k].y]);
                        nay2k = lz_dup(-H.cuy[jy] * (float)g.sy[cells[k].z]);
                    }
                    int jx = pl, j0 = 4 * t;
#pragma unroll 1
                    for (int st = 0; st < J; ++st) {
                        if (st == Jh) lz_bd(H.mus[k][2], H.v, jy, qz, ac.bdx);   // the left cell now
                        // The slots read last stage take the stage kLzStages - 1
                        // ahead; then this stage's copies have landed.
                        if (TMA) {
                            lz_prefetch_tma(pf, qd, g, a, cells, hin_t, ncell, H, prod);
                            lz_ring_wait(lz_saddr(&H.bar_full[cidx]), fpar >> cidx & 1u, H.tma_err);
                            fpar ^= 1u << cidx;
                        } else {
                            lz_prefetch(pf, qd, g, a, cells, hin_t, ncell);
                            lz_cp_wait_stage();
                        }
                        if (streams)
                            lz_stream_stage<G, SX>(cslot, jx, j0, k, H, tcx, tcy, ac, dst, smask, swpre, Af,
                                                   eps2, one2, nay2k, fx2);
                        if (TMA) {
                            // The warp has read the slot: release it to the producer.
                            if (wallk) lz_fence_proxy_async();
                            __syncwarp();
                            if (lane == 0) lz_mbar_arrive(lz_saddr(&H.bar_empty[cidx]));
                        }
                        cslot += kLzSlotStride;
                        if (TMA) {
                            if (++cidx == kLzStages) {
                                cidx = 0;
                                cslot = ring0;
                            }
                        } else if (cslot == qd.ring_end) {
                            cslot = ring0;
                        }
                        jx += P4;
                        j0 += 4 * S;
                        dst += S;
                    }
                    // The 26 monomial sums of the thread's nodes, summed over the warp.
                    float Msum[32];
#pragma unroll
                    for (int r = 0; r < 32; ++r) Msum[r] = 0.f;
                    if (streams) {
                        const float Ay = H.A[jy];
                        const float sv[4][5] = {
                            {ac.s0[0].x, ac.s1[0].x, ac.s2[0].x, ac.s3[0].x, ac.s4[0].x},
                            {ac.s0[0].y, ac.s1[0].y, ac.s2[0].y, ac.s3[0].y, ac.s4[0].y},
                            {ac.s0[1].x, ac.s1[1].x, ac.s2[1].x, ac.s3[1].x, ac.s4[1].x},
                            {ac.s0[1].y, ac.s1[1].y, ac.s2[1].y, ac.s3[1].y, ac.s4[1].y}};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float Ayz = Ay * H.A[4 * qz + i];
                            float si[5];
#pragma unroll
                            for (int pp = 0; pp < 5; ++pp) si[pp] = sv[i][pp] * Ayz;
                            lz_mono_from_powers(si, H.v[jy], H.v[4 * qz + i], Msum);
                        }
                    }
                    H.fpart[it % 3][k][warp][lane] = lz_warp_reduce_scatter(Msum);
                }
                if (!TMA) lz_cp_wait_all();
            }
            if (clk && t == 0) a.clk[it * kClkPhases + 1] = clock64();
            // One warp per cell of group it - 2: totals over the warps, then the
            // correction and the moments.
            if (it >= 2) {
                const int grp = grp0 + (it - 2) * gstride, fb = (it - 2) % 3, db = it & 1;
                const int k = warp, kc = grp * G + k;
                if (k < G && kc < g.nr) {
                    if (lane < kLzMono) {
                        // Compensated totals over the warps: T = F + D (the
                        // sums of N_c) and D.
                        float f = 0.f, fc = 0.f, d = 0.f, dc = 0.f;
#pragma unroll
                        for (int w = 0; w < kLzRoleWarps; ++w) {
                            float e;
                            two_sum(f, H.fpart[fb][k][w][lane], f, e);
                            fc = __fadd_rn(fc, e);
                            two_sum(d, H.dpart[db][k][w][lane], d, e);
                            dc = __fadd_rn(dc, e);
                        }
                        float tt, te;
                        two_sum(f, d, tt, te);
                        H.fpart[fb][k][0][lane] = __fadd_rn(tt, __fadd_rn(te, __fadd_rn(fc, dc)));
                        H.dpart[db][k][0][lane] = __fadd_rn(d, dc);
                    }
                    __syncwarp();
                    lz_finish(g, a, cell_of(g, kc), H.fpart[fb][k][0], H.dpart[db][k][0], &fallback);
                    __syncwarp();
                    // The slots take the increment sums of a later group (atomically).
                    for (int i = lane; i < kLzRoleWarps * 32; i += 32) (&H.dpart[db][k][0][0])[i] = 0.f;
                }
            }
            if (clk && t == 0) a.clk[it * kClkPhases + 5] = clock64();
        } else if (it >= 1 && it <= nmine) {
            const int tc = t - kLzRoleT, buf = (it - 1) & 1;
            char *Ab = smem_raw + kLzAOff + buf * so.abytes;
            float *Af = reinterpret_cast<float *>(Ab);
            int ncell = 0, cg[G];
#pragma unroll
            for (int k = 0; k < G; ++k) {
                cg[k] = H.cell[buf][k].x;
                ncell += cg[k] >= 0 ? 1 : 0;
            }
            // ---- Monte Carlo terms (Eq. monteCarloInt) ----------------------
            // The increments start from zero; the zero entry M of h~ stands for
            // nodes outside the grid, and cells missing from a short group hold 0.
            for (int i = tc; i < M + 1; i += kLzRoleT) lz_set_zero(Bv[i]);
            if (tc < G) Af[M * G + tc] = 0.f;
            if (tc == 0) H.tail_next = 0;
            if (ncell < G)
                for (int i = tc; i < M * G; i += kLzRoleT)
                    if (i % G >= ncell) Af[i] = 0.f;
            lz_role_bar(2);
            {
                // Each thread applies its run of the destination-sorted terms:
                // it sums one destination's terms in registers and stores the
                // sum when the destination's last term has passed (atomically
                // for its first destination and its unfinished last one, which
                // neighbouring runs may share).
                const int C = a.meta[3];
                if (C > 0) {
                    constexpr uint32_t amask = G == 4 ? 0xFFF0u : 0xFFF8u;
                    LzRun<V> st;
                    lz_set_zero(st.acc);
                    st.dest = a.dest0[tc];
                    st.first = true;
                    // Batches of 8 records in three register buffers: a buffer
                    // is refilled as soon as it has been applied, two batches
                    // ahead (the records stream from L2).  A run is C records,
                    // C a multiple of 8, zero-padded by the plan.
                    const uint2 *rp = a.rec + tc;
                    constexpr int Ts = kLzRoleT, Bs = 8 * kLzRoleT;
                    uint2 r0[8], r1[8], r2[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        r0[u] = rp[u * Ts];
                        r1[u] = C > 8 ? rp[Bs + u * Ts] : make_uint2(0u, 0u);
                        r2[u] = C > 16 ? rp[2 * Bs + u * Ts] : make_uint2(0u, 0u);
                    }
                    for (int i = 0; i < C; i += 24) {
                        rp += 3 * Bs;
                        lz_apply8<V, amask>(r0, Ab, eps2, st, Bv);
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (i + 24 < C) r0[u] = rp[u * Ts];
                        if (i + 8 < C) {
                            lz_apply8<V, amask>(r1, Ab, eps2, st, Bv);
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (i + 32 < C) r1[u] = rp[Bs + u * Ts];
                        }
                        if (i + 16 < C) {
                            lz_apply8<V, amask>(r2, Ab, eps2, st, Bv);
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (i + 40 < C) r2[u] = rp[2 * Bs + u * Ts];
                        }
                    }
                    lz_atomic_add(Bv + st.dest, st.acc);
                }
            }
            if (clk && tc == 0) a.clk[it * kClkPhases + 2] = clock64();
            if (NV != 32 && a.early_tail) {
                // The increments are complete once every collision thread is here.
                lz_role_bar(2);
                lz_terms_done_arrive();
            }
        }
        // ---- sums of the collision increment and h_c = h~ + dN / w on the
        // active nodes of group it - 1, two cells at a time.  Either all
        // warps after a CTA barrier, each with a fixed share of the nodes and
        // its partial sums added to the slots of warp (warp mod 8); or
        // (early tail, for when the collision terms take less time than the
        // streaming; never at 32^3 velocities) the collision warps as soon as
        // their terms are complete and the streaming warps once they are
        // done, every warp claiming chunks of kLzTailChunk nodes of one cell
        // pair at a time (pair 0 first) and adding its partial sums of a pair
        // to the slots when it moves on.
        if (it >= 1 && it <= nmine) {
            const bool early = NV != 32 && a.early_tail;
            if (early) {
                if (streamer) lz_terms_done_wait();
            } else {
                __syncthreads();
            }
            const int buf = (it - 1) & 1;
            const float *Af = reinterpret_cast<const float *>(smem_raw + kLzAOff + buf * so.abytes);
            int ncell = 0, cg[G];
#pragma unroll
            for (int k = 0; k < G; ++k) {
                cg[k] = H.cell[buf][k].x;
                ncell += cg[k] >= 0 ? 1 : 0;
            }
            if (!early) {
                const int u = t ^ kLzRoleT;
#pragma unroll
                for (int k2 = 0; k2 < G; k2 += 2) {
                    float2 D2[32];
#pragma unroll
                    for (int r = 0; r < 32; ++r) D2[r] = lz_zero2();
                    if (k2 < ncell) {
                        for (int mm = u; mm < M; mm += kLzThreads) {
                            const int j = sact[mm], jxy = j / N;
                            const int jx = jxy / N, jyy = jxy - jx * N, jz = j - jxy * N;
                            const float2 d = *reinterpret_cast<const float2 *>(Bf + mm * G + k2);
                            const float2 h = *reinterpret_cast<const float2 *>(Af + mm * G + k2);
                            const float x = H.v[jx], x2 = x * x;
                            const float2 sp[5] = {d, lz_mul2(d, lz_dup(x)), lz_mul2(d, lz_dup(x2)),
                                                  lz_mul2(d, lz_dup(x2 * x)), lz_mul2(d, lz_dup(x2 * x2))};
                            lz_mono_from_powers2(sp, H.v[jyy], H.v[jz], D2);
                            const float iw = H.IA[jx] * H.IA[jyy] * H.IA[jz];
                            a.hout[(int64_t)cg[k2] * nvt + j] = fmaf(d.x, iw, h.x);
                            if (k2 + 1 < ncell) a.hout[(int64_t)cg[k2 + 1] * nvt + j] = fmaf(d.y, iw, h.y);
                        }
                    }
                    const float2 r = lz_warp_reduce_scatter2(D2);
                    atomicAdd(&H.dpart[buf][k2][warp & (kLzRoleWarps - 1)][lane], r.x);
                    atomicAdd(&H.dpart[buf][k2 + 1][warp & (kLzRoleWarps - 1)][lane], r.y);
                }
            } else {
                const int npair = (ncell + 1) / 2, per = (M + kLzTailChunk - 1) / kLzTailChunk;
                const int nchunk = npair * per;
                float2 D2[32];
#pragma unroll
                for (int r = 0; r < 32; ++r) D2[r] = lz_zero2();
                int kcur = -1;
                for (;;) {
                    int ch = 0;
                    if (lane == 0) ch = atomicAdd(&H.tail_next, 1);
                    ch = __shfl_sync(0xFFFFFFFFu, ch, 0);
                    const int k2 = ch < nchunk ? 2 * (ch / per) : -1;
                    if (k2 != kcur) {
                        if (kcur >= 0) {
                            const float2 r = lz_warp_reduce_scatter2(D2);
                            atomicAdd(&H.dpart[buf][kcur][warp & (kLzRoleWarps - 1)][lane], r.x);
                            atomicAdd(&H.dpart[buf][kcur + 1][warp & (kLzRoleWarps - 1)][lane], r.y);
#pragma unroll
                            for (int r2 = 0; r2 < 32; ++r2) D2[r2] = lz_zero2();
                        }
                        kcur = k2;
                    }
                    if (k2 < 0) break;
                    const int m0 = (ch - (k2 / 2) * per) * kLzTailChunk, m1 = min(M, m0 + kLzTailChunk);
                    for (int mm = m0 + lane; mm < m1; mm += 32) {
                        const int j = sact[mm], jxy = j / N;
                        const int jx = jxy / N, jyy = jxy - jx * N, jz = j - jxy * N;
                        const float2 d = *reinterpret_cast<const float2 *>(Bf + mm * G + k2);
                        const float2 h = *reinterpret_cast<const float2 *>(Af + mm * G + k2);
                        const float x = H.v[jx], x2 = x * x;
                        const float2 sp[5] = {d, lz_mul2(d, lz_dup(x)), lz_mul2(d, lz_dup(x2)),
                                              lz_mul2(d, lz_dup(x2 * x)), lz_mul2(d, lz_dup(x2 * x2))};
                        lz_mono_from_powers2(sp, H.v[jyy], H.v[jz], D2);
                        const float iw = H.IA[jx] * H.IA[jyy] * H.IA[jz];
                        a.hout[(int64_t)cg[k2] * nvt + j] = fmaf(d.x, iw, h.x);
                        if (k2 + 1 < ncell) a.hout[(int64_t)cg[k2 + 1] * nvt + j] = fmaf(d.y, iw, h.y);
                    }
                }
            }
            if (clk && t == kLzRoleT) a.clk[it * kClkPhases + 3] = clock64();
            if (clk && t == kLzRoleT) a.clk[it * kClkPhases + 4] = clock64();
        }
        __syncthreads();
    }
    if (fallback && a.stats) atomicAdd(a.stats + 3, (unsigned long long)fallback);
    if (TMA && t == 0 && H.tma_err) {
        // A wait gave up: report it, and wait (bounded) for the last copy
        // issued into each slot before the CTA leaves (after the first
        // timeout nothing more was issued).
        if (a.err) atomicOr(a.err, 1ull);
        for (int s = 0; s < kLzStages; ++s)
            if (prod.pending >> s & 1u) lz_mbar_wait(lz_saddr(&H.bar_full[s]), (prod.ipar >> s & 1u) ^ 1u);
    }
}

template <int G, int NV, bool SX, bool TMA = false>
__global__ void __launch_bounds__(kLzThreads, 1) k_lz(Geo g, LzArgs a)
{
    extern __shared__ __align__(16) char smem_raw[];
    const int ngroups = (g.nr + G - 1) / G;
    const int nmine = blockIdx.x < ngroups ? (ngroups - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    lz_run<G, NV, SX, TMA>(g, a, smem_raw, blockIdx.x, gridDim.x, nmine);
}

}  // namespace bzk
