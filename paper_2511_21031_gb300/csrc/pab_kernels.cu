// Kernels of the bubble source update on sm_103a.
//
// Work decomposition: a CTA owns a tile of 32 consecutive cells and a range of
// their bins (all Nb bins, except where a small grid is split over more SMs:
// then a range per CTA, and the last CTA of a tile to finish sums its moments
// from terms the others stored).  Its warps advance
// the tile's (bin, cell) items lane by lane (pab_stream.cuh): bin-major, so the
// loads and stores of the bin-major state stay coalesced while the lanes run
// together, and a lane that finishes an item takes the next one instead of
// waiting for its neighbours' stiffer items.  After the items, one warp reads
// the tile's new state back and writes the 7 moments of its 32 cells, summing
// each cell's bins in bin order.  No atomics touch the state: every (bin, cell)
// has one owner (Sec. 4).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "pab_check.cuh"
#include "pab_device.cuh"
#include "pab_internal.h"
#include "pab_reduce.cuh"
#include "pab_stream.cuh"

PAB_CHECK_UNIT(kernels)

namespace pab {
namespace {

// Fixed mode: n equal trials per item, the same for every item, so each thread carries one
// cell of the CTA through the bin range.
template <bool MIXED>
__device__ __forceinline__ void fixed_items(const StepConst &K, const StepArgs &a, const TileIO &io,
                                            TileCounts &tc)
{
    if ((int)threadIdx.x >= io.nc)
        return;
    const long long c = io.c0 + threadIdx.x;
    const long long ns = (long long)K.B * K.C;
    const double p_inf = PAB_LD(a.p_inf, c, K.C);
    const bool p_ok = finite64(p_inf);
    for (int b = io.b0; b < io.b1; ++b) {
        const BinConst &bc = K.bins[b];
        const size_t k = (size_t)b * (size_t)K.C + (size_t)c;
        double R = PAB_LD(a.R, k, ns), V = PAB_LD(a.V, k, ns);
        uint32_t fl = 0;
        int na = 0;
        if (!p_ok || !finite64(R) || !finite64(V)) {
            fl = PAB_FLAG_NONFINITE;
        } else {
            GasBase g;
            g.reset();
            const float A = MIXED ? bc.dpeqf + d2f(K.p0 - p_inf) : 0.0f;
            advance_fixed<MIXED>(K, bc, p_inf, A, a.dt_sub, R, V, g);
            na = K.n_fixed;
            if (!finite64(R) || !finite64(V))
                fl |= PAB_FLAG_NONFINITE;
            else if (!gt0(R))
                fl |= PAB_FLAG_NONPOS;
            if (abs_ge(V, K.c))
                fl |= PAB_FLAG_SUPERSONIC;
            PAB_ST(a.R, k, ns, R);
            PAB_ST(a.V, k, ns, V);
        }
        if (a.attempts)
            PAB_ST(a.attempts, k, ns, na);
        tc.fl_or |= fl;
        tc.n_flag += (fl != 0);
        tc.n_att += na;
    }
}

// The moments of a grid split by bins (gridDim.y CTAs per tile, one per bin range), without a
// second launch.  Each CTA writes the quadrature terms of its items from their new state (every
// lane at once, after the items: computed where an item finishes they would hold up the warp's
// other lanes once per finishing item), then takes a ticket of its tile; the CTA that takes the
// last one sums the tile's terms in bin order and writes its moments (the arithmetic and order
// of cell_moments, so the bits of an unsplit launch), and resets the ticket for the next step.
// No CTA waits for another.
template <bool MIXED>
__device__ __forceinline__ void split_moments(const StepConst &K, const StepArgs &a, const TileIO &io)
{
    __shared__ unsigned int s_last;
    const long long ns = (long long)K.B * K.C;
    const int n_items = (io.b1 - io.b0) * io.nc;
    for (int j = threadIdx.x; j < n_items; j += blockDim.x) {
        int b, cl;
        size_t k;
        item_of(io, j, b, cl, k);
        store_terms<MIXED>(K, a.terms, b, k, PAB_LDCG(a.R, k, ns), PAB_LDCG(a.V, k, ns),
                           MIXED ? nullptr : a.G);
    }
    __threadfence();
    __syncthreads();
    const long long tiles = (K.C + kTile - 1) / kTile;
    if (threadIdx.x == 0)
        s_last = atomicAdd(PAB_AT(a.tickets, (long long)blockIdx.x, tiles), 1u) == gridDim.y - 1;
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    for (int cl = threadIdx.x; cl < io.nc; cl += blockDim.x) {
        const long long c = io.c0 + cl;
        sum_cell_terms<MIXED>(K, a.terms, c, a.nb ? PAB_LD(a.nb, c, K.C) : K.nb_default, a.out);
    }
    if (threadIdx.x == 0)
        *PAB_AT(a.tickets, (long long)blockIdx.x, tiles) = 0u;
}

// One CTA of nw warps.  With one bin range (gridDim.y == 1) it owns nw tiles (32 nw cells from
// blockIdx.x * 32 nw) and all their bins, and ends with their moments (warp w: tile w);
// otherwise one tile (blockIdx.x) and bin range blockIdx.y.  Dynamic shared memory: the lot of
// parked items (32 per warp) in adaptive mixed precision, nothing otherwise.
template <bool MIXED, bool TERMS>
__device__ __forceinline__ void step_body(const StepConst &K, const StepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PoolCounters sh;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int cells = gridDim.y == 1 ? kTile * nw : kTile;
    TileIO io;
    io.p_inf = a.p_inf;
    io.R = a.R;
    io.V = a.V;
    io.h = a.h;
    io.attempts = a.attempts;
    io.C = K.C;
    io.c0 = (long long)blockIdx.x * cells;
    io.nc = (int)min((long long)cells, K.C - io.c0);
    const int per = (K.B + (int)gridDim.y - 1) / (int)gridDim.y;
    io.b0 = min(K.B, (int)blockIdx.y * per);
    io.b1 = min(K.B, io.b0 + per);
    io.dt = a.dt;
    TileCounts tc;
    if (K.n_fixed > 0) {
        fixed_items<MIXED>(K, a, io, tc);
    } else {
        // the cells' pressure terms, once per cell rather than once per (bin, cell) item
        constexpr int kCellBytes = MIXED ? (int)sizeof(float) : 2 * (int)sizeof(double);
        __shared__ __align__(8) unsigned char s_cell[kMaxWarps * kTile * kCellBytes];
        double *cB0 = reinterpret_cast<double *>(s_cell);
        double *cB0c = cB0 + kMaxWarps * kTile;
        float *cA0 = reinterpret_cast<float *>(s_cell);
        for (int cl = threadIdx.x; cl < io.nc; cl += blockDim.x) {
            const double p = PAB_LD(a.p_inf, io.c0 + cl, K.C);
            if (MIXED) {
                cA0[cl] = d2f(K.p0 - p);
            } else {
                const double B0 = (K.pv - p) * K.inv_rho;
                cB0[cl] = B0;
                cB0c[cl] = B0 * K.inv_c;
            }
        }
        io.cB0 = cB0;
        io.cB0c = cB0c;
        io.cA0 = cA0;
        io.G = (!MIXED && a.G_valid) ? a.G : nullptr;
        if (threadIdx.x == 0)
            sh = PoolCounters{0, 0, 0};
        __syncthreads();
        if (MIXED) {
            stream_mixed(K, io, sh, reinterpret_cast<Parked *>(smem), kLotPerWarp * nw, tc);
        } else {
            stream_fp64(K, io, sh, tc);
        }
    }
    // block-wide counters; the barrier inside also orders the state writes before the reads below
    flush_counters(tc.fl_or, tc.n_flag, tc.n_att, tc.n64, a.counters);
    const long long c = io.c0 + (long long)kTile * warp + lane;
    if (a.out && gridDim.y == 1 && c < io.c0 + io.nc)
        cell_moments<MIXED>(K, a.R, a.V, K.C, c, a.nb ? PAB_LD(a.nb, c, K.C) : K.nb_default, a.out,
                            MIXED ? nullptr : a.G);
    if (TERMS)
        split_moments<MIXED>(K, a, io);
}

#ifndef PAB_STEP64_MAXNREG
#define PAB_STEP64_MAXNREG 96
#endif
#ifndef PAB_STEPMX_MAXNREG
#define PAB_STEPMX_MAXNREG 64
#endif
template <bool MIXED, bool TERMS>
__global__ void step_kernel(const __grid_constant__ StepConst K, const StepArgs a);
template <>
__global__ void __maxnreg__(PAB_STEP64_MAXNREG)
    step_kernel<false, false>(const __grid_constant__ StepConst K, const StepArgs a)
{
    step_body<false, false>(K, a);
}
template <>
__global__ void __maxnreg__(PAB_STEPMX_MAXNREG)
    step_kernel<true, false>(const __grid_constant__ StepConst K, const StepArgs a)
{
    step_body<true, false>(K, a);
}
template <>
__global__ void __maxnreg__(PAB_STEP64_MAXNREG)
    step_kernel<false, true>(const __grid_constant__ StepConst K, const StepArgs a)
{
    step_body<false, true>(K, a);
}
template <>
__global__ void __maxnreg__(PAB_STEPMX_MAXNREG)
    step_kernel<true, true>(const __grid_constant__ StepConst K, const StepArgs a)
{
    step_body<true, true>(K, a);
}

// Reduce-only: one lane per cell, the bins in order (the pass the step kernel ends with), eight
// bins of loads in flight; 128-thread CTAs.
constexpr int kMomThreads = 128;
template <bool MIXED>
__global__ void __launch_bounds__(kMomThreads)
    moments_kernel(const __grid_constant__ StepConst K, const double *__restrict__ nbp,
                   const double *R, const double *V, double *out)
{
    const long long c = (long long)blockIdx.x * kMomThreads + threadIdx.x;
    if (c < K.C)
        cell_moments<MIXED, 8>(K, R, V, K.C, c, nbp ? PAB_LD(nbp, c, K.C) : K.nb_default, out);
}

__global__ void init_kernel(const __grid_constant__ StepConst K, double rdot_scale, double *R,
                            double *V, float *h)
{
    const size_t n = (size_t)K.B * (size_t)K.C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / (size_t)K.C);
        const double R0 = K.bins[b].R0;
        PAB_ST(R, i, n, R0);
        PAB_ST(V, i, n, rdot_scale * R0);
        PAB_ST(h, i, n, 0.0f);
    }
}


}  // namespace

// SMs of the current device (cached per device).
static int sm_count()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return 152;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 152;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

cudaError_t launch_moments(const StepConst &K, int precision, const double *nb, const double *R,
                           const double *V, double *out, int /*block_warps*/, cudaStream_t s)
{
    const dim3 grid((unsigned)((K.C + kMomThreads - 1) / kMomThreads));
    if (precision == PAB_MIXED)
        moments_kernel<true><<<grid, kMomThreads, 0, s>>>(K, nb, R, V, out);
    else
        moments_kernel<false><<<grid, kMomThreads, 0, s>>>(K, nb, R, V, out);
    return cudaGetLastError();
}

cudaError_t launch_step(const StepConst &K, int precision, const StepArgs &a, int block_warps,
                        cudaStream_t s)
{
    int nw = block_warps <= 0 ? default_warps(precision) : std::min(block_warps, kMaxWarps);
    const long long tiles = (K.C + kTile - 1) / kTile;
    // A CTA of nw warps owns nw tiles.  A grid of fewer tiles than SMs is instead split by bins
    // over more CTAs of one tile each (a latency-bound call: each CTA's trials are serial on its
    // SM's FP64 pipe), one warp per 32 items, and its moments come from the reduce-only kernel
    // afterwards.
    int groups = 1;
    long long ctas = (tiles + nw - 1) / nw;
    const int n_sm = sm_count();
    if (tiles < n_sm && K.B > 1) {
        groups = (int)std::min((long long)K.B, ((long long)n_sm + tiles - 1) / tiles);
        const int per = (K.B + groups - 1) / groups;
        groups = (K.B + per - 1) / per;
        nw = std::min(nw, per);
        ctas = tiles;
    }
    const dim3 grid((unsigned)ctas, (unsigned)groups);
    const bool mixed_adaptive = precision == PAB_MIXED && K.n_fixed == 0;
    const size_t smem = mixed_adaptive ? lot_bytes(kLotPerWarp * nw) : 0;
    // a split grid with a terms buffer and tickets ends with its moments (split_moments)
    const bool terms = groups > 1 && a.out && a.terms && a.tickets;
    if (precision == PAB_MIXED) {
        if (terms)
            step_kernel<true, true><<<grid, nw * 32, smem, s>>>(K, a);
        else
            step_kernel<true, false><<<grid, nw * 32, smem, s>>>(K, a);
    } else {
        if (terms)
            step_kernel<false, true><<<grid, nw * 32, smem, s>>>(K, a);
        else
            step_kernel<false, false><<<grid, nw * 32, smem, s>>>(K, a);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && groups > 1 && a.out && !terms)
        e = launch_moments(K, precision, a.nb, a.R, a.V, a.out, 0, s);
    return e;
}

bool step_splits_by_bins(const StepConst &K)
{
    const long long tiles = (K.C + kTile - 1) / kTile;
    return tiles < sm_count() && K.B > 1;
}

cudaError_t launch_init(const StepConst &K, double Rdot0_ref, double R0ref, double *R, double *V,
                        float *h, cudaStream_t s)
{
    const double scale = (R0ref > 0.0) ? Rdot0_ref / R0ref : 0.0;
    init_kernel<<<152 * 8, 256, 0, s>>>(K, scale, R, V, h);
    return cudaGetLastError();
}

}  // namespace pab
