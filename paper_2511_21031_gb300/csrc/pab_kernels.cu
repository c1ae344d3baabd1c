// Kernels of the bubble source update on sm_103a.
//
// Work decomposition: a CTA owns a tile of 32 consecutive cells (one per
// lane) and all Nb bins of those cells; its warps stride over the bins.  All
// lanes of a warp therefore advance the same bin of 32 neighbouring cells:
// loads and stores of the bin-major state are 256-byte coalesced, the bin
// constants are warp-uniform constant-bank reads, and neighbouring cells
// (similar pressure) need similar sub-step counts, which keeps the adaptive
// loop's divergence low.  Each lane keeps running quadrature sums for its
// cell over the bins its warp visits; the warps' partial sums are combined in
// shared memory and one warp writes the 7 moments of the 32 cells.  No
// atomics touch the state: every (bin, cell) has one owner (Sec. 4).
#include <cuda_runtime.h>

#include "pab_device.cuh"
#include "pab_internal.h"
#include "pab_reduce.cuh"

namespace pab {
namespace {

// FP64 mode (and the reduce-only kernel in both modes): terms from the FP64 state.
template <bool MIXED>
__device__ __forceinline__ void accumulate(const StepConst &K, const BinConst &bc, double R,
                                           double V, MomAcc<MIXED> &acc, GasBase &g)
{
    const double wr2 = bc.w * R * R;
    const double wr3 = wr2 * R;
    if (MIXED) {
        const float xi = d2f(R - bc.R0);
        const float Rf = d2f(R);
        const float Vf = d2f(V);
        const float u = xi * bc.invR0f;
        const float pgdev = (K.gas_mode == PAB_GAS_POLYTROPIC) ? gas_dev32(K, bc, u) : 0.0f;
        const float dev = pgdev + div32(K.two_sigmaf * u - K.four_muf * Vf, Rf);
        const float wr3f = d2f(wr3);
        acc.add_m3(wr3);
        acc.m3pf = fmaf(wr3f, bc.dpeqf + dev, acc.m3pf);
        acc.m2vf = fmaf(d2f(wr2), Vf, acc.m2vf);
        acc.m3v2f = fmaf(wr3f * Vf, Vf, acc.m3v2f);
    } else {
        // w R^3 p_bw/rho = w R^3 p_b/rho - w R^2 s/rho, s = 4 mu Rdot + 2 sigma
        acc.add_m3(wr3);
        acc.m2v = fma(wr2, V, acc.m2v);
        acc.m3p = fma(wr3, bubble_pressure_rho64(K, bc, R, g), acc.m3p);
        acc.m3p = fma(-wr2, fma(K.fmu_rho, V, K.tsig_rho), acc.m3p);
        acc.m3v2 = fma(wr3 * V, V, acc.m3v2);
    }
}

// MIXED step kernel: the FP32 images xi = R - R0 and Rdot the advance left
// behind spare their conversions; w R^3 stays FP64 for the compensated sum.
template <bool MIXED>
__device__ __forceinline__ void accumulate_mixed(const StepConst &K, const BinConst &bc, double R,
                                                 float xi, float v, MomAcc<MIXED> &acc)
{
    const float Rf = bc.R0f + xi;
    const float u = xi * bc.invR0f;
    const float pgdev = (K.gas_mode == PAB_GAS_POLYTROPIC) ? gas_dev32(K, bc, u) : 0.0f;
    const float iRf = rcp32(Rf);
    const float dev = pgdev + (K.two_sigmaf * u - K.four_muf * v) * iRf;
    const double wr3 = bc.w * R * R * R;
    const float wr3f = d2f(wr3);
    const float wr2f = wr3f * iRf;  // w R^2 = w R^3 / R
    acc.add_m3(wr3);
    acc.m3pf = fmaf(wr3f, bc.dpeqf + dev, acc.m3pf);
    acc.m2vf = fmaf(wr2f, v, acc.m2vf);
    acc.m3v2f = fmaf(wr3f * v, v, acc.m3v2f);
}

template <bool MIXED>
__device__ __forceinline__ void step_body(const StepConst &K, const StepArgs a)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * kTile + lane;
    const bool valid = c < K.C;
    const double p_inf = valid ? a.p_inf[c] : K.p0;
    const bool p_ok = finite64(p_inf);
    const double nb = valid ? (a.nb ? a.nb[c] : K.nb_default) : 0.0;

    MomAcc<MIXED> acc;
    uint32_t fl_or = 0, n_flag = 0, n_att = 0, n64 = 0;
    const float dp_cell = MIXED ? d2f(K.p0 - p_inf) : 0.0f;  // p_eq - p_inf = dpeq + dp_cell
    for (int b = warp; b < K.B; b += nw) {
        if (!valid)
            continue;
        const BinConst &bc = K.bins[b];
        const size_t k = (size_t)b * (size_t)K.C + (size_t)c;
        double R = a.R[k];
        double V = a.V[k];
        uint32_t fl = 0;
        int na = 0;
        GasBase g;
        g.reset();
        if (!p_ok || !finite64(R) || !finite64(V)) {
            fl = PAB_FLAG_NONFINITE;
        } else if (MIXED && K.n_fixed == 0) {  // (only reachable in the MIXED instantiation)
            const float A = bc.dpeqf + dp_cell;
            float hc = a.h[k];
            int nd = 0;
            float xi, v;
            fl = advance_mixed(K, bc, p_inf, A, a.dt, R, V, hc, na, nd, xi, v);
            a.h[k] = hc;
            n64 += nd;
            // the checks read the FP32 images of the new state
            if (!isfinite(xi) || !isfinite(v))
                fl |= PAB_FLAG_NONFINITE;
            else if (!(bc.R0f + xi > 0.0f))
                fl |= PAB_FLAG_NONPOS;
            if (fabsf(v) >= K.cf)
                fl |= PAB_FLAG_SUPERSONIC;
            a.R[k] = R;
            a.V[k] = V;
            // a finite state has finite FP32 images (|R - R0| and |Rdot| are far below the
            // FP32 range) and a non-finite one gives NaN moments either way
            if (a.out)
                accumulate_mixed<MIXED>(K, bc, R, xi, v, acc);
            if (a.attempts)
                a.attempts[k] = na;
            fl_or |= fl;
            n_flag += (fl != 0);
            n_att += na;
            continue;
        } else {
            const float A = MIXED ? bc.dpeqf + dp_cell : 0.0f;
            if (K.n_fixed > 0) {
                advance_fixed<MIXED>(K, bc, p_inf, A, a.dt_sub, R, V, g);
                na = K.n_fixed;
            } else {
                float hc = a.h[k];
                fl = advance_adaptive(K, bc, p_inf, a.dt, R, V, hc, na, g);
                a.h[k] = hc;
            }
            if (!finite64(R) || !finite64(V))
                fl |= PAB_FLAG_NONFINITE;
            else if (!gt0(R))
                fl |= PAB_FLAG_NONPOS;
            if (abs_ge(V, K.c))
                fl |= PAB_FLAG_SUPERSONIC;
            a.R[k] = R;
            a.V[k] = V;
        }
        if (a.attempts)
            a.attempts[k] = na;
        fl_or |= fl;
        n_flag += (fl != 0);
        n_att += na;
        if (a.out)
            accumulate<MIXED>(K, bc, R, V, acc, g);
    }
    if (a.out)
        reduce_and_store<MIXED>(K, acc, nb, c, valid, a.out);
    flush_counters(fl_or, n_flag, n_att, n64, a.counters);
}

// One kernel per precision with its own register bound.  MIXED: 64 registers
// (kMaxWarps x 32 threads x 2 CTAs), so 8 CTAs of the default 4 warps fit on an
// SM; left to itself the compiler takes 110 and 4 CTAs fit (13.2e9 against
// 17.5e9 bin-steps/s on the 128^3 x 31 line).  FP64: no minimum, where the
// compiler settles on 64 registers itself (3 % faster than 64 under the bound).
template <bool MIXED>
__global__ void step_kernel(const __grid_constant__ StepConst K, const StepArgs a);
template <>
__global__ void __launch_bounds__(kMaxWarps * 32)
    step_kernel<false>(const __grid_constant__ StepConst K, const StepArgs a)
{
    step_body<false>(K, a);
}
template <>
__global__ void __launch_bounds__(kMaxWarps * 32, 2)
    step_kernel<true>(const __grid_constant__ StepConst K, const StepArgs a)
{
    step_body<true>(K, a);
}

template <bool MIXED>
__global__ void __launch_bounds__(kMaxWarps * 32)
    moments_kernel(const __grid_constant__ StepConst K, const double *__restrict__ nbp,
                   const double *__restrict__ Rp, const double *__restrict__ Vp,
                   double *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * kTile + lane;
    const bool valid = c < K.C;
    const double nb = valid ? (nbp ? nbp[c] : K.nb_default) : 0.0;
    MomAcc<MIXED> acc;
    for (int b = warp; b < K.B; b += nw) {
        if (!valid)
            continue;
        const size_t k = (size_t)b * (size_t)K.C + (size_t)c;
        GasBase g;
        g.reset();
        accumulate<MIXED>(K, K.bins[b], Rp[k], Vp[k], acc, g);
    }
    reduce_and_store<MIXED>(K, acc, nb, c, valid, out);
}

__global__ void init_kernel(const __grid_constant__ StepConst K, double rdot_scale, double *R,
                            double *V, float *h)
{
    const size_t n = (size_t)K.B * (size_t)K.C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / (size_t)K.C);
        const double R0 = K.bins[b].R0;
        R[i] = R0;
        V[i] = rdot_scale * R0;
        h[i] = 0.0f;
    }
}


}  // namespace

cudaError_t launch_step(const StepConst &K, int precision, const StepArgs &a, int block_warps,
                        cudaStream_t s)
{
    const int nw = clamp_warps(block_warps, K.B);
    const dim3 grid((unsigned)((K.C + kTile - 1) / kTile));
    if (precision == PAB_MIXED)
        step_kernel<true><<<grid, nw * 32, reduce_smem_bytes(nw), s>>>(K, a);
    else
        step_kernel<false><<<grid, nw * 32, reduce_smem_bytes(nw), s>>>(K, a);
    return cudaGetLastError();
}

cudaError_t launch_moments(const StepConst &K, int precision, const double *nb, const double *R,
                           const double *V, double *out, int block_warps, cudaStream_t s)
{
    const int nw = clamp_warps(block_warps, K.B);
    const dim3 grid((unsigned)((K.C + kTile - 1) / kTile));
    if (precision == PAB_MIXED)
        moments_kernel<true><<<grid, nw * 32, reduce_smem_bytes(nw), s>>>(K, nb, R, V, out);
    else
        moments_kernel<false><<<grid, nw * 32, reduce_smem_bytes(nw), s>>>(K, nb, R, V, out);
    return cudaGetLastError();
}

cudaError_t launch_init(const StepConst &K, double Rdot0_ref, double R0ref, double *R, double *V,
                        float *h, cudaStream_t s)
{
    const double scale = (R0ref > 0.0) ? Rdot0_ref / R0ref : 0.0;
    init_kernel<<<152 * 8, 256, 0, s>>>(K, scale, R, V, h);
    return cudaGetLastError();
}

}  // namespace pab
