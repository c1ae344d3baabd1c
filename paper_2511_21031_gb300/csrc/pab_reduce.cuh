// Per-cell quadrature reduction shared by the step kernels: running sums of
// one lane (one cell), the combination of a tile's warps in shared memory with
// the store of the 7 moments, and the CTA's status counters.
#pragma once

#include <cuda_runtime.h>

#include "pab_bits.cuh"
#include "pab_check.cuh"
#include "pab_internal.h"

namespace pab {
namespace {

constexpr int kTile = 32;
constexpr int kMaxWarps = 16;

// Running quadrature sums of one lane (one cell).  FP64 mode: plain FP64
// sums (the pressure sum of w R^3 p_bw/rho).  MIXED mode: the alpha sum
// sum w R^3 is FP64 and compensated (Neumaier); sum w R^3 p_bw splits into
// p0 sum w R^3, formed once per cell from the alpha sum, and an FP32 sum of
// w R^3 (p_bw - p0); sum w R^2 Rdot and sum w R^3 Rdot^2 are FP32 sums of
// FP32 terms.
template <bool MIXED>
struct MomAcc {
    double m3 = 0.0, m3c = 0.0, m2v = 0.0, m3p = 0.0, m3v2 = 0.0;
    float m2vf = 0.0f, m3pf = 0.0f, m3v2f = 0.0f;

    __device__ __forceinline__ void add_m3(double x)
    {
        if (MIXED) {
            neumaier_add(m3, m3c, x);
        } else {
            m3 += x;
        }
    }

    // per-lane totals as doubles
    __device__ __forceinline__ double M2V() const { return MIXED ? f2d(m2vf) : m2v; }
    __device__ __forceinline__ double M3P() const { return MIXED ? f2d(m3pf) : m3p; }
    __device__ __forceinline__ double M3V2() const { return MIXED ? f2d(m3v2f) : m3v2; }
};

// Dynamic shared memory of the kernels that call reduce_and_store: the five
// partial sums of each warp and lane, sized by the launch's warps (a static
// array for the largest CTA would hold L1 capacity that the gas table uses).
constexpr size_t reduce_smem_bytes(int nw) { return (size_t)5 * nw * kTile * sizeof(double); }

// Combine the warps' partial sums of one tile and write the moments.
template <bool MIXED>
__device__ __forceinline__ void reduce_and_store(const StepConst &K, const MomAcc<MIXED> &acc,
                                                 double nb, int64_t c, bool valid, double *out)
{
    extern __shared__ double red[];  // [5][nw][kTile], reduce_smem_bytes(nw)
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const auto at = [&](int m, int w) -> double & { return red[((size_t)m * nw + w) * kTile + lane]; };
    at(0, warp) = acc.m3;
    at(1, warp) = acc.m3c;
    at(2, warp) = acc.M2V();
    at(3, warp) = acc.M3P();
    at(4, warp) = acc.M3V2();
    __syncthreads();
    if (warp == 0 && valid) {
        double m3 = at(0, 0), m3c = at(1, 0);
        double m2v = at(2, 0), m3p = at(3, 0), m3v2 = at(4, 0);
        for (int w = 1; w < nw; ++w) {
            const double x = at(0, w);
            if (MIXED) {
                neumaier_add(m3, m3c, x);
                m3c += at(1, w);
            } else {
                m3 += x;
            }
            m2v += at(2, w);
            m3p += at(3, w);
            m3v2 += at(4, w);
        }
        if (MIXED)
            m3 += m3c;
        const double alpha = (4.0 / 3.0 * 3.14159265358979323846) * nb * m3;
        const double inv_m3 = 1.0 / m3;
        const int64_t C = K.C;
        const long long no = 7 * C;
        PAB_ST(out, 0 * C + c, no, nb);
        PAB_ST(out, 1 * C + c, no, alpha);
        PAB_ST(out, 2 * C + c, no, m3);
        PAB_ST(out, 3 * C + c, no, m2v);
        PAB_ST(out, 4 * C + c, no, 3.0 * alpha * m2v * inv_m3);
        PAB_ST(out, 5 * C + c, no, MIXED ? fma(m3p, inv_m3, K.p0) : K.rho * m3p * inv_m3);
        PAB_ST(out, 6 * C + c, no, m3v2 * inv_m3);
    }
}

// Block-wide sums of the status counters, one atomic per CTA and counter.
__device__ __forceinline__ void flush_counters(uint32_t fl_or, uint32_t n_flag, uint32_t n_att,
                                               uint32_t n64, Counters *cnt)
{
    __shared__ uint32_t sc[4][kMaxWarps];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    fl_or = __reduce_or_sync(0xffffffffu, fl_or);
    n_flag = __reduce_add_sync(0xffffffffu, n_flag);
    n_att = __reduce_add_sync(0xffffffffu, n_att);
    n64 = __reduce_add_sync(0xffffffffu, n64);
    if (lane == 0) {
        sc[0][warp] = fl_or;
        sc[1][warp] = n_flag;
        sc[2][warp] = n_att;
        sc[3][warp] = n64;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t f = 0;
        unsigned long long a = 0, b = 0, d = 0;
        for (int w = 0; w < nw; ++w) {
            f |= sc[0][w];
            a += sc[1][w];
            b += sc[2][w];
            d += sc[3][w];
        }
        if (f)
            atomicOr(&cnt->flags_or, f);
        if (a)
            atomicAdd(&cnt->n_flagged, a);
        if (b)
            atomicAdd(&cnt->n_attempts, b);
        if (d)
            atomicAdd(&cnt->n_fp64, d);
    }
}

__host__ __device__ inline int clamp_warps(int w, int B)
{
    if (w <= 0)
        w = kDefaultWarps;
    if (w > kMaxWarps)
        w = kMaxWarps;
    if (w > B)
        w = B;
    return w < 1 ? 1 : w;
}

}  // namespace
}  // namespace pab
