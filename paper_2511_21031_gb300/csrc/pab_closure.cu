// Kernels of the carrier-facing forms (include/pab_closure.h): conservative
// bubble variables n_b R_i, n_b Rdot_i (Listing 2, Eq. e:ndf), the mixture
// pressure of Eq. (e:pressure) and the stiffened-gas liquid pressure of
// Eq. (eos_liquid).  All are memory-bound elementwise or per-cell passes.
#include <cuda_runtime.h>

#include "pab_bits.cuh"
#include "pab_check.cuh"
#include "pab_internal.h"
#include "pab_intmul.cuh"

PAB_CHECK_UNIT(closure)

namespace pab {
namespace {

// qR = n_b R, qV = n_b Rdot; grid.y walks the bins, grid.x the cells.
__global__ void cons_from_prim_kernel(long long C, const double *__restrict__ nb, double nb_default,
                                      const double *__restrict__ R, const double *__restrict__ V,
                                      double *__restrict__ qR, double *__restrict__ qV)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C)
        return;
    const size_t k = (size_t)blockIdx.y * (size_t)C + (size_t)c;
    const long long ns = (long long)gridDim.y * C;
    const double n = nb ? PAB_LD(nb, c, C) : nb_default;
    PAB_ST(qR, k, ns, n * PAB_LD(R, k, ns));
    PAB_ST(qV, k, ns, n * PAB_LD(V, k, ns));
}

// One thread per cell: the sum of w qR^3 over the bins, n_b = sqrt(4/3 pi S / alpha), then the
// rescale of every bin.  Consecutive threads read consecutive cells of one bin row (coalesced),
// and the bin loops are unrolled so that each thread keeps a chunk of loads in flight; the
// second read of qR comes from L2 (a CTA's rows were just read).  Each (bin, cell) takes three
// products (the cube of qR, and qR and qV times 1/n_b) and one FMA into the sum: in FP64, at
// GB300's 2 FP64 operations per clock and SM, the five would take longer than the 32 bytes take
// to stream, so the products are formed on the integer pipe (pab_intmul.cuh, within 1 ulp of
// the FP64 ones) and the FMA alone runs in FP64.  Small CTAs at 32 registers keep 64 warps on
// each SM, which matters more here than deeper unrolling (a few spilled registers cost less
// than half the warps).  A layout with the bins spread over a CTA's warps, each value read once
// and kept in registers, ran slower: a CTA then touches each of 62 rows for 256 bytes only.
constexpr int kCellsPerCta = 128;
constexpr int kUnroll = 4;     // rescale: qR and qV of 4 bins in flight per thread
constexpr int kUnrollSum = 8;  // sum: qR of 8 bins in flight per thread
__global__ void __launch_bounds__(kCellsPerCta, 16)
    prim_from_cons_kernel(const __grid_constant__ StepConst K, const double *__restrict__ alpha,
                          const double *__restrict__ qR, const double *__restrict__ qV,
                          double *__restrict__ R, double *__restrict__ V, double *__restrict__ nb_out)
{
    // the weights in shared memory: read per bin by every thread, they would otherwise be indexed
    // constant-bank loads on the sum's critical path
    __shared__ double sw[PAB_MAX_BINS];
    for (int b = threadIdx.x; b < K.B; b += blockDim.x)
        sw[b] = K.bins[b].w;
    __syncthreads();
    const long long c = (long long)blockIdx.x * kCellsPerCta + threadIdx.x;
    if (c >= K.C)
        return;
    const size_t C = (size_t)K.C;
    const long long ns = (long long)K.B * K.C;
    // the bins in whole chunks, every load of a chunk issued before its arithmetic, then the rest
    // in fours and ones (a predicated last chunk would run its FP64 operations for the missing
    // bins too)
    bool ok = true;
    double s = 0.0;
    int b = 0;
    for (; b + kUnrollSum <= K.B; b += kUnrollSum) {
        double q[kUnrollSum];
#pragma unroll
        for (int i = 0; i < kUnrollSum; ++i)
            q[i] = PAB_LD(qR, (size_t)(b + i) * C + (size_t)c, ns);
#pragma unroll
        for (int i = 0; i < kUnrollSum; ++i)
            s = fma(sw[b + i], cube_int(q[i], ok), s);
    }
    for (; b + 4 <= K.B; b += 4) {
        double q[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            q[i] = PAB_LD(qR, (size_t)(b + i) * C + (size_t)c, ns);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            s = fma(sw[b + i], cube_int(q[i], ok), s);
    }
    for (; b < K.B; ++b)
        s = fma(sw[b], cube_int(PAB_LD(qR, (size_t)b * C + (size_t)c, ns), ok), s);
    if (!ok) {
        // a subnormal, infinite or NaN value, or a cube outside the normal range: the sum in FP64
        s = 0.0;
        for (b = 0; b < K.B; ++b) {
            const double q = PAB_LD(qR, (size_t)b * C + (size_t)c, ns);
            s = fma(sw[b] * q, q * q, s);
        }
    }
    // n_b = sqrt(4/3 pi S / alpha) and 1/n_b from one reciprocal and one inverse square root,
    // which leave the FP64 pipe less to do than an IEEE square root and two divisions
    double n = (double)NAN, in = (double)NAN;
    const double a = PAB_LD(alpha, c, K.C);
    if (a > 0.0 && a <= 1.0e300) {
        const double x = (4.0 / 3.0 * 3.14159265358979323846) * s * rcp64(a);
        in = rsqrt64(x);
        n = x * in;
    }
    if (nb_out)
        PAB_ST(nb_out, c, K.C, n);
    const IntFactor f = int_factor(in);
    ok = f.normal;
    if (ok) {
        b = 0;
        for (; b + kUnroll <= K.B; b += kUnroll) {
            double qr[kUnroll], qv[kUnroll];
#pragma unroll
            for (int i = 0; i < kUnroll; ++i) {
                const size_t k = (size_t)(b + i) * C + (size_t)c;
                qr[i] = PAB_LD(qR, k, ns);
                qv[i] = PAB_LD(qV, k, ns);
            }
#pragma unroll
            for (int i = 0; i < kUnroll; ++i) {
                const size_t k = (size_t)(b + i) * C + (size_t)c;
                PAB_ST(R, k, ns, mul_int(qr[i], f, ok));
                PAB_ST(V, k, ns, mul_int(qv[i], f, ok));
            }
        }
        for (; b < K.B; ++b) {
            const size_t k = (size_t)b * C + (size_t)c;
            PAB_ST(R, k, ns, mul_int(PAB_LD(qR, k, ns), f, ok));
            PAB_ST(V, k, ns, mul_int(PAB_LD(qV, k, ns), f, ok));
        }
    }
    if (!ok) {
        // 1/n_b or a value not normal, or a product outside the normal range: the cell's
        // products again in FP64, over what the fast loop stored
        for (b = 0; b < K.B; ++b) {
            const size_t k = (size_t)b * C + (size_t)c;
            PAB_ST(R, k, ns, PAB_LD(qR, k, ns) * in);
            PAB_ST(V, k, ns, PAB_LD(qV, k, ns) * in);
        }
    }
}

__global__ void mixture_pressure_kernel(long long C, const double *__restrict__ m,
                                        const double *__restrict__ p_l,
                                        const double *__restrict__ rho_l, double rho_default,
                                        double *__restrict__ p)
{
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        const double a = PAB_LD(m, 1 * C + c, 7 * C);
        const double rho = rho_l ? PAB_LD(rho_l, c, C) : rho_default;
        PAB_ST(p, c, C, (1.0 - a) * PAB_LD(p_l, c, C) + a * (PAB_LD(m, 5 * C + c, 7 * C) - rho * PAB_LD(m, 6 * C + c, 7 * C)));
    }
}

__global__ void stiffened_gas_kernel(long long n, const double *__restrict__ rho,
                                     const double *__restrict__ e, double gm1, double gpi,
                                     double *__restrict__ p)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        PAB_ST(p, i, n, gm1 * PAB_LD(rho, i, n) * PAB_LD(e, i, n) - gpi);
}

unsigned grid_for(long long n, int threads)
{
    long long g = (n + threads - 1) / threads;
    const long long cap = 152LL * 32;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t launch_cons_from_prim(const StepConst &K, const double *nb, const double *R,
                                  const double *V, double *qR, double *qV, cudaStream_t s)
{
    const dim3 grid((unsigned)((K.C + 255) / 256), (unsigned)K.B);
    cons_from_prim_kernel<<<grid, 256, 0, s>>>(K.C, nb, K.nb_default, R, V, qR, qV);
    return cudaGetLastError();
}

cudaError_t launch_prim_from_cons(const StepConst &K, const double *alpha, const double *qR,
                                  const double *qV, double *R, double *V, double *nb_out,
                                  cudaStream_t s)
{
    const dim3 grid((unsigned)((K.C + kCellsPerCta - 1) / kCellsPerCta));
    prim_from_cons_kernel<<<grid, kCellsPerCta, 0, s>>>(K, alpha, qR, qV, R, V, nb_out);
    return cudaGetLastError();
}

cudaError_t launch_mixture_pressure(long long C, const double *moments, const double *p_l,
                                    const double *rho_l, double rho_default, double *p,
                                    cudaStream_t s)
{
    mixture_pressure_kernel<<<grid_for(C, 256), 256, 0, s>>>(C, moments, p_l, rho_l, rho_default, p);
    return cudaGetLastError();
}

cudaError_t launch_stiffened_gas(long long n, const double *rho, const double *e, double gamma_l,
                                 double pi_inf, double *p, cudaStream_t s)
{
    stiffened_gas_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, rho, e, gamma_l - 1.0,
                                                          gamma_l * pi_inf, p);
    return cudaGetLastError();
}

}  // namespace pab
