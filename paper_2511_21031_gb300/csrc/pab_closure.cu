// Kernels of the carrier-facing forms (include/pab_closure.h): conservative
// bubble variables n_b R_i, n_b Rdot_i (Listing 2, Eq. e:ndf), the mixture
// pressure of Eq. (e:pressure) and the stiffened-gas liquid pressure of
// Eq. (eos_liquid).  All are memory-bound elementwise or per-cell passes.
#include <cuda_runtime.h>

#include "pab_internal.h"

namespace pab {
namespace {

constexpr int kTile = 32;
constexpr int kWarps = 8;

// qR = n_b R, qV = n_b Rdot; grid.y walks the bins, grid.x the cells.
__global__ void cons_from_prim_kernel(long long C, const double *__restrict__ nb, double nb_default,
                                      const double *__restrict__ R, const double *__restrict__ V,
                                      double *__restrict__ qR, double *__restrict__ qV)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C)
        return;
    const size_t k = (size_t)blockIdx.y * (size_t)C + (size_t)c;
    const double n = nb ? nb[c] : nb_default;
    qR[k] = n * R[k];
    qV[k] = n * V[k];
}

// Per 32-cell tile: the warps sum w qR^3 over a strided subset of bins, the
// partial sums meet in shared memory, n_b = sqrt(4/3 pi S / alpha), then every
// warp rescales its bins.
__global__ void __launch_bounds__(kWarps * 32)
    prim_from_cons_kernel(const __grid_constant__ StepConst K, const double *__restrict__ alpha,
                          const double *__restrict__ qR, const double *__restrict__ qV,
                          double *__restrict__ R, double *__restrict__ V, double *__restrict__ nb_out)
{
    __shared__ double part[kWarps][kTile];
    __shared__ double inv_nb[kTile];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long c = (long long)blockIdx.x * kTile + lane;
    const bool valid = c < K.C;
    double s = 0.0;
    for (int b = warp; b < K.B; b += kWarps) {
        if (valid) {
            const double q = qR[(size_t)b * (size_t)K.C + (size_t)c];
            s += K.bins[b].w * q * q * q;
        }
    }
    part[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
        double S = 0.0;
        for (int w = 0; w < kWarps; ++w)
            S += part[w][lane];
        double n = (double)NAN;
        if (valid) {
            const double a = alpha[c];
            if (a > 0.0 && a <= 1.0e300)
                n = sqrt((4.0 / 3.0 * 3.14159265358979323846) * S / a);
            if (nb_out)
                nb_out[c] = n;
        }
        inv_nb[lane] = 1.0 / n;
    }
    __syncthreads();
    if (!valid)
        return;
    const double in = inv_nb[lane];
    for (int b = warp; b < K.B; b += kWarps) {
        const size_t k = (size_t)b * (size_t)K.C + (size_t)c;
        R[k] = qR[k] * in;
        V[k] = qV[k] * in;
    }
}

__global__ void mixture_pressure_kernel(long long C, const double *__restrict__ m,
                                        const double *__restrict__ p_l,
                                        const double *__restrict__ rho_l, double rho_default,
                                        double *__restrict__ p)
{
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        const double a = m[1 * C + c];
        const double rho = rho_l ? rho_l[c] : rho_default;
        p[c] = (1.0 - a) * p_l[c] + a * (m[5 * C + c] - rho * m[6 * C + c]);
    }
}

__global__ void stiffened_gas_kernel(long long n, const double *__restrict__ rho,
                                     const double *__restrict__ e, double gm1, double gpi,
                                     double *__restrict__ p)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = gm1 * rho[i] * e[i] - gpi;
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
    const dim3 grid((unsigned)((K.C + kTile - 1) / kTile));
    prim_from_cons_kernel<<<grid, kWarps * 32, 0, s>>>(K, alpha, qR, qV, R, V, nb_out);
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
