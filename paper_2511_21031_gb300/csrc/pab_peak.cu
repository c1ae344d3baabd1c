// FMA throughput microbenchmark (measurement aid for the roofline).
#include <cuda_runtime.h>

#include <cfloat>

#include <vector>

#include "pab_device.cuh"
#include "pab_exp.cuh"
#include "pab_intmul.cuh"
#include "pab_internal.h"
#include "pab_measure.h"

namespace {

template <typename T>
__global__ void fma_streams(int iters, double *sink)
{
    T a0 = (T)threadIdx.x * (T)1e-3, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
    T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
    const T m = (T)0.999999, c = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a0 = a0 * m + c; a1 = a1 * m + c; a2 = a2 * m + c; a3 = a3 * m + c;
            a4 = a4 * m + c; a5 = a5 * m + c; a6 = a6 * m + c; a7 = a7 * m + c;
        }
    }
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] =
        (double)(a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7);
}

__global__ void math_check_kernel(const __grid_constant__ pab::StepConst K, const double *tab,
                                  long long n, const double *R, const double *Rb, double *gas,
                                  double *gas_tab, double *exact)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const pab::BinConst &bc = K.bins[0];  // R0 = 1
        pab::GasBase g;
        g.reset();
        (void)pab::gas_factor(K, bc, Rb[i], g);  // exact at the base
        gas[i] = pab::gas_factor(K, bc, R[i], g);
        pab::StepConst Kt = K;  // the same constants with the node table attached
        Kt.gas_tab = tab;
        pab::GasBase g2;
        g2.reset();
        gas_tab[i] = pab::gas_factor(Kt, Kt.bins[0], R[i], g2);
        exact[i] = exp(K.three_gamma * log(1.0 / R[i]));
    }
}

__global__ void bits_check_kernel(long long n, const float *f, const double *x, const double *y,
                                  double *f2d, double *f2d_hw, double *rcp, double *dv, double *seed,
                                  uint16_t *cmp)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        f2d[i] = pab::f2d(f[i]);
        f2d_hw[i] = (double)f[i];
        const double xi = x[i], yi = y[i];
        rcp[i] = pab::rcp64(xi);
        dv[i] = 1.0 / xi;
        double s0;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(s0) : "d"(xi));
        seed[i] = s0;
        const double ax = fabs(xi);
        uint32_t bad = 0;
        bad |= (pab::gt0(xi) != (xi > 0.0)) << 0;
        bad |= (pab::le(xi, yi) != (xi <= yi)) << 1;
        bad |= (pab::finite64(xi) != (bool)isfinite(xi)) << 2;
        bad |= (pab::abs_ge(xi, yi) != (ax >= yi)) << 3;
        if (!isnan(xi)) {  // the max/min helpers take numbers >= +0
            bad |= (pab::ubits(pab::max_nn(ax, yi)) != pab::ubits(fmax(ax, yi))) << 4;
            bad |= (pab::ubits(pab::min_nn(ax, yi)) != pab::ubits(fmin(ax, yi))) << 5;
            // the library flushes subnormal float results to a signed zero
            float hw = __double2float_rn(xi);
            if (fabsf(hw) < FLT_MIN)
                hw = copysignf(0.0f, hw);
            bad |= (__float_as_uint(pab::d2f(xi)) != __float_as_uint(hw)) << 6;
            // 2x on the integer units, for |x| and for a subnormal made from its bits
            const double sub = pab::from_bits(pab::ubits(ax) >> 12);
            if (ax < 0x1p1023)
                bad |= (pab::ubits(pab::twice_nn(ax)) != pab::ubits(__dadd_rn(ax, ax))) << 8;
            bad |= (pab::ubits(pab::twice_nn(sub)) != pab::ubits(__dadd_rn(sub, sub))) << 8;
        } else {
            bad |= (!isnan(pab::d2f(xi))) << 6;
        }
        // the embedded difference against the same quantity in FP64: within
        // 2^-46 of the terms (the library combines the two FP32 rounding errors
        // in FP32, an error of at most 2^-47 of them; the FP64 reference rounds
        // twice)
        const float k1 = f[i], k2 = __double2float_rn(xi), k3 = __double2float_rn(yi);
        if (isfinite(k1) && isfinite(k2) && isfinite(k3) && fabsf(k1) < 0x1p100f &&
            fabsf(k2) < 0x1p100f && fabsf(k3) < 0x1p100f) {  // the helper's domain
            const double ref = 2.0 * (double)k3 - ((double)k1 + (double)k2);
            float d32;
            const double got = pab::embedded_diff(k1, k2, k3, d32);
            const double tol = 0x1p-46 * (fabs(2.0 * (double)k3) + fabs((double)k1) +
                                           fabs((double)k2));
            bad |= (!(fabs(got - ref) <= tol)) << 7;
        }
        // the short float -> double on its domain (finite, |f| < 2^104)
        if (isfinite(f[i]) && fabsf(f[i]) < 0x1p104f)
            bad |= (pab::ubits(pab::f2d_fin(f[i])) != pab::ubits((double)f[i])) << 11;
        // FP32 quotient and reciprocal from the approximate seed, within an ulp of
        // the IEEE operations on their domain (normal operands and results between
        // 2^-100 and 2^100 in magnitude)
        const float qa = f[i], qb = __double2float_rn(xi);
        const auto in_dom = [](float z) { return fabsf(z) >= 0x1p-100f && fabsf(z) <= 0x1p100f; };
        if (in_dom(qa) && in_dom(qb) && in_dom(qa / qb)) {
            const float q = pab::div32(qa, qb), qr = __fdiv_rn(qa, qb);
            const float r = pab::rcp32(qb), rr = __frcp_rn(qb);
            const int dq = abs((int)__float_as_uint(q) - (int)__float_as_uint(qr));
            const int dr = abs((int)__float_as_uint(r) - (int)__float_as_uint(rr));
            bad |= (dq > 1) << 9;
            bad |= (dr > 1) << 10;
        }
        cmp[i] = (uint16_t)bad;
    }
}

}  // namespace

extern "C" pab_status pab_bits_check(int64_t n, const float *f_dev, const double *x_dev,
                                     const double *y_dev, double *f2d_dev, double *f2d_hw,
                                     double *rcp_dev, double *div_dev, double *seed_dev,
                                     uint16_t *cmp_dev, void *stream)
{
    if (n < 0 || (n > 0 && (!f_dev || !x_dev || !y_dev || !f2d_dev || !f2d_hw || !rcp_dev ||
                            !div_dev || !seed_dev || !cmp_dev)))
        return PAB_EINVAL;
    if (n == 0)
        return PAB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    bits_check_kernel<<<152 * 4, 256, 0, s>>>(n, f_dev, x_dev, y_dev, f2d_dev, f2d_hw, rcp_dev,
                                               div_dev, seed_dev, cmp_dev);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? PAB_OK : PAB_ECUDA;
}

namespace {
__global__ void accept_check_kernel(const __grid_constant__ pab::StepConst K, long long n,
                                    const double *trial, const float *k, uint8_t *out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        pab::Trial t;
        t.R = trial[4 * i + 0];
        t.V = trial[4 * i + 1];
        t.eR = trial[4 * i + 2];
        t.eV = trial[4 * i + 3];
        t.ok = true;
        const double aR = pab::abs_nn(t.R);
        const double vs = pab::max_nn(pab::abs_nn(t.V), K.v_floor);
        out[4 * i + 0] = ((uint8_t)pab::decide64(K, t).accept);
        out[4 * i + 1] =
            (uint8_t)(pab::le(pab::abs_nn(t.eR), K.tol3 * aR) && pab::le(pab::abs_nn(t.eV), K.tol3 * vs));
        const float k1 = k[4 * i + 0], k2 = k[4 * i + 1];
        const float k3 = k[4 * i + 2], T = k[4 * i + 3];
        float d1, d2;
        out[4 * i + 2] = ((uint8_t)pab::embedded_within(k1, k2, k3, T, d1));
        out[4 * i + 3] =
            (uint8_t)pab::le(pab::abs_nn(pab::embedded_diff(k1, k2, k3, d2)), pab::f2d_fin(T));
    }
}

__global__ void exp_check_kernel(long long n, const double *x, double *mine, double *lib)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        mine[i] = pab::exp_tab(x[i]);
        lib[i] = exp(x[i]);
    }
}

__global__ void intmul_check_kernel(long long n, const double *x, const double *y, double *prod,
                                    double *cube, double *rcp)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        bool ok = true;
        const double p = pab::mul_int(x[i], pab::int_factor(y[i]), ok);
        prod[i] = ok ? p : x[i] * y[i];
        ok = true;
        const double c = pab::cube_int(x[i], ok);
        cube[i] = ok ? c : x[i] * x[i] * x[i];
        ok = true;
        const double r = pab::rcp_int(x[i], ok);
        rcp[i] = ok ? r : 1.0 / x[i];
    }
}

__global__ void gas32_check_kernel(long long n, const float *u, float a, float *out, float *lib)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        out[i] = pab::pow_m1_32(u[i], a);
        lib[i] = expm1f(-a * log1pf(u[i]));
    }
}
}  // namespace

extern "C" pab_status pab_accept_check(int64_t n, const double *trial_dev, const float *k_dev,
                                       double tol, double v_floor, uint8_t *out_dev, void *stream)
{
    if (n < 0 || (n > 0 && (!trial_dev || !k_dev || !out_dev)) || !(tol > 0.0) || !(tol < 1.0) ||
        !(v_floor >= 0.0) || !std::isfinite(v_floor))
        return PAB_EINVAL;
    if (n == 0)
        return PAB_OK;
    pab_config c;
    pab_config_default(&c);
    c.n_cells = 1;
    c.n_bins = 1;
    c.tol = tol;
    c.v_floor = v_floor;
    const double R0 = 1e-5, w = 1.0;
    pab::StepConst K;
    pab::make_const(&c, &R0, &w, &K);
    cudaStream_t s = (cudaStream_t)stream;
    accept_check_kernel<<<152 * 4, 256, 0, s>>>(K, n, trial_dev, k_dev, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? PAB_OK : PAB_ECUDA;
}

extern "C" pab_status pab_exp_check(int64_t n, const double *x_dev, double *mine_dev, double *lib_dev,
                                    void *stream)
{
    if (n < 0 || (n > 0 && (!x_dev || !mine_dev || !lib_dev)))
        return PAB_EINVAL;
    if (n == 0)
        return PAB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    exp_check_kernel<<<152 * 4, 256, 0, s>>>(n, x_dev, mine_dev, lib_dev);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? PAB_OK : PAB_ECUDA;
}

extern "C" pab_status pab_intmul_check(int64_t n, const double *x_dev, const double *y_dev,
                                       double *prod_dev, double *cube_dev, double *rcp_dev,
                                       void *stream)
{
    if (n < 0 || (n > 0 && (!x_dev || !y_dev || !prod_dev || !cube_dev || !rcp_dev)))
        return PAB_EINVAL;
    if (n == 0)
        return PAB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    intmul_check_kernel<<<152 * 4, 256, 0, s>>>(n, x_dev, y_dev, prod_dev, cube_dev, rcp_dev);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? PAB_OK : PAB_ECUDA;
}

extern "C" pab_status pab_gas32_check(int64_t n, const float *u_dev, float a, float *out_dev,
                                      float *lib_dev, void *stream)
{
    if (n < 0 || !(a > 0.0f) || (n > 0 && (!u_dev || !out_dev || !lib_dev)))
        return PAB_EINVAL;
    if (n == 0)
        return PAB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    gas32_check_kernel<<<152 * 4, 256, 0, s>>>(n, u_dev, a, out_dev, lib_dev);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? PAB_OK : PAB_ECUDA;
}

extern "C" pab_status pab_math_check(int64_t n, const double *R_dev, const double *Rb_dev, double a,
                                     double *gas_dev, double *gas_tab_dev, double *exact_dev,
                                     void *stream)
{
    if (n < 0 || !(a > 0.0) || (n > 0 && (!R_dev || !Rb_dev || !gas_dev || !gas_tab_dev || !exact_dev)))
        return PAB_EINVAL;
    if (n == 0)
        return PAB_OK;
    pab_config c;
    pab_config_default(&c);
    c.n_bins = 1;
    c.gamma = a / 3.0;
    c.sigma = 0.0;
    c.pv = 0.0;
    c.p0 = 1.0;
    const double R0 = 1.0, w = 1.0;
    pab::StepConst K;
    pab::make_const(&c, &R0, &w, &K);  // pg0 = p0 + 0 - 0 = 1
    std::vector<double> tab;
    int J = 0;
    double il2q = 0.0;
    pab::gas_table(a, K.gas_dmax_tab, &tab, &J, &il2q);
    K.gas_J = J;
    K.gas_inv_log2q = (float)il2q;
    cudaStream_t s = (cudaStream_t)stream;
    double *tab_dev = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&tab_dev, tab.size() * sizeof(double), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tab_dev, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        math_check_kernel<<<152 * 4, 256, 0, s>>>(K, tab_dev, n, R_dev, Rb_dev, gas_dev, gas_tab_dev,
                                                   exact_dev);
        e = cudaGetLastError();
    }
    if (tab_dev)
        cudaFreeAsync(tab_dev, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? PAB_OK : PAB_ECUDA;
}

extern "C" pab_status pab_peak_fma(int32_t precision, int32_t blocks, int32_t threads, int32_t iters,
                                   double *sink_dev, float *ms_out, double *fma_out, void *stream)
{
    if (blocks < 1 || threads < 32 || threads > 1024 || iters < 1 || !sink_dev || !ms_out || !fma_out)
        return PAB_EINVAL;
    if (precision != PAB_FP64 && precision != PAB_MIXED)
        return PAB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return PAB_ECUDA;
    cudaEventRecord(e0, s);
    if (precision == PAB_FP64)
        fma_streams<double><<<blocks, threads, 0, s>>>(iters, sink_dev);
    else
        fma_streams<float><<<blocks, threads, 0, s>>>(iters, sink_dev);
    cudaError_t e = cudaGetLastError();
    cudaEventRecord(e1, s);
    if (e == cudaSuccess)
        e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess)
        return PAB_ECUDA;
    *ms_out = ms;
    *fma_out = (double)blocks * threads * (double)iters * 32.0;
    return PAB_OK;
}
