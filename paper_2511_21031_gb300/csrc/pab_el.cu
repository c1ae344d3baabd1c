// Volume-averaged (Euler-Lagrange) subgrid model: Lagrangian bubbles advanced
// by the Keller-Miksis stepper of the EE path, and their volumes smeared onto
// the grid with the truncated Gaussian kernel of Eq. (kernel3D)
// (include/pab_el.h).
//
//   el_advance_kernel  one thread per bubble; the bubble's constants (R0,
//                      p_g0, ...) come from a per-bubble table in global memory,
//                      its pressure from the cell that contains it.
//   el_smear_kernel    one warp per bubble.  The kernel exp(-d^2/(2h^2)) is
//                      separable: the warp evaluates the 3 x (2m+1) one-
//                      dimensional factors once (for stencil half-widths m up to
//                      24 cells; wider kernels evaluate every point), then its
//                      lanes walk the (2m+1)^3 stencil cube in FP32, queue the
//                      cells with d/h < 3 (about a sixth of the cube) and add
//                      V delta and Vdot delta for 32 of them at a time with FP64
//                      atomics (nearby bubbles overlap, Listing 1's "atomic
//                      update").
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pab.h"
#include "pab_device.cuh"
#include "pab_exp.cuh"
#include "pab_el.h"
#include "pab_check.cuh"
#include "pab_internal.h"

PAB_CHECK_UNIT(el)

namespace pab {
namespace {

// A stencil point's weight fx fy fz and its rate term with FP64 products: out of line, for the
// points whose products the integer form (pab_intmul.cuh) does not take; returned by value.
struct Weight2 {
    double a, ad;
};
static __device__ __noinline__ Weight2 smear_weight_fp64(double f0, double f1, double f2, double rate)
{
    const double a = f0 * f1 * f2;
    return Weight2{a, a * rate};
}

constexpr int kSmearWarps = 4;
constexpr int kCacheHalf = 24;  // stencil half-widths up to this use the separable cache
constexpr int kSide = 2 * kCacheHalf + 1;

__global__ void __launch_bounds__(256)
    el_advance_kernel(const __grid_constant__ StepConst K, long long N, const BinConst *__restrict__ bub,
                      const long long *__restrict__ cell, const double *__restrict__ p_cell, double dt,
                      double *__restrict__ R, double *__restrict__ V, float *__restrict__ h,
                      Counters *cnt, long long n_grid)
{
    __shared__ uint32_t sc[3][8];
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t fl = 0;
    int na = 0;
    if (n < N) {
        const BinConst bc = PAB_LD(bub, n, N);
        const long long ci = PAB_LD(cell, n, N);
        const double p_inf = ci >= 0 ? PAB_LD(p_cell, ci, n_grid) : CUDART_NAN;
        double r = PAB_LD(R, n, N), v = PAB_LD(V, n, N);
        float hc = PAB_LD(h, n, N);
        int nd = 0;
        GasBase g;
        g.reset();
        fl = advance_bin<false>(K, bc, p_inf, cell_terms<false>(K, p_inf), isfinite(p_inf), dt, 0.0, r, v,
                                hc, na, nd, g);  // adaptive
        PAB_ST(R, n, N, r);  // unchanged when the input was not finite
        PAB_ST(V, n, N, v);
        PAB_ST(h, n, N, hc);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t f = __reduce_or_sync(0xffffffffu, fl);
    const uint32_t nf = __reduce_add_sync(0xffffffffu, fl != 0 ? 1u : 0u);
    const uint32_t a = __reduce_add_sync(0xffffffffu, (uint32_t)na);
    if (lane == 0) {
        sc[0][warp] = f;
        sc[1][warp] = nf;
        sc[2][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t F = 0;
        unsigned long long NF = 0, A = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            F |= sc[0][w];
            NF += sc[1][w];
            A += sc[2][w];
        }
        if (F)
            atomicOr(&cnt->flags_or, F);
        if (NF)
            atomicAdd(&cnt->n_flagged, NF);
        if (A)
            atomicAdd(&cnt->n_attempts, A);
    }
}

// Whether stencil point (oi, oj, ok) of the cached factors lies inside the
// truncated kernel: FP32 sum of the squared offsets against 9 h^2, and within
// 1e-5 of the cut the FP64 decision d/h < 3.
__device__ __forceinline__ bool smear_inside(const double (*sq)[kSide], const float (*sqf)[kSide], int oi,
                                             int oj, int ok, float lim2f, double h)
{
    const float d2f = sqf[0][oi] + sqf[1][oj] + sqf[2][ok];
    bool inside = d2f < lim2f;
    if (fabsf(d2f - lim2f) <= 1e-5f * lim2f) {
        const double d2 = sq[0][oi] + sq[1][oj] + sq[2][ok];
        inside = sqrt(d2) / h < 3.0;
    }
    return inside;
}

__global__ void __launch_bounds__(kSmearWarps * 32)
    el_smear_kernel(long long N, const double *__restrict__ px, const double *__restrict__ py,
                    const double *__restrict__ pz, const double *__restrict__ R,
                    const double *__restrict__ V, int nx, int ny, int nz, double dx, double inv_dx,
                    double *__restrict__ alpha, double *__restrict__ alpha_dot)
{
    // per warp and axis offset: the squared distance (FP64 and FP32) and the 1-D
    // Gaussian factor; the x factor carries V/(h^3 (2 pi)^{3/2}) so that a stencil
    // point costs two multiplies (three with the rate), formed on the integer pipe
    __shared__ double fac[kSmearWarps][3][kSide];
    __shared__ double sq[kSmearWarps][3][kSide];
    __shared__ float sqf[kSmearWarps][3][kSide];
    // inside points waiting for a full warp (ring of 64 stencil indices per warp)
    __shared__ int ring[kSmearWarps][64];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const double norm = 15.749609945722419;  // (2 pi)^{3/2}
    for (long long n = (long long)blockIdx.x * kSmearWarps + warp; n < N;
         n += (long long)gridDim.x * kSmearWarps) {
        const long long ng = (long long)nx * ny * nz;
        const double r = PAB_LD(R, n, N);
        const double h = r < dx ? dx : r;
        // cells whose centre can lie within 3h: m > 3h/dx (the 1e-9 keeps the product's
        // rounding from taking m one too small); m >= 4 for every number r (h >= dx)
        const int m = (int)floor(fma(3.0 * h, inv_dx, 1e-9)) + 1;
        if (m < 4)
            continue;  // r is NaN: the bubble adds nothing
        const int side = 2 * m + 1;
        const bool cached = m <= kCacheHalf;
        const double x0 = PAB_LD(px, n, N), y0 = PAB_LD(py, n, N), z0 = PAB_LD(pz, n, N);
        // the base cell may be off by one where x0/dx rounds across an integer: the window
        // [f - m, f + m] still holds every centre within 3h of x0 then
        const int bx = (int)floor(x0 * inv_dx) - m, by = (int)floor(y0 * inv_dx) - m,
                  bz = (int)floor(z0 * inv_dx) - m;
        const double ir = rcp64(r);
        const double ih = r < dx ? inv_dx : ir;  // 1/h
        const double inv2h2 = 0.5 * ih * ih;
        const double rh = r * ih;
        // V/(h^3 (2 pi)^{3/2}) = (4 pi/3) (r/h)^3 / (2 pi)^{3/2}, and alpha_dot/alpha = 3 Rdot/r
        const double amp = (4.0 / 3.0 * 3.14159265358979323846 / norm) * (rh * rh * rh);
        const double rate = 3.0 * PAB_LD(V, n, N) * ir;
        const double lim2 = 9.0 * h * h;
        // stencil point t = oi + side (oj + side ok); each lane walks t = lane, lane + 32,
        // ... with its offsets carried forward (32 = q32 side + r32, side >= 9 since
        // h >= dx), so the loops divide nothing
        const int q32 = 32 / side, r32 = 32 - q32 * side;
        int oi = lane % side, oj = lane / side, ok = 0;
        const auto next32 = [&]() {
            oi += r32;
            oj += q32;
            if (oi >= side) {
                oi -= side;
                ++oj;
            }
            if (oj >= side) {
                oj -= side;
                ++ok;
            }
        };
        if (cached) {
            for (int t = lane; t < 3 * side; t += 32) {
                const int a = t / side, o = t % side;
                const double pa = a == 0 ? x0 : (a == 1 ? y0 : z0);
                const int ba = a == 0 ? bx : (a == 1 ? by : bz);
                const double cc = ((double)(ba + o) + 0.5) * dx - pa;
                const double c2 = cc * cc;
                sq[warp][a][o] = c2;
                sqf[warp][a][o] = (float)c2;
                const double f = exp_tab(-c2 * inv2h2);
                fac[warp][a][o] = a == 0 ? f * amp : f;
            }
            __syncwarp();
            const float lim2f = (float)lim2;
            // the lanes test 32 stencil points at a time; the inside ones (about 16 % of the
            // cube) queue up, and every 32 of them are added by the whole warp at once
            // (queued points are kept as oi | oj << 8 | ok << 16, side <= 49 here)
            int queued = 0, tail = 0;
            for (int base = 0; base < side * side * side; base += 32) {
                bool in = false;
                if (ok < side) {
                    const int i = bx + oi, j = by + oj, k = bz + ok;
                    in = i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz &&
                         smear_inside(sq[warp], sqf[warp], oi, oj, ok, lim2f, h);
                }
                const unsigned mask = __ballot_sync(0xffffffffu, in);
                if (in)
                    ring[warp][(tail + queued + __popc(mask & lt_mask)) & 63] = oi | (oj << 8) | (ok << 16);
                queued += __popc(mask);
                next32();
                __syncwarp();
                const bool flush_all = base + 32 >= side * side * side;
                while (queued >= 32 || (flush_all && queued > 0)) {
                    if (lane < queued) {
                        const int tq = ring[warp][(tail + lane) & 63];
                        const int qi = tq & 255, qj = (tq >> 8) & 255, qk = tq >> 16;
                        // the weight and its rate term from the significands on the integer
                        // pipe (each product within 1 ulp of FP64), GB300's FP64 pipe being the
                        // bound of the smear
                        const double f0 = fac[warp][0][qi], f1 = fac[warp][1][qj], f2 = fac[warp][2][qk];
                        bool okw = true;
                        double a = mul2_int(mul2_int(f0, f1, okw), f2, okw);
                        double ad = mul2_int(a, rate, okw);
                        if (!okw) {
                            const Weight2 w = smear_weight_fp64(f0, f1, f2, rate);
                            a = w.a;
                            ad = w.ad;
                        }
                        const long long c = ((long long)(bz + qk) * ny + (by + qj)) * nx + (bx + qi);
                        atomicAdd(PAB_AT(alpha, c, ng), a);
                        if (alpha_dot)
                            atomicAdd(PAB_AT(alpha_dot, c, ng), ad);
                    }
                    const int done = queued < 32 ? queued : 32;
                    tail = (tail + done) & 63;
                    queued -= done;
                    __syncwarp();
                }
            }
        } else {
            for (; ok < side; next32()) {
                const int i = bx + oi, j = by + oj, k = bz + ok;
                if (i < 0 || i >= nx || j < 0 || j >= ny || k < 0 || k >= nz)
                    continue;
                const double cx = ((double)i + 0.5) * dx - x0;
                const double cy = ((double)j + 0.5) * dx - y0;
                const double cz = ((double)k + 0.5) * dx - z0;
                const double d2 = cx * cx + cy * cy + cz * cz;
                if (!(sqrt(d2) / h < 3.0))
                    continue;
                const double a = amp * exp_tab(-d2 * inv2h2);
                const long long c = ((long long)k * ny + j) * nx + i;
                atomicAdd(PAB_AT(alpha, c, ng), a);
                if (alpha_dot)
                    atomicAdd(PAB_AT(alpha_dot, c, ng), a * rate);
            }
        }
        __syncwarp();
    }
}

}  // namespace
}  // namespace pab

struct pab_el_s {
    pab_config cfg;
    pab::StepConst K;
    long long N = 0;
    int nx = 0, ny = 0, nz = 0;
    double dx = 0.0;
    cudaStream_t create_stream = nullptr;
    double *pos = nullptr;  // [3][N]
    long long *cell = nullptr;
    pab::BinConst *bub = nullptr;
    double *R = nullptr;
    double *V = nullptr;
    float *h = nullptr;
    pab::Counters *counters = nullptr;
    pab::Counters *counters_host = nullptr;
    double *gas_tab = nullptr;  // gas-term nodes (K.gas_tab points here), shared by every bubble
    char err[512] = {0};
};

namespace {

pab_status efail(pab_el_t *e, pab_status s, const char *fmt, ...)
{
    if (e) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(e->err, sizeof(e->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

pab_status ecuda(pab_el_t *e, cudaError_t c, const char *what)
{
    return efail(e, c == cudaErrorMemoryAllocation ? PAB_ENOMEM : PAB_ECUDA, "%s: %s", what,
                 cudaGetErrorString(c));
}

cudaError_t launch_smear(pab_el_t *e, double *alpha, double *alpha_dot, cudaStream_t s)
{
    const size_t cells = (size_t)e->nx * e->ny * e->nz;
    cudaError_t c = cudaMemsetAsync(alpha, 0, cells * sizeof(double), s);
    if (c == cudaSuccess && alpha_dot)
        c = cudaMemsetAsync(alpha_dot, 0, cells * sizeof(double), s);
    if (c != cudaSuccess || e->N == 0)
        return c;
    long long blocks = (e->N + pab::kSmearWarps - 1) / pab::kSmearWarps;
    if (blocks > 152LL * 64)
        blocks = 152LL * 64;
    pab::el_smear_kernel<<<(unsigned)blocks, pab::kSmearWarps * 32, 0, s>>>(
        e->N, e->pos, e->pos + e->N, e->pos + 2 * e->N, e->R, e->V, e->nx, e->ny, e->nz, e->dx,
        1.0 / e->dx, alpha, alpha_dot);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

const char *pab_el_last_error(const pab_el_t *e) { return e ? e->err : "NULL handle"; }

pab_status pab_el_create(const pab_config *liquid, int64_t n_bubbles, const double *pos_host,
                         const double *R0_host, int32_t nx, int32_t ny, int32_t nz, double dx,
                         void *stream, pab_el_t **out)
{
    if (!out)
        return PAB_EINVAL;
    *out = nullptr;
    if (!liquid || n_bubbles < 0 || nx < 1 || ny < 1 || nz < 1 || !(dx > 0.0) || !std::isfinite(dx) ||
        (double)nx * (double)ny * (double)nz > (double)PAB_MAX_CELLS ||
        (n_bubbles > 0 && (!pos_host || !R0_host))) {
        fprintf(stderr, "pab_el_create: invalid arguments\n");
        return PAB_EINVAL;
    }
    pab_config c = *liquid;
    c.n_cells = n_bubbles > 0 ? n_bubbles : 1;
    c.n_bins = 1;
    c.R0_host = nullptr;
    c.w_host = nullptr;
    c.stepper = PAB_ADAPTIVE;
    c.precision = PAB_FP64;
    c.block_warps = 0;
    char msg[256];
    if (pab::validate_config(&c, msg, sizeof(msg)) != PAB_OK) {
        fprintf(stderr, "pab_el_create: %s\n", msg);
        return PAB_EINVAL;
    }
    if (c.gas_mode == PAB_GAS_TRANSFER) {
        fprintf(stderr, "pab_el_create: gas_mode PAB_GAS_TRANSFER is not available here\n");
        return PAB_EINVAL;
    }
    const long long N = n_bubbles;
    std::vector<pab::BinConst> bub((size_t)N);
    std::vector<long long> cell((size_t)N);
    for (long long n = 0; n < N; ++n) {
        const double x = pos_host[n], y = pos_host[N + n], z = pos_host[2 * N + n];
        const double r0 = R0_host[n];
        if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z) || !(r0 > 0.0) ||
            !std::isfinite(r0)) {
            fprintf(stderr, "pab_el_create: bubble %lld has a bad position or radius\n", n);
            return PAB_EINVAL;
        }
        bub[(size_t)n] = pab::make_bin(&c, r0, 1.0);
        // range-checked in FP64 before the conversion, so a bubble far outside the grid
        // (or at an infinite x / dx) never meets an out-of-range integer conversion
        const double fi = std::floor(x / dx), fj = std::floor(y / dx), fk = std::floor(z / dx);
        const bool in = fi >= 0.0 && fi < (double)nx && fj >= 0.0 && fj < (double)ny && fk >= 0.0 &&
                        fk < (double)nz;
        cell[(size_t)n] = in ? ((long long)fk * ny + (long long)fj) * nx + (long long)fi : -1;
    }
    pab_el_t *e = new (std::nothrow) pab_el_t();
    if (!e)
        return PAB_ENOMEM;
    e->cfg = c;
    const double one = 1.0;
    pab::make_const(&c, &one, &one, &e->K);
    e->N = N;
    e->nx = nx;
    e->ny = ny;
    e->nz = nz;
    e->dx = dx;
    e->create_stream = (cudaStream_t)stream;
    cudaStream_t s = e->create_stream;
    const size_t n = (size_t)(N > 0 ? N : 1);
    cudaError_t err = cudaMallocAsync((void **)&e->pos, 3 * n * sizeof(double), s);
    if (err == cudaSuccess)
        err = cudaMallocAsync((void **)&e->cell, n * sizeof(long long), s);
    if (err == cudaSuccess)
        err = cudaMallocAsync((void **)&e->bub, n * sizeof(pab::BinConst), s);
    if (err == cudaSuccess)
        err = cudaMallocAsync((void **)&e->R, n * sizeof(double), s);
    if (err == cudaSuccess)
        err = cudaMallocAsync((void **)&e->V, n * sizeof(double), s);
    if (err == cudaSuccess)
        err = cudaMallocAsync((void **)&e->h, n * sizeof(float), s);
    if (err == cudaSuccess)
        err = cudaMallocAsync((void **)&e->counters, sizeof(pab::Counters), s);
    if (err == cudaSuccess)
        err = cudaMallocHost((void **)&e->counters_host, sizeof(pab::Counters));
    if (err == cudaSuccess)
        err = cudaMemsetAsync(e->counters, 0, sizeof(pab::Counters), s);
    if (err == cudaSuccess && N > 0) {
        err = cudaMemcpyAsync(e->pos, pos_host, 3 * (size_t)N * sizeof(double), cudaMemcpyHostToDevice, s);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(e->cell, cell.data(), (size_t)N * sizeof(long long),
                                  cudaMemcpyHostToDevice, s);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(e->bub, bub.data(), (size_t)N * sizeof(pab::BinConst),
                                  cudaMemcpyHostToDevice, s);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(e->R, R0_host, (size_t)N * sizeof(double), cudaMemcpyHostToDevice, s);
        if (err == cudaSuccess)
            err = cudaMemsetAsync(e->V, 0, (size_t)N * sizeof(double), s);
        if (err == cudaSuccess)
            err = cudaMemsetAsync(e->h, 0, (size_t)N * sizeof(float), s);
    }
    // the gas-term node table of the polytropic gas (a function of R/R0 alone, so one
    // table serves every bubble)
    std::vector<double> tab;
    if (err == cudaSuccess && c.gas_mode == PAB_GAS_POLYTROPIC) {
        int J = 0;
        double il2q = 0.0;
        pab::gas_table(3.0 * c.gamma, e->K.gas_dmax_tab, &tab, &J, &il2q);
        err = cudaMallocAsync((void **)&e->gas_tab, tab.size() * sizeof(double), s);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(e->gas_tab, tab.data(), tab.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, s);
        if (err == cudaSuccess) {
            e->K.gas_tab = e->gas_tab;
            e->K.gas_J = J;
            e->K.gas_inv_log2q = (float)il2q;
        }
    }
    if (err == cudaSuccess)
        err = cudaStreamSynchronize(s);  // the host tables above go out of scope
    if (err != cudaSuccess) {
        fprintf(stderr, "pab_el_create: %s\n", cudaGetErrorString(err));
        pab_status st = err == cudaErrorMemoryAllocation ? PAB_ENOMEM : PAB_ECUDA;
        cudaGetLastError();
        pab_el_destroy(e);
        return st;
    }
    *out = e;
    return PAB_OK;
}

void pab_el_destroy(pab_el_t *e)
{
    if (!e)
        return;
    cudaStream_t s = e->create_stream;
    void *bufs[] = {e->pos, e->cell, e->bub, e->R, e->V, e->h, e->counters, e->gas_tab};
    for (void *b : bufs)
        if (b)
            cudaFreeAsync(b, s);
    cudaStreamSynchronize(s);
    if (e->counters_host)
        cudaFreeHost(e->counters_host);
    delete e;
}

pab_status pab_el_step(pab_el_t *e, const double *p_cell_dev, double dt, double *alpha_dev,
                       double *alpha_dot_dev, void *stream)
{
    if (!e)
        return PAB_EINVAL;
    if (!p_cell_dev)
        return efail(e, PAB_EINVAL, "pab_el_step: p_cell_dev is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt))
        return efail(e, PAB_EINVAL, "pab_el_step: dt must be positive and finite");
    cudaStream_t s = (cudaStream_t)stream;
    if (e->N > 0) {
        const unsigned blocks = (unsigned)((e->N + 255) / 256);
        pab::el_advance_kernel<<<blocks, 256, 0, s>>>(e->K, e->N, e->bub, e->cell, p_cell_dev, dt,
                                                      e->R, e->V, e->h, e->counters,
                                                      (long long)e->nx * e->ny * e->nz);
        cudaError_t c = cudaGetLastError();
        if (c != cudaSuccess)
            return ecuda(e, c, "pab_el_step advance");
    }
    if (alpha_dev) {
        cudaError_t c = launch_smear(e, alpha_dev, alpha_dot_dev, s);
        if (c != cudaSuccess)
            return ecuda(e, c, "pab_el_step smear");
    }
    return PAB_OK;
}

pab_status pab_el_smear(pab_el_t *e, double *alpha_dev, double *alpha_dot_dev, void *stream)
{
    if (!e)
        return PAB_EINVAL;
    if (!alpha_dev)
        return efail(e, PAB_EINVAL, "pab_el_smear: alpha_dev is NULL");
    cudaError_t c = launch_smear(e, alpha_dev, alpha_dot_dev, (cudaStream_t)stream);
    return c == cudaSuccess ? PAB_OK : ecuda(e, c, "pab_el_smear");
}

pab_status pab_el_status(pab_el_t *e, uint32_t *flags, int64_t *n_flagged, int64_t *n_attempts,
                         void *stream)
{
    if (!e)
        return PAB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t c = cudaMemcpyAsync(e->counters_host, e->counters, sizeof(pab::Counters),
                                    cudaMemcpyDeviceToHost, s);
    if (c == cudaSuccess)
        c = cudaMemsetAsync(e->counters, 0, sizeof(pab::Counters), s);
    if (c == cudaSuccess)
        c = cudaStreamSynchronize(s);
    if (c != cudaSuccess)
        return ecuda(e, c, "pab_el_status");
    const pab::Counters k = *e->counters_host;
    if (flags)
        *flags = k.flags_or;
    if (n_flagged)
        *n_flagged = (int64_t)k.n_flagged;
    if (n_attempts)
        *n_attempts = (int64_t)k.n_attempts;
    if (k.flags_or & PAB_FLAG_NONFINITE)
        return efail(e, PAB_ENONFINITE, "non-finite pressure or state (bubble outside the grid?)");
    if (k.flags_or & PAB_FLAG_STEP_LIMIT)
        return efail(e, PAB_ESTEP_LIMIT, "max_attempts exhausted");
    return PAB_OK;
}

pab_status pab_el_get_state(pab_el_t *e, double *R_dev, double *Rdot_dev, float *h_dev, void *stream)
{
    if (!e)
        return PAB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)e->N;
    cudaError_t c = cudaSuccess;
    if (n && R_dev)
        c = cudaMemcpyAsync(R_dev, e->R, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (c == cudaSuccess && n && Rdot_dev)
        c = cudaMemcpyAsync(Rdot_dev, e->V, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (c == cudaSuccess && n && h_dev)
        c = cudaMemcpyAsync(h_dev, e->h, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return c == cudaSuccess ? PAB_OK : ecuda(e, c, "pab_el_get_state");
}

pab_status pab_el_set_state(pab_el_t *e, const double *R_dev, const double *Rdot_dev, const float *h_dev,
                            void *stream)
{
    if (!e)
        return PAB_EINVAL;
    if (e->N > 0 && (!R_dev || !Rdot_dev))
        return efail(e, PAB_EINVAL, "pab_el_set_state: R_dev and Rdot_dev are required");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)e->N;
    cudaError_t c = cudaSuccess;
    if (n)
        c = cudaMemcpyAsync(e->R, R_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (c == cudaSuccess && n)
        c = cudaMemcpyAsync(e->V, Rdot_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (c == cudaSuccess && n && h_dev)
        c = cudaMemcpyAsync(e->h, h_dev, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return c == cudaSuccess ? PAB_OK : ecuda(e, c, "pab_el_set_state");
}

}  // extern "C"
