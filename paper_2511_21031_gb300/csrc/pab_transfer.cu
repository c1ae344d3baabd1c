// The bubble source update with heat and mass transfer in the contents
// (gas_mode PAB_GAS_TRANSFER, FP64): four states per (bin, cell), R, Rdot, the
// bubble pressure p_b and the vapour mass m_v.  The work decomposition is the
// one of step_kernel (pab_stream.cuh: a CTA of w warps owns w tiles of 32 cells
// and streams their (bin, cell) items lane by lane from one pool; the moments
// come from a closing pass that sums each cell's bins in bin order); the model
// is stated in pab_transfer.h.
#include <cuda_runtime.h>

#include "pab_check.cuh"
#include "pab_device.cuh"
#include "pab_internal.h"
#include "pab_reduce.cuh"
#include "pab_stream.cuh"

PAB_CHECK_UNIT(transfer)

namespace pab {
namespace {

constexpr double kPi = 3.14159265358979323846;

struct State4 {
    double R, V, pb, mv;
};

struct Trial4 {
    State4 y;        // third-order result
    double eR, eV;   // 3 (y3 - z) of R and Rdot (three times the embedded difference)
    bool ok;         // stage radii positive and Rdot finite
};

// m_g R_g of a bin: the gas of equilibrium at R0, (p0 + 2 sigma/R0 - pv) V0 / T_w.
__device__ __forceinline__ double gas_mRg(const StepConst &K, const BinConst &bc)
{
    const double V0 = (4.0 / 3.0 * kPi) * bc.R0 * bc.R0 * bc.R0;
    return (K.p0 + K.two_sigma * bc.invR0 - K.pv) * V0 * (K.tr_Rg * K.tr_inv_RgTw);  // ... / T_w
}

// INT: the products and reciprocals formed from the significands on the integer pipe
// (pab_intmul.cuh, each within 1 ulp of the FP64 operation), GB300's FP64 pipe being the bound of
// the step; ok is cleared where one of them meets a subnormal, infinite or NaN value or leaves the
// normal range, and the trial is then formed again in FP64.
template <bool INT>
__device__ __forceinline__ double mul_t(double x, double y, bool &ok)
{
    return INT ? mul2_int(x, y, ok) : x * y;
}

template <bool INT>
__device__ __forceinline__ double rcp_t(double x, bool &ok)
{
    return INT ? rcp_int(x, ok) : rcp64(x);
}

// dp_b/dt and dm_v/dt (Ando's pressure equation and Eq. massVaporRate with
// constant-coefficient wall gradients), iR = 1/R.  With chi_vw = rho_vw/rho_bw
// and 1 - chi_vw = rho_gw/rho_bw the vapour flux is
//   mdot = D beta_c rho_bw (rho_vw - chi_mean rho_bw) / (rho_gw R) = X / R,
// so the wall fraction needs no reciprocal; with the mean mass fraction
// chi_mean = m_v R_g / D2, D2 = m_v R_g + m_g R_g, the two remaining divisions
// share one reciprocal: X = D beta_c rho_bw (rho_vw D2 - m_v R_g rho_bw) / (D2 rho_gw).
// The heat term (gamma - 1)/gamma k_bw beta_T (T_w - T_mean)/R shares the factor 1/R:
//   dp_b/dt = 3 gamma/R ((R_v T_w X + kT (T_w - T_mean))/R - Rdot p_b),
//   dm_v/dt = 4 pi R^2 mdot = 4 pi R X,
// with the constants folded in: X4 = 4 pi X, and kT T_mean = (4 pi/3) kT p_b R^3/(m_v R_v + m_g R_g).
template <bool INT>
__device__ __forceinline__ void transfer_rates(const StepConst &K, double mRg, const State4 &s,
                                               double iR, double &dpb, double &dmv, bool &ok)
{
    // T_mean 3/(4 pi)
    const double T3 = mul_t<INT>(
        mul_t<INT>(mul_t<INT>(mul_t<INT>(s.pb, s.R, ok), s.R, ok), s.R, ok),
        rcp_t<INT>(fma(s.mv, K.tr_Rv, mRg), ok), ok);
    const double mvRg = mul_t<INT>(s.mv, K.tr_Rg, ok);
    const double D2 = mvRg + mRg;                                    // (m_v + m_g) R_g
    const double rho_gw = mul_t<INT>(s.pb - K.pv, K.tr_inv_RgTw, ok);  // gas density at the wall
    const double rho_bw = K.tr_rho_vw + rho_gw;
    const double X4 = mul_t<INT>(
        mul_t<INT>(mul_t<INT>(K.tr_Dc_4pi, rho_bw, ok),
                   fma(K.tr_rho_vw, D2, -mul_t<INT>(mvRg, rho_bw, ok)), ok),
        rcp_t<INT>(mul_t<INT>(D2, rho_gw, ok), ok), ok);
    const double q = fma(K.tr_RvTw_4pi, X4, fma(-K.tr_kT_43pi, T3, K.tr_kT_Tw));
    dpb = mul_t<INT>(mul_t<INT>(K.three_gamma, iR, ok), fma(q, iR, -mul_t<INT>(s.V, s.pb, ok)), ok);
    dmv = mul_t<INT>(s.R, X4, ok);
}

// Keller-Miksis, Eq. (keller_miksis), with the state p_b, regrouped as in
// accel64: the s/R terms (s = 4 mu Rdot + 2 sigma) of (p_bw - p_inf)(1 + Rdot/c)/rho
// and of (R/(rho c)) d/dt p_bw add up to -s/(rho R), which leaves
//   Rddot = (N0 R - s/rho) / (R den),
//   N0 = P (1 + Rdot/c) + R dp_b/dt /(rho c) - Rdot^2 (3/2 - Rdot/(2c)),  P = (p_b - p_inf)/rho,
// taken as N0 = P + R dp_b/dt /(rho c) + Rdot (P/c - Rdot (3/2 - Rdot/(2c))).
template <bool INT>
__device__ __forceinline__ State4 rhs4(const StepConst &K, double mRg, double pinf_rho, const State4 &s,
                                       bool &ok)
{
    const double den = fma(s.R, fma(s.V, -K.inv_c, 1.0), K.fmu_ic_rho);
    const double inv = rcp_t<INT>(mul_t<INT>(s.R, den, ok), ok);
    const double iR = mul_t<INT>(den, inv, ok);
    double dpb, dmv;
    transfer_rates<INT>(K, mRg, s, iR, dpb, dmv, ok);
    const double P = fma(s.pb, K.inv_rho, -pinf_rho);
    const double t = fma(-s.V, fma(s.V, K.m05_inv_c, 1.5), mul_t<INT>(P, K.inv_c, ok));
    const double N0 = fma(s.V, t, fma(mul_t<INT>(s.R, K.ic_rho, ok), dpb, P));
    const double s_rho = fma(K.fmu_rho, s.V, K.tsig_rho);
    return State4{s.V, mul_t<INT>(fma(N0, s.R, -s_rho), inv, ok), dpb, dmv};
}

template <bool INT>
__device__ __forceinline__ State4 scale(double h, const State4 &f, bool &ok)
{
    return State4{mul_t<INT>(h, f.R, ok), mul_t<INT>(h, f.V, ok), mul_t<INT>(h, f.pb, ok),
                  mul_t<INT>(h, f.mv, ok)};
}

// Shu-Osher SSP-RK3 with the embedded Heun member in increment form (as trial64),
// on four components: k1 = h f(y), y1 = y + k1, s = k1 + k2, y2 = y + s/4,
// e = 2 k3 - s = (2h) f(y2) - s = 3 (y3 - z) with 2h exact, y3 = y + s/2 + e/3.
template <bool INT>
__device__ __forceinline__ Trial4 trial4_body(const StepConst &K, double mRg, double pinf_rho,
                                              const State4 &y, double h, bool &ok)
{
    const State4 k1 = scale<INT>(h, rhs4<INT>(K, mRg, pinf_rho, y, ok), ok);
    const State4 y1{y.R + k1.R, y.V + k1.V, y.pb + k1.pb, y.mv + k1.mv};
    const State4 f2 = rhs4<INT>(K, mRg, pinf_rho, y1, ok);
    const State4 s{fma(h, f2.R, k1.R), fma(h, f2.V, k1.V), fma(h, f2.pb, k1.pb), fma(h, f2.mv, k1.mv)};
    const State4 y2{fma(0.25, s.R, y.R), fma(0.25, s.V, y.V), fma(0.25, s.pb, y.pb), fma(0.25, s.mv, y.mv)};
    const State4 f3 = rhs4<INT>(K, mRg, pinf_rho, y2, ok);
    const double h2 = twice_nn(h);
    const State4 e{fma(h2, f3.R, -s.R), fma(h2, f3.V, -s.V), fma(h2, f3.pb, -s.pb), fma(h2, f3.mv, -s.mv)};
    Trial4 t;
    t.y = State4{fma(1.0 / 3.0, e.R, fma(0.5, s.R, y.R)), fma(1.0 / 3.0, e.V, fma(0.5, s.V, y.V)),
                 fma(1.0 / 3.0, e.pb, fma(0.5, s.pb, y.pb)), fma(1.0 / 3.0, e.mv, fma(0.5, s.mv, y.mv))};
    t.eR = e.R;
    t.eV = e.V;
    t.ok = gt0(y1.R) && gt0(y2.R) && gt0(t.y.R) && finite64(t.y.V);
    return t;
}

// The trial with its products and reciprocals on the integer pipe, and again in FP64 where one
// of them met a subnormal, infinite or NaN value or left the normal range.
__device__ __forceinline__ Trial4 trial4(const StepConst &K, double mRg, double pinf_rho, const State4 &y,
                                         double h)
{
    bool ok = true;
    Trial4 t = trial4_body<true>(K, mRg, pinf_rho, y, h, ok);
    if (!ok)
        t = trial4_body<false>(K, mRg, pinf_rho, y, h, ok);
    return t;
}

// The controller of advance_adaptive (or n equal sub-steps in fixed mode);
// the error norm reads R and Rdot.
__device__ __forceinline__ uint32_t advance4(const StepConst &K, double mRg, double p_inf, double dt,
                                             double dt_sub, State4 &y, float &hc, int &n_att)
{
    const double pinf_rho = p_inf * K.inv_rho;
    if (K.n_fixed > 0) {
        for (int i = 0; i < K.n_fixed; ++i)
            y = trial4(K, mRg, pinf_rho, y, dt_sub).y;
        n_att = K.n_fixed;
        return 0;
    }
    double h = start_h(hc, dt);
    double rem = dt;  // time left of the flow step, counted down
    uint32_t flags = 0;
    int n = 0;
    for (;;) {
        if (n >= K.max_attempts) {
            flags |= PAB_FLAG_STEP_LIMIT;
            break;
        }
        const bool last = le(rem, h);
        const double ht = last ? rem : h;
        const Trial4 tr = trial4(K, mRg, pinf_rho, y, ht);
        ++n;
        const Decision vd = decide64(K, Trial{tr.y.R, tr.y.V, tr.eR, tr.eV, tr.ok});
        const double fac = f2d_fin(vd.fac);
        if (vd.accept) {
            y = tr.y;
            if (last) {
                const bool clipped = !le(h, rem);
                h = (clipped && vd.fac >= 1.0f) ? h : ht * fac;
                break;
            }
            rem -= ht;
            h = ht * fac;
        } else {
            h = ht * fac;
        }
    }
    hc = d2f(h);
    n_att = n;
    return flags;
}

// One lane's item: the four states of one (bin, cell), with the controller of advance4.
struct ItemT {
    long long c;
    size_t k;
    double mRg, pinf_rho;
    State4 y;
    double h, rem;
    int n;
    uint32_t fl;

    // The start of the flow step from the stored state; false for a non-finite input (flagged,
    // counted, left as it is).
    // (mRg_b: the bin's gas constant; pinf_c: the cell's p_inf / rho, both formed once per CTA)
    __device__ __forceinline__ bool start(const StepConst &K, const StepArgs &a, int b, long long c_,
                                          double mRg_b, double pinf_c, TileCounts &tc)
    {
        c = c_;
        k = (size_t)b * (size_t)K.C + (size_t)c;
        const long long ns = (long long)K.B * K.C;
        const double p_inf = PAB_LD(a.p_inf, c, K.C);
        y = State4{PAB_LD(a.R, k, ns), PAB_LD(a.V, k, ns), PAB_LD(a.pb, k, ns), PAB_LD(a.mv, k, ns)};
        n = 0;
        fl = 0;
        if (!finite64(p_inf) || !finite64(y.R) || !finite64(y.V) || !finite64(y.pb) || !finite64(y.mv)) {
            if (a.attempts)
                PAB_ST(a.attempts, k, ns, 0);
            tc.fl_or |= PAB_FLAG_NONFINITE;
            tc.n_flag += 1;
            return false;
        }
        mRg = mRg_b;
        pinf_rho = pinf_c;
        h = start_h(PAB_LD(a.h, k, ns), a.dt);
        rem = a.dt;
        return true;
    }

    // One trial and the controller; true when the flow step is done.
    __device__ __forceinline__ bool trial(const StepConst &K)
    {
        if (n >= K.max_attempts) {
            fl |= PAB_FLAG_STEP_LIMIT;
            return true;
        }
        bool done = false;
        const bool last = le(rem, h);
        const double ht = last ? rem : h;
        const Trial4 tr = trial4(K, mRg, pinf_rho, y, ht);
        ++n;
        const Decision vd = decide64(K, Trial{tr.y.R, tr.y.V, tr.eR, tr.eV, tr.ok});
        const double fac = f2d_fin(vd.fac);
        if (vd.accept) {
            y = tr.y;
            if (last) {
                const bool clipped = !le(h, rem);
                h = (clipped && vd.fac >= 1.0f) ? h : ht * fac;
                done = true;
            } else {
                rem -= ht;
                h = ht * fac;
            }
        } else {
            h = ht * fac;
        }
        if (!done && n >= K.max_attempts) {
            fl |= PAB_FLAG_STEP_LIMIT;
            done = true;
        }
        return done;
    }

    __device__ __forceinline__ void finish(const StepConst &K, const StepArgs &a, TileCounts &tc)
    {
        if (!finite64(y.R) || !finite64(y.V) || !finite64(y.pb) || !finite64(y.mv))
            fl |= PAB_FLAG_NONFINITE;
        else if (!gt0(y.R))
            fl |= PAB_FLAG_NONPOS;
        if (abs_ge(y.V, K.c))
            fl |= PAB_FLAG_SUPERSONIC;
        const long long ns = (long long)K.B * K.C;
        PAB_ST(a.R, k, ns, y.R);
        PAB_ST(a.V, k, ns, y.V);
        PAB_ST(a.pb, k, ns, y.pb);
        PAB_ST(a.mv, k, ns, y.mv);
        PAB_ST(a.h, k, ns, d2f(h));
        if (a.attempts)
            PAB_ST(a.attempts, k, ns, n);
        tc.fl_or |= fl;
        tc.n_flag += (fl != 0);
        tc.n_att += n;
    }
};

// Fixed mode: n equal trials per item; one thread per cell walks the bins.
__device__ __forceinline__ void transfer_fixed(const StepConst &K, const StepArgs &a, long long c0, int nc,
                                               TileCounts &tc)
{
    if ((int)threadIdx.x >= nc)
        return;
    const long long c = c0 + threadIdx.x;
    const long long ns = (long long)K.B * K.C;
    const double p_inf = PAB_LD(a.p_inf, c, K.C);
    for (int b = 0; b < K.B; ++b) {
        const size_t k = (size_t)b * (size_t)K.C + (size_t)c;
        State4 y{PAB_LD(a.R, k, ns), PAB_LD(a.V, k, ns), PAB_LD(a.pb, k, ns), PAB_LD(a.mv, k, ns)};
        uint32_t fl = 0;
        int na = 0;
        if (!finite64(p_inf) || !finite64(y.R) || !finite64(y.V) || !finite64(y.pb) || !finite64(y.mv)) {
            fl = PAB_FLAG_NONFINITE;
        } else {
            float hc = 0.0f;
            fl = advance4(K, gas_mRg(K, K.bins[b]), p_inf, a.dt, a.dt_sub, y, hc, na);
            if (!finite64(y.R) || !finite64(y.V) || !finite64(y.pb) || !finite64(y.mv))
                fl |= PAB_FLAG_NONFINITE;
            else if (!gt0(y.R))
                fl |= PAB_FLAG_NONPOS;
            if (abs_ge(y.V, K.c))
                fl |= PAB_FLAG_SUPERSONIC;
            PAB_ST(a.R, k, ns, y.R);
            PAB_ST(a.V, k, ns, y.V);
            PAB_ST(a.pb, k, ns, y.pb);
            PAB_ST(a.mv, k, ns, y.mv);
        }
        if (a.attempts)
            PAB_ST(a.attempts, k, ns, na);
        tc.fl_or |= fl;
        tc.n_flag += (fl != 0);
        tc.n_att += na;
    }
}

// The moments of cell c from the four-state contents, its bins summed in bin order (FP64), with
// p_bw = p_b - (4 mu Rdot + 2 sigma)/R and the pressure sum over rho.
__device__ __forceinline__ void transfer_cell_moments(const StepConst &K, const double *R, const double *V,
                                                      const double *pb, long long c, double nb, double *out)
{
    const long long ns = (long long)K.B * K.C;
    TermSums S;
    for (int b = 0; b < K.B; ++b) {
        const size_t k = (size_t)b * (size_t)K.C + (size_t)c;
        const double r = PAB_LDCG(R, k, ns), v = PAB_LDCG(V, k, ns), p = PAB_LDCG(pb, k, ns);
        const double w = K.bins[b].w;
        const double wr2 = __dmul_rn(__dmul_rn(w, r), r);
        const double wr3 = __dmul_rn(wr2, r);
        const double t[3] = {__dmul_rn(wr2, v),
                             fma(wr3, p * K.inv_rho, -__dmul_rn(wr2, fma(K.fmu_rho, v, K.tsig_rho))),
                             __dmul_rn(__dmul_rn(wr3, v), v)};
        add_terms<false>(S, wr3, nullptr, t);
    }
    write_moments<false>(K, nb, K.C, c, S, out);
}

// One CTA of nw warps owns nw tiles (32 nw cells) and streams their items lane by lane.
// 96 registers (up to 16 warps a CTA fit): with the trial's arithmetic on the integer pipe the
// kernel takes 128 uncapped, and 96 (a few bytes spilled, 5 CTAs of 4 warps per SM) ran 3.5 %
// faster than 128 and 104, 7 % faster than 112.
__global__ void __maxnreg__(96)
    transfer_step_kernel(const __grid_constant__ StepConst K, const StepArgs a)
{
    __shared__ PoolCounters sh;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const long long c0 = (long long)blockIdx.x * kTile * nw;
    const int nc = (int)min((long long)kTile * nw, K.C - c0);
    TileCounts tc;
    if (K.n_fixed > 0) {
        transfer_fixed(K, a, c0, nc, tc);
    } else {
        // the bins' gas constants and the cells' p_inf / rho, once per CTA rather than per item
        __shared__ double s_mRg[PAB_MAX_BINS];
        __shared__ double s_pinf[kMaxWarps * kTile];
        for (int b = threadIdx.x; b < K.B; b += blockDim.x)
            s_mRg[b] = gas_mRg(K, K.bins[b]);
        for (int cl = threadIdx.x; cl < nc; cl += blockDim.x)
            s_pinf[cl] = PAB_LD(a.p_inf, c0 + cl, K.C) * K.inv_rho;
        if (threadIdx.x == 0)
            sh = PoolCounters{0, 0, 0};
        __syncthreads();
        TileIO io;  // the pool's layout (item j: bin j / nc, cell c0 + j mod nc)
        io.C = K.C;
        io.c0 = c0;
        io.nc = nc;
        io.b0 = 0;
        io.b1 = K.B;
        const int total = K.B * nc;
        bool exhausted = total <= 0;
        bool have = false;
        ItemT it;
        for (;;) {
            const unsigned want = __ballot_sync(0xffffffffu, !have);
            if (want && !exhausted) {
                const int j = grab(want, total, &sh.next, exhausted);
                if (j >= 0 && j < total) {
                    int b, cl;
                    size_t k;
                    item_of(io, j, b, cl, k);
                    have = it.start(K, a, b, c0 + cl, s_mRg[b], s_pinf[cl], tc);
                }
            }
            if (!__any_sync(0xffffffffu, have)) {
                if (exhausted)
                    break;
                continue;
            }
            if (have && it.trial(K)) {
                it.finish(K, a, tc);
                have = false;
            }
        }
    }
    // block-wide counters; the barrier inside orders the state writes before the reads below
    flush_counters(tc.fl_or, tc.n_flag, tc.n_att, 0u, a.counters);
    const long long c = c0 + (long long)kTile * warp + lane;
    if (a.out && c < c0 + nc)
        transfer_cell_moments(K, a.R, a.V, a.pb, c, a.nb ? PAB_LD(a.nb, c, K.C) : K.nb_default, a.out);
}

// Reduce-only: one lane per cell, the closing pass of the step kernel.
__global__ void __launch_bounds__(128)
    transfer_moments_kernel(const __grid_constant__ StepConst K, const double *__restrict__ nbp,
                            const double *Rp, const double *Vp, const double *pbp, double *out)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < K.C)
        transfer_cell_moments(K, Rp, Vp, pbp, c, nbp ? PAB_LD(nbp, c, K.C) : K.nb_default, out);
}

// Equilibrium contents: p_b = p0 + 2 sigma/R0, m_v = (pv/(R_v T_w)) V0.
__global__ void transfer_init_kernel(const __grid_constant__ StepConst K, double *pb, double *mv)
{
    const size_t n = (size_t)K.B * (size_t)K.C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const BinConst &bc = K.bins[(int)(i / (size_t)K.C)];
        PAB_ST(pb, i, n, K.p0 + K.two_sigma * bc.invR0);
        PAB_ST(mv, i, n, K.tr_rho_vw * ((4.0 / 3.0 * kPi) * bc.R0 * bc.R0 * bc.R0));
    }
}

}  // namespace

cudaError_t launch_transfer_step(const StepConst &K, const StepArgs &a, int block_warps, cudaStream_t s)
{
    if (!a.pb || !a.mv || !a.h)
        return cudaErrorInvalidValue;
    const int nw = block_warps <= 0 ? kDefaultWarps : (block_warps > kMaxWarps ? kMaxWarps : block_warps);
    const long long cells = (long long)kTile * nw;
    const dim3 grid((unsigned)((K.C + cells - 1) / cells));
    transfer_step_kernel<<<grid, nw * 32, 0, s>>>(K, a);
    return cudaGetLastError();
}

cudaError_t launch_transfer_moments(const StepConst &K, const double *nb, const double *R,
                                    const double *V, const double *pb, double *out, int block_warps,
                                    cudaStream_t s)
{
    (void)block_warps;
    const dim3 grid((unsigned)((K.C + 127) / 128));
    transfer_moments_kernel<<<grid, 128, 0, s>>>(K, nb, R, V, pb, out);
    return cudaGetLastError();
}

cudaError_t launch_transfer_init(const StepConst &K, double *pb, double *mv, cudaStream_t s)
{
    transfer_init_kernel<<<152 * 8, 256, 0, s>>>(K, pb, mv);
    return cudaGetLastError();
}

}  // namespace pab
