// Device arithmetic of the bubble source update: Keller-Miksis acceleration
// in FP64 and in an FP32 deviation form, one SSP-RK3/RK2 trial, the error
// norm, the step-size controller and the adaptive advance of one bin.
#pragma once

#include <math_constants.h>

#include <cfloat>
#include <cstdint>

#include "pab_internal.h"

namespace pab {

// Gas pressure p_g0 (R0/R)^(3 gamma) at the last exact evaluation, the base
// from which nearby radii are reached by the binomial series.
struct GasBase {
    double Rb, invRb, Pb;
    __device__ __forceinline__ void reset()
    {
        Rb = CUDART_NAN;  // forces an exact evaluation first
        invRb = CUDART_NAN;
        Pb = 0.0;
    }
};

// (1 + d)^(-3 gamma) by its binomial series (degree 11); callers keep |d| within
// gas_dmax, where the first omitted term is below half an ulp.
__device__ __forceinline__ double gas_series(const StepConst &K, double d)
{
    double s = K.gas_c[kGasTerms - 1];
#pragma unroll
    for (int k = kGasTerms - 2; k >= 0; --k)
        s = fma(s, d, K.gas_c[k]);
    return s;
}

// p_g0 (R0/R)^(3 gamma) given R and 1/R.
//  - With a node table (a handle's gas_tab): x = R/R0 goes to the nearest node
//    x_j = q^j (picked with an FP32 log2), and (R0/R)^(3 gamma) = T_j (1 + d)^(-3 gamma)
//    with d = (x - x_j)/x_j, |d| <= sqrt(q) - 1 < gas_dmax.  A pure function of R:
//    no exp or log while R/R0 stays within the table.
//  - Otherwise (or outside the table): the radii of one step stay close to the
//    last exact evaluation R_b in g, reached by the same series in
//    d = (R - R_b)/R_b; farther away the value is exact, exp(3 gamma log(R0/R)),
//    and becomes the new base.
__device__ __forceinline__ double gas_pressure(const StepConst &K, const BinConst &bc, double R,
                                               double iR, GasBase &g)
{
    if (K.gas_tab) {
        const double x = R * bc.invR0;
        const int j = __float2int_rn(__log2f((float)x) * (float)K.gas_inv_log2q);
        if (j >= -K.gas_J && j <= K.gas_J) {
            const double *e = K.gas_tab + 3 * (j + K.gas_J);
            const double d = (x - e[0]) * e[1];
            return bc.pg0 * e[2] * gas_series(K, d);
        }
    }
    const double d = (R - g.Rb) * g.invRb;
    if (fabs(d) <= K.gas_dmax)
        return g.Pb * gas_series(K, d);
    const double P = bc.pg0 * exp(K.three_gamma * log(bc.R0 * iR));
    g.Rb = R;
    g.invRb = iR;
    g.Pb = P;
    return P;
}

// x^(-1/3) for x > 0: FP32 seed rcbrtf, then one Newton step for y^-3 = x in
// FP64, y <- y + y (1 - x y^3)/3 (relative error ~1e-14; the seed's ~1e-7 squared).
__device__ __forceinline__ double rcbrt_newton(double x)
{
    const double y = (double)rcbrtf((float)x);
    const double e = fma(-x, y * y * y, 1.0);
    return fma(y * (1.0 / 3.0), e, y);
}

struct Trial {
    double R, V;    // third-order result y3
    double eR, eV;  // |y3 - y2| per component (embedded second-order difference)
    bool ok;        // every stage radius positive and y3 finite
};

// ---------------------------------------------------------------------------
// Keller-Miksis acceleration, Eq. (keller_miksis), FP64.
//   p_b = pv + p_g0 (R0/R)^(3 gamma)       (Ando's ODE without transfer terms)
//   p_bw = p_b - (4 mu Rdot + 2 sigma)/R
//   d/dt p_bw = -3 gamma (p_b - pv) Rdot/R + (4 mu Rdot + 2 sigma) Rdot/R^2 - 4 mu Rddot/R
// The Rddot inside d/dt p_bw moves to the left-hand side, whose coefficient
// becomes R (1 - Rdot/c) + 4 mu/(rho c).  1/c = 0 gives Rayleigh-Plesset.
// The gas term comes from gas_pressure (binomial series around the last exact
// evaluation exp(3 gamma log(R0/R)), a few ulp from pow).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double accel64(const StepConst &K, const BinConst &bc, double p_inf,
                                          double R, double V, GasBase &g)
{
    const double icV = V * K.inv_c;
    const double den = fma(R, 1.0 - icV, K.fmu_ic_rho);
    // one division gives both reciprocals: 1/R = den/(R den), 1/den = R/(R den)
    const double inv = 1.0 / (R * den);
    const double iR = den * inv;
    const double iden = R * inv;
    const double VR = V * iR;
    double pg = 0.0;
    if (K.gas_mode == PAB_GAS_POLYTROPIC)
        pg = gas_pressure(K, bc, R, iR, g);  // p_g0 (R0/R)^(3 gamma)
    const double s = fma(K.four_mu, V, K.two_sigma);
    const double pbw = (K.pv + pg) - s * iR;
    const double dpbw = (s * iR - K.three_gamma * pg) * VR;
    const double num = (pbw - p_inf) * K.inv_rho * (1.0 + icV) + R * K.ic_rho * dpbw
                     - 1.5 * V * V * (1.0 - icV * (1.0 / 3.0));
    return num * iden;
}

// Wall pressure p_bw at (R, Rdot) in FP64 (for the <R^3 p_bw> moment).
__device__ __forceinline__ double wall_pressure64(const StepConst &K, const BinConst &bc, double R,
                                                  double V, GasBase &g)
{
    const double iR = 1.0 / R;
    double pg = 0.0;
    if (K.gas_mode == PAB_GAS_POLYTROPIC)
        pg = gas_pressure(K, bc, R, iR, g);
    return (K.pv + pg) - fma(K.four_mu, V, K.two_sigma) * iR;
}

// ---------------------------------------------------------------------------
// The same acceleration in FP32, written in deviations from equilibrium so
// that nothing cancels: with xi = R - R0, u = xi/R0,
//   p_b - pv - p_g0          = p_g0 expm1(-3 gamma log1p(u))
//   p_bw - p_inf             = A + (p_b - pv - p_g0) + (2 sigma u - 4 mu Rdot)/R
// where A = pv + p_g0 - 2 sigma/R0 - p_inf is formed in FP64 once per bin-step
// (for the polytropic gas A = p0 - p_inf).  Each term is then accurate
// relative to itself rather than to p0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float gas_dev32(const StepConst &K, const BinConst &bc, float u)
{
    return bc.pg0f * expm1f(-K.three_gammaf * log1pf(u));
}

__device__ __forceinline__ float accel32(const StepConst &K, const BinConst &bc, float A, float xi,
                                         float V)
{
    const float R = bc.R0f + xi;
    const float iR = 1.0f / R;
    const float u = xi * bc.invR0f;
    float pgdev = 0.0f, pg = 0.0f;
    if (K.gas_mode == PAB_GAS_POLYTROPIC) {
        pgdev = gas_dev32(K, bc, u);
        pg = bc.pg0f + pgdev;
    }
    const float VR = V * iR;
    const float s = fmaf(K.four_muf, V, K.two_sigmaf);
    const float dp = A + pgdev + (K.two_sigmaf * u - K.four_muf * V) * iR;
    const float dpbw = (s * iR - K.three_gammaf * pg) * VR;
    const float icV = V * K.inv_cf;
    const float num = dp * K.inv_rhof * (1.0f + icV) + R * K.ic_rhof * dpbw
                    - 1.5f * V * V * (1.0f - icV * (1.0f / 3.0f));
    const float den = fmaf(R, 1.0f - icV, K.fmu_ic_rhof);
    return num / den;
}

// ---------------------------------------------------------------------------
// One trial of the Shu-Osher SSP-RK3 scheme with the embedded SSP-RK2 (Heun)
// member sharing its first two evaluations (Sec. 3):
//   y1 = y + h f(y);  u = y1 + h f(y1)
//   y2 = 3/4 y + 1/4 u;  z = 1/2 (y + u)      (z: second order)
//   y3 = 1/3 y + 2/3 (y2 + h f(y2))           (third order, the one kept)
// ---------------------------------------------------------------------------
__device__ __forceinline__ Trial trial64(const StepConst &K, const BinConst &bc, double p_inf,
                                         double R, double V, double h, GasBase &g)
{
    const double a1 = accel64(K, bc, p_inf, R, V, g);
    const double y1R = fma(h, V, R), y1V = fma(h, a1, V);
    const double a2 = accel64(K, bc, p_inf, y1R, y1V, g);
    const double uR = fma(h, y1V, y1R), uV = fma(h, a2, y1V);
    const double zR = 0.5 * (R + uR), zV = 0.5 * (V + uV);
    const double y2R = fma(0.75, R, 0.25 * uR), y2V = fma(0.75, V, 0.25 * uV);
    const double a3 = accel64(K, bc, p_inf, y2R, y2V, g);
    const double wR = fma(h, y2V, y2R), wV = fma(h, a3, y2V);
    Trial t;
    t.R = fma(2.0 / 3.0, wR, R * (1.0 / 3.0));
    t.V = fma(2.0 / 3.0, wV, V * (1.0 / 3.0));
    t.eR = fabs(t.R - zR);
    t.eV = fabs(t.V - zV);
    t.ok = (y1R > 0.0) && (y2R > 0.0) && (t.R > 0.0) && (fabs(t.V) <= DBL_MAX);
    return t;
}

// The same trial with the three right-hand sides in FP32 on increments from
// y: k_j = h f(stage j).  y3 - y = (k1 + k2)/6 + 2/3 k3 and the embedded
// difference y3 - z = (2 k3 - k1 - k2)/3 is formed in FP64 from the k's, so
// the error estimate suffers no FP32 cancellation.  The new state is y plus
// the FP32 increment, added in FP64.
__device__ __forceinline__ Trial trial32(const StepConst &K, const BinConst &bc, float A, double R,
                                         double V, double h)
{
    const float xi0 = (float)(R - bc.R0);
    const float v0 = (float)V;
    const float hf = (float)h;
    const float a1 = accel32(K, bc, A, xi0, v0);
    const float k1R = hf * v0, k1V = hf * a1;
    const float v1 = v0 + k1V;
    const float a2 = accel32(K, bc, A, xi0 + k1R, v1);
    const float k2R = hf * v1, k2V = hf * a2;
    const float e2R = 0.25f * (k1R + k2R), e2V = 0.25f * (k1V + k2V);
    const float v2 = v0 + e2V;
    const float a3 = accel32(K, bc, A, xi0 + e2R, v2);
    const float k3R = hf * v2, k3V = hf * a3;
    const float d3R = (k1R + k2R) * (1.0f / 6.0f) + (2.0f / 3.0f) * k3R;
    const float d3V = (k1V + k2V) * (1.0f / 6.0f) + (2.0f / 3.0f) * k3V;
    Trial t;
    t.R = R + (double)d3R;
    t.V = V + (double)d3V;
    t.eR = fabs(2.0 * (double)k3R - ((double)k1R + (double)k2R)) * (1.0 / 3.0);
    t.eV = fabs(2.0 * (double)k3V - ((double)k1V + (double)k2V)) * (1.0 / 3.0);
    const float r1 = bc.R0f + (xi0 + k1R), r2 = bc.R0f + (xi0 + e2R);
    t.ok = (r1 > 0.0f) && (r2 > 0.0f) && (t.R > 0.0) && (fabs(t.V) <= DBL_MAX)
        && isfinite(a1 + a2 + a3);
    return t;
}

// Relative error of a trial: max(|dR|/|R3|, |dRdot|/max(|Rdot3|, v_floor)).
__device__ __forceinline__ double error_norm(const StepConst &K, const Trial &t)
{
    const double aR = fabs(t.R);
    const double vs = fmax(fabs(t.V), K.v_floor);
    return fmax(t.eR * vs, t.eV * aR) / (aR * vs);
}

// Step-size factor clamp(0.9 (tol/err)^(1/3), 0.2, 5); 0.2 after a failed trial.
// Below err = 1e-30 the clamp gives 5 for any tol >= 1e-18; past FP32 range, 0.2.
__device__ __forceinline__ double step_factor(const StepConst &K, double err, bool ok)
{
    if (!ok || !(err <= 3.0e38))
        return 0.2;
    if (err <= 1e-30)
        return 5.0;
    return fmin(fmax(0.9 * K.cbrt_tol * rcbrt_newton(err), 0.2), 5.0);
}

// ---------------------------------------------------------------------------
// Adaptive advance of one bin over dt with the carried proposal hc:
//   h = min(hc, dt) (dt when hc is not a positive number); the trial size is
//   min(h, dt - t) and the trial that reaches dt is marked last, so the call
//   ends exactly at dt; accepted: t += h_try, proposal h_try * fac (on the
//   last trial the unclipped h is kept when it was clipped and fac >= 1);
//   rejected: h = h_try * fac; at most max_attempts trials.
// MIXED selects the FP64 trial only where R < r_collapse R0 or
// |Rdot| > v_collapse, else the FP32 trial.
// ---------------------------------------------------------------------------
template <bool MIXED>
__device__ __forceinline__ uint32_t advance_adaptive(const StepConst &K, const BinConst &bc,
                                                     double p_inf, float A, double dt, double &R,
                                                     double &V, float &hc, int &n_att, int &n64,
                                                     GasBase &g)
{
    double h = (double)hc;
    if (!(h > 0.0) || h > dt)
        h = dt;
    double t = 0.0;
    uint32_t flags = 0;
    int n = 0;
    for (;;) {
        if (n >= K.max_attempts) {
            flags |= PAB_FLAG_STEP_LIMIT;
            break;
        }
        const double rem = dt - t;
        const bool last = h >= rem;
        const double ht = last ? rem : h;
        Trial tr;
        if (MIXED) {
            const bool stiff = (R < K.r_collapse * bc.R0) || (fabs(V) > K.v_collapse);
            if (stiff) {
                tr = trial64(K, bc, p_inf, R, V, ht, g);
                ++n64;
            } else {
                tr = trial32(K, bc, A, R, V, ht);
            }
        } else {
            tr = trial64(K, bc, p_inf, R, V, ht, g);
        }
        ++n;
        const double err = error_norm(K, tr);
        const double fac = step_factor(K, err, tr.ok);
        if (tr.ok && err <= K.tol) {
            R = tr.R;
            V = tr.V;
            if (last) {
                const bool clipped = rem < h;
                h = (clipped && fac >= 1.0) ? h : ht * fac;
                break;
            }
            t += ht;
            h = ht * fac;
        } else {
            h = ht * fac;
        }
    }
    hc = (float)h;
    n_att = n;
    return flags;
}

// ---------------------------------------------------------------------------
// Mixed-precision adaptive advance.  Same controller as advance_adaptive, with
// the trial's three right-hand sides in FP32 (deviation form) on increments
// k_j = h f(stage j) from the accepted state:
//   y3 - y = (k1 + k2)/6 + 2/3 k3,   y3 - z = (2 k3 - k1 - k2)/3.
// FP64 holds the state, the embedded error estimate (the k's promoted and
// combined in FP64), its norm and the accept decision, and the controller's
// time bookkeeping (t, dt - t, landing on dt).  The growth factor is formed in
// FP32: the proposal it scales is stored in FP32 between calls anyway.  The
// FP32 images of the state (xi = R - R0, Rdot) are refreshed only when a trial
// is accepted.  Bins near collapse (R < r_collapse R0 or |Rdot| > v_collapse)
// take the FP64 trial.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t advance_mixed(const StepConst &K, const BinConst &bc,
                                                  double p_inf, float A, double dt, double &R,
                                                  double &V, float &hc, int &n_att, int &n64,
                                                  float &xi, float &v)
{
    double h = (double)hc;
    if (!(h > 0.0) || h > dt)
        h = dt;
    double t = 0.0;
    uint32_t flags = 0;
    int n = 0;
    xi = (float)(R - bc.R0);
    v = (float)V;
    const float xi_collapse = (K.r_collapsef - 1.0f) * bc.R0f;
    for (;;) {
        if (n >= K.max_attempts) {
            flags |= PAB_FLAG_STEP_LIMIT;
            break;
        }
        const double rem = dt - t;
        const bool last = h >= rem;
        const double ht = last ? rem : h;
        double err, nR = 0.0, nV = 0.0;
        float d3R = 0.0f, d3V = 0.0f;
        bool ok, full64;
        if (xi < xi_collapse || fabsf(v) > K.v_collapsef) {
            GasBase g;
            g.reset();
            const Trial tr = trial64(K, bc, p_inf, R, V, ht, g);
            ++n64;
            err = error_norm(K, tr);
            ok = tr.ok;
            nR = tr.R;
            nV = tr.V;
            full64 = true;
        } else {
            const float hf = (float)ht;
            const float a1 = accel32(K, bc, A, xi, v);
            const float k1R = hf * v, k1V = hf * a1;
            const float v1 = v + k1V;
            const float a2 = accel32(K, bc, A, xi + k1R, v1);
            const float k2R = hf * v1, k2V = hf * a2;
            const float e2R = 0.25f * (k1R + k2R), e2V = 0.25f * (k1V + k2V);
            const float v2 = v + e2V;
            const float a3 = accel32(K, bc, A, xi + e2R, v2);
            const float k3R = hf * v2, k3V = hf * a3;
            d3R = (k1R + k2R) * (1.0f / 6.0f) + (2.0f / 3.0f) * k3R;
            d3V = (k1V + k2V) * (1.0f / 6.0f) + (2.0f / 3.0f) * k3V;
            const double eR = fabs(2.0 * (double)k3R - ((double)k1R + (double)k2R));
            const double eV = fabs(2.0 * (double)k3V - ((double)k1V + (double)k2V));
            const float R3f = bc.R0f + (xi + d3R);
            const float rR = 1.0f / (3.0f * fabsf(R3f));
            const float rV = 1.0f / (3.0f * fmaxf(fabsf(v + d3V), K.v_floorf));
            err = fmax(eR * (double)rR, eV * (double)rV);
            ok = (bc.R0f + (xi + k1R) > 0.0f) && (bc.R0f + (xi + e2R) > 0.0f) && (R3f > 0.0f)
              && isfinite(a1 + a2 + a3);
            full64 = false;
        }
        ++n;
        const float errf = (float)err;
        float fac;
        if (!ok || !(errf <= FLT_MAX))
            fac = 0.2f;
        else if (errf == 0.0f)
            fac = 5.0f;
        else
            fac = fminf(fmaxf(0.9f * K.cbrt_tolf * rcbrtf(errf), 0.2f), 5.0f);
        if (ok && err <= K.tol) {
            if (full64) {
                R = nR;
                V = nV;
            } else {
                R += (double)d3R;
                V += (double)d3V;
            }
            xi = (float)(R - bc.R0);
            v = (float)V;
            if (last) {
                const bool clipped = rem < h;
                h = (clipped && fac >= 1.0f) ? h : ht * (double)fac;
                break;
            }
            t += ht;
            h = ht * (double)fac;
        } else {
            h = ht * (double)fac;
        }
    }
    hc = (float)h;
    n_att = n;
    return flags;
}

// Fixed mode: n equal trials of dt/n, no error estimate (MIXED: FP64 trials
// only for bins near collapse, as in the adaptive mode).
template <bool MIXED>
__device__ __forceinline__ void advance_fixed(const StepConst &K, const BinConst &bc, double p_inf,
                                              float A, double dt, double &R, double &V, GasBase &g)
{
    const double h = dt / (double)K.n_fixed;
    for (int i = 0; i < K.n_fixed; ++i) {
        Trial tr;
        if (MIXED && !((R < K.r_collapse * bc.R0) || (fabs(V) > K.v_collapse)))
            tr = trial32(K, bc, A, R, V, h);
        else
            tr = trial64(K, bc, p_inf, R, V, h, g);
        R = tr.R;
        V = tr.V;
    }
}

// ---------------------------------------------------------------------------
// One (bin, cell) over one flow step: non-finite checks, fixed or adaptive
// advance, status bits.  R, V and hc are updated in place.
// ---------------------------------------------------------------------------
template <bool MIXED>
__device__ __forceinline__ uint32_t advance_bin(const StepConst &K, const BinConst &bc, double p_inf,
                                                bool p_ok, double dt, double &R, double &V, float &hc,
                                                int &na, int &n64, GasBase &g)
{
    na = 0;
    n64 = 0;
    if (!p_ok || !isfinite(R) || !isfinite(V))
        return PAB_FLAG_NONFINITE;
    uint32_t fl = 0;
    const float A = MIXED ? (float)(bc.peq - p_inf) : 0.0f;
    if (K.n_fixed > 0) {
        advance_fixed<MIXED>(K, bc, p_inf, A, dt, R, V, g);
        na = K.n_fixed;
    } else if (MIXED) {
        float xi, v;
        fl = advance_mixed(K, bc, p_inf, A, dt, R, V, hc, na, n64, xi, v);
    } else {
        fl = advance_adaptive<false>(K, bc, p_inf, A, dt, R, V, hc, na, n64, g);
    }
    if (!isfinite(R) || !isfinite(V))
        fl |= PAB_FLAG_NONFINITE;
    else if (!(R > 0.0))
        fl |= PAB_FLAG_NONPOS;
    if (fabs(V) >= K.c)
        fl |= PAB_FLAG_SUPERSONIC;
    return fl;
}

// Quadrature terms of one bin at (R, Rdot): w R^3, w R^2 Rdot, w R^3 p_bw,
// w R^3 Rdot^2 (the wall pressure in FP64, or in FP32 deviation form in MIXED).
template <bool MIXED>
__device__ __forceinline__ void quad_terms(const StepConst &K, const BinConst &bc, double R, double V,
                                           double t[4], GasBase &g)
{
    const double wr2 = bc.w * R * R;
    const double wr3 = wr2 * R;
    double pbw;
    if (MIXED) {
        const float xi = (float)(R - bc.R0);
        const float u = xi * bc.invR0f;
        const float pgdev = (K.gas_mode == PAB_GAS_POLYTROPIC) ? gas_dev32(K, bc, u) : 0.0f;
        pbw = bc.peq + (double)(pgdev + (K.two_sigmaf * u - K.four_muf * (float)V) / (float)R);
    } else {
        pbw = wall_pressure64(K, bc, R, V, g);
    }
    t[0] = wr3;
    t[1] = wr2 * V;
    t[2] = wr3 * pbw;
    t[3] = wr3 * V * V;
}

}  // namespace pab
