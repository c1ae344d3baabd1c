// Device arithmetic of the bubble source update: Keller-Miksis acceleration
// in FP64 and in an FP32 deviation form, one SSP-RK3/RK2 trial, the error
// norm, the step-size controller and the adaptive advance of one bin.
#pragma once

#include <math_constants.h>

#include <cfloat>
#include <cstdint>

#include "pab_bits.cuh"
#include "pab_check.cuh"
#include "pab_internal.h"
#include "pab_intmul.cuh"

namespace pab {

// Gas factor G = (R0/R)^(3 gamma) at the last exact evaluation, the base from
// which nearby radii are reached by the binomial series.
struct GasBase {
    double Rb, invRb, Gb;
    __device__ __forceinline__ void reset()
    {
        Rb = CUDART_NAN;  // forces an exact evaluation first
        invRb = CUDART_NAN;
        Gb = 0.0;
    }
};

// (1 + d)^(-3 gamma) by its binomial series truncated after N terms; callers
// keep |d| within the bound for N (gas_dmax for kGasTerms, gas_dmax_tab for
// kGasTabTerms), where the first omitted term is below half an ulp.
template <int N>
__device__ __forceinline__ double gas_series(const StepConst &K, double d)
{
    double s = K.gas_c[N - 1];
#pragma unroll
    for (int k = N - 2; k >= 0; --k)
        s = fma(s, d, K.gas_c[k]);
    return s;
}

// G = (R0/R)^(3 gamma) for R > 0.
//  - With a node table (a handle's gas_tab): x = R/R0 goes to the nearest node
//    x_j = q^j (picked in FP32: log2(x)/log2(q) rounded), and G is the node's
//    binomial series in delta = x - x_j, sum_k c_k delta^k (degree 3,
//    |delta| < x_j gas_dmax_tab). A pure function of R: no exp or log while R/R0
//    stays within the table.
//  - Otherwise (or outside the table): the radii of one step stay close to the
//    last exact evaluation R_b in g, reached by the degree-11 series in
//    d = (R - R_b)/R_b; farther away the value is exact, exp(-3 gamma log(R/R0)),
//    and becomes the new base.
static_assert(kGasTabStride == 6 && kGasTabTerms == 4, "gas table node layout");
__device__ __forceinline__ double gas_factor(const StepConst &K, const BinConst &bc, double R,
                                             GasBase &g)
{
    if (K.gas_tab) {
        const float xf = d2f(R) * bc.invR0f;
        const int j = __float2int_rn(__log2f(xf) * K.gas_inv_log2q);
        if (j >= -K.gas_J && j <= K.gas_J) {
            // {x_j, c_0}, {c_1, c_2}, {c_3, 0}
            const double2 *tab = reinterpret_cast<const double2 *>(K.gas_tab);
            const int e = 3 * (j + K.gas_J);
            const int ne = 3 * (2 * K.gas_J + 1);
            const double2 n0 = PAB_LDG(tab, e, ne), n1 = PAB_LDG(tab, e + 1, ne);
            const double c3 = PAB_LDG(K.gas_tab, 2 * (e + 2), 2 * ne);
            const double d = fma(R, bc.invR0, -n0.x);
            double s = fma(c3, d, n1.y);
            s = fma(s, d, n1.x);
            return fma(s, d, n0.y);
        }
    }
    const double d = (R - g.Rb) * g.invRb;
    if (le(abs_nn(d), K.gas_dmax))
        return g.Gb * gas_series<kGasTerms>(K, d);
    const double G = exp(-K.three_gamma * log(R * bc.invR0));
    g.Rb = R;
    g.invRb = rcp64(R);
    g.Gb = G;
    return G;
}


// The first trial size of a flow step from the carried FP32 proposal hc: hc
// itself when it is a number in (0, dt], else dt.  hc > 0 is tested in FP32
// (false for NaN); f2d_fin is exact below 2^104 and takes larger values, inf
// included, to at least 2^104, above any dt, so they fall back to dt too.
__device__ __forceinline__ double start_h(float hc, double dt)
{
    const double h = hc > 0.0f ? f2d_fin(hc) : dt;
    return le(h, dt) ? h : dt;
}

struct Trial {
    double R, V;    // third-order result y3
    double eR, eV;  // 3 (y3 - z) = 2 k3 - (k1 + k2) per component: three times the embedded
                    // second-order difference (its sign is dropped where it is multiplied)
    bool ok;        // every stage radius positive and y3 finite
};

// ---------------------------------------------------------------------------
// Keller-Miksis acceleration, Eq. (keller_miksis), FP64.
//   p_b = pv + p_g0 G,  G = (R0/R)^(3 gamma)   (Ando's ODE without transfer terms)
//   p_bw = p_b - s/R,   s = 4 mu Rdot + 2 sigma
//   d/dt p_bw = -3 gamma p_g0 G Rdot/R + s Rdot/R^2 - 4 mu Rddot/R
// The Rddot inside d/dt p_bw moves to the left-hand side, whose coefficient
// becomes den = R (1 - Rdot/c) + 4 mu/(rho c).  Collecting the right-hand side
// over rho, the s/R terms of (p_bw - p_inf)(1 + Rdot/c)/rho and of
// (R/(rho c)) d/dt p_bw add up to -s/(rho R), which leaves
//   Rddot = (N0 R - s/rho) / (R den),
//   N0 = P (1 + Rdot/c) - Rdot (3 gamma A1 G/c + Rdot (3/2 - Rdot/(2c))),  P = B0 + A1 G,
// with B0 = (pv - p_inf)/rho per cell and A1 = p_g0/rho per bin.  Regrouped on
// Rdot: N0 = P + Rdot (A3 G + B0/c - Rdot (3/2 - Rdot/(2c))) with the per-bin
// A3 = (1 - 3 gamma) A1/c and the per-cell B0/c: one reciprocal and no other
// division.  1/c = 0 gives Rayleigh-Plesset.
// ---------------------------------------------------------------------------
// The gas factor (R0/R)^(3 gamma) of the polytropic contents (0 for an empty cavity).
__device__ __forceinline__ double gas_G(const StepConst &K, const BinConst &bc, double R, GasBase &g)
{
    return (K.gas_mode == PAB_GAS_POLYTROPIC) ? gas_factor(K, bc, R, g) : 0.0;
}

// The acceleration for a given gas factor G at R.  INT: its two products (R den and the
// numerator times 1/(R den)) and the reciprocal formed on the integer pipe (pab_intmul.cuh),
// clearing ok where an operand or a result is not a normal number or zero.
template <bool INT>
__device__ __forceinline__ double accel64_G(const StepConst &K, const BinConst &bc, double B0,
                                            double B0c, double R, double V, double G, bool &ok)
{
    const double den = fma(R, fma(V, -K.inv_c, 1.0), K.fmu_ic_rho);
    const double inv = INT ? rcp_int(mul_int(R, int_factor(den), ok), ok) : rcp64(R * den);
    const double P = fma(bc.A1, G, B0);
    const double t = fma(-V, fma(V, K.m05_inv_c, 1.5), fma(bc.A3, G, B0c));
    const double N0 = fma(V, t, P);
    const double s_rho = fma(K.fmu_rho, V, K.tsig_rho);
    const double num = fma(N0, R, -s_rho);
    return INT ? mul_int(num, int_factor(inv), ok) : num * inv;
}

__device__ __forceinline__ double accel64_G(const StepConst &K, const BinConst &bc, double B0,
                                            double B0c, double R, double V, double G)
{
    bool ok = true;
    return accel64_G<false>(K, bc, B0, B0c, R, V, G, ok);
}

template <bool INT>
__device__ __forceinline__ double accel64(const StepConst &K, const BinConst &bc, double B0,
                                          double B0c, double R, double V, GasBase &g, bool &ok)
{
    return accel64_G<INT>(K, bc, B0, B0c, R, V, gas_G(K, bc, R, g), ok);
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
//
// The FP32 arithmetic of the mixed trial is written with explicit roundings
// (__fadd_rn, __fmul_rn, __fmaf_rn: never fused or split by the compiler), so
// every kernel that inlines it computes the same bits whatever its register
// budget; the divisions are IEEE (correctly rounded) divisions.
// ---------------------------------------------------------------------------
// (1 + u)^(-a) - 1 in FP32 for 1 + u > 0, accurate relative to itself near
// u = 0.  w = 1 + u = 2^k f with f in [sqrt(1/2), sqrt(2)), and
//   log2(1 + u) = k + t P(t) + c/(w ln 2),  t = f - 1,  c = u - (w - 1)
// (c the rounding of w, divided by w from the reciprocal seed: it is below an
// ulp of w); y = -a log2(1 + u), clamped to [-125, 125], splits as n + r with
// n an integer and |r| <= 1/2, and
//   (1 + u)^(-a) - 1 = 2^n (2^r - 1) + (2^n - 1),  2^r - 1 = r Q(r),
// with 2^n formed in the exponent field.  P (degree 8) and Q (degree 5) are
// minimax fits in relative error on those intervals (csrc/fit_gas32.py).
// Within 6 ulp for |u| < 1/2 and 11 ulp for u in (-0.8, 1000] at a = 4.2, as
// the composition expm1f(-a log1pf(u)) is; no branches and no library call.
__device__ __forceinline__ float pow_m1_32(float u, float a)
{
    const float w = __fadd_rn(1.0f, u);
    const float c = __fsub_rn(u, __fsub_rn(w, 1.0f));
    const uint32_t wb = __float_as_uint(w);
    const int k = (int)(wb - 0x3f3504f3u) >> 23;
    const float t = __fsub_rn(__uint_as_float(wb - ((uint32_t)k << 23)), 1.0f);
    float p = 0x1.01b48cp-3f;
    p = __fmaf_rn(p, t, -0x1.a87c04p-3f);
    p = __fmaf_rn(p, t, 0x1.b9c97ap-3f);
    p = __fmaf_rn(p, t, -0x1.e95c12p-3f);
    p = __fmaf_rn(p, t, 0x1.26d382p-2f);
    p = __fmaf_rn(p, t, -0x1.715c4ep-2f);
    p = __fmaf_rn(p, t, 0x1.ec73d6p-2f);
    p = __fmaf_rn(p, t, -0x1.71547p-1f);
    p = __fmaf_rn(p, t, 0x1.715476p+0f);
    const float cw = __fmul_rn(__fmul_rn(c, rcp_seed32(w)), 0x1.715476p+0f);  // c / (w ln 2)
    const float l2 = __fadd_rn(__int2float_rn(k), __fmaf_rn(t, p, cw));
    const float y = fminf(fmaxf(__fmul_rn(-a, l2), -125.0f), 125.0f);
    const float mg = __fadd_rn(y, 0x1.8p23f);  // y rounded to an integer in the low bits
    const float r = __fsub_rn(y, __fsub_rn(mg, 0x1.8p23f));
    const int n = (int)(__float_as_uint(mg) - 0x4b400000u);
    float q = 0x1.4308eap-13f;
    q = __fmaf_rn(q, r, 0x1.5f07b6p-10f);
    q = __fmaf_rn(q, r, 0x1.3b2ba0p-7f);
    q = __fmaf_rn(q, r, 0x1.c6af6ep-5f);
    q = __fmaf_rn(q, r, 0x1.ebfbdep-3f);
    q = __fmaf_rn(q, r, 0x1.62e430p-1f);
    const float sc = __uint_as_float((uint32_t)(n + 127) << 23);
    return __fmaf_rn(sc, __fmul_rn(r, q), __fsub_rn(sc, 1.0f));
}

// (BC: BinConst, or any bin type with the FP32 fields R0f, invR0f and pg0f.)
template <class BC>
__device__ __forceinline__ float gas_dev32(const StepConst &K, const BC &bc, float u)
{
    return __fmul_rn(bc.pg0f, pow_m1_32(u, K.three_gammaf));
}

// With iR = 1/R the numerator of the deviation form is P + Q iR,
//   P = L (A + pgdev) - 3 gamma (1/c)/rho p_g Rdot - 3/2 Rdot^2 (1 - Rdot/(3c)),
//   Q = L (2 sigma u - 4 mu Rdot) + (1/c)/rho Rdot (2 sigma + 4 mu Rdot),
// with L = (1 + Rdot/c)/rho, so Rddot = (P R + Q) / (R den): one division.
template <class BC>
__device__ __forceinline__ float accel32(const StepConst &K, const BC &bc, float A, float xi,
                                         float V)
{
    const float R = __fadd_rn(bc.R0f, xi);
    const float u = __fmul_rn(xi, bc.invR0f);
    float pgdev = 0.0f, pg = 0.0f;
    if (K.gas_mode == PAB_GAS_POLYTROPIC) {
        pgdev = gas_dev32(K, bc, u);
        pg = __fadd_rn(bc.pg0f, pgdev);
    }
    const float icV = __fmul_rn(V, K.inv_cf);
    const float L = __fmul_rn(K.inv_rhof, __fadd_rn(1.0f, icV));
    const float s = __fmaf_rn(K.four_muf, V, K.two_sigmaf);                  // 2 sigma + 4 mu Rdot
    const float st = __fmaf_rn(K.two_sigmaf, u, __fmul_rn(-K.four_muf, V));  // 2 sigma u - 4 mu Rdot
    const float kin = __fmul_rn(__fmul_rn(V, V), __fmaf_rn(-0.5f, icV, 1.5f));
    const float gas = __fmul_rn(__fmul_rn(K.tg_ic_rhof, pg), V);
    const float P = __fmaf_rn(L, __fadd_rn(A, pgdev), -__fadd_rn(gas, kin));
    const float Q = __fmaf_rn(L, st, __fmul_rn(__fmul_rn(K.ic_rhof, V), s));
    const float den = __fmaf_rn(R, __fsub_rn(1.0f, icV), K.fmu_ic_rhof);
    return div32(__fmaf_rn(P, R, Q), __fmul_rn(R, den));
}

// ---------------------------------------------------------------------------
// One trial of the Shu-Osher SSP-RK3 scheme with the embedded SSP-RK2 (Heun)
// member sharing its first two evaluations (Sec. 3):
//   y1 = y + h f(y);  u = y1 + h f(y1)
//   y2 = 3/4 y + 1/4 u;  z = 1/2 (y + u)      (z: second order)
//   y3 = 1/3 y + 2/3 (y2 + h f(y2))           (third order, the one kept)
// written with the increments k1 = h f(y), k2 = h f(y1), k3 = h f(y2):
//   y1 = y + k1,  y2 = y + (k1 + k2)/4,  y3 = y + (k1 + k2)/6 + 2/3 k3,
//   3 (y3 - z) = 2 k3 - (k1 + k2).
// ---------------------------------------------------------------------------
// (haveG: G0 is the gas factor at the trial's start R, known from before, and the first
// right-hand side takes it instead of evaluating it; G0used returns the factor it used.)
// INT: the trial's plain products (k1 = h f(y) and the two of each right-hand side) formed on
// the integer pipe, each within 1 ulp of the FP64 product, GB300's FP64 pipe being the bound of
// the step; ok is cleared where one of them meets a value that is not a normal number or zero.
template <bool INT>
__device__ __forceinline__ Trial trial64_body(const StepConst &K, const BinConst &bc, double B0,
                                              double B0c, double R, double V, double h, GasBase &g,
                                              bool haveG, double G0, double &G0used, bool &ok)
{
    G0used = haveG ? G0 : gas_G(K, bc, R, g);
    const double a1 = accel64_G<INT>(K, bc, B0, B0c, R, V, G0used, ok);
    // y1 = y + h f(y) as one FMA (k1 itself is still formed for k1 + k2): every product-sum of
    // the trial is an explicit fma, so the compiler contracts nothing and the bits do not depend
    // on the kernel the trial is inlined into or on its register budget
    double k1R, k1V;
    if (INT) {
        const IntFactor fh = int_factor(h);
        k1R = mul_int(V, fh, ok);
        k1V = mul_int(a1, fh, ok);
    } else {
        k1R = h * V;
        k1V = h * a1;
    }
    const double y1R = fma(h, V, R), y1V = fma(h, a1, V);
    const double a2 = accel64<INT>(K, bc, B0, B0c, y1R, y1V, g, ok);
    const double sR = fma(h, y1V, k1R), sV = fma(h, a2, k1V);   // k1 + k2
    const double y2R = fma(0.25, sR, R), y2V = fma(0.25, sV, V);
    const double a3 = accel64<INT>(K, bc, B0, B0c, y2R, y2V, g, ok);
    // 2 k3 = (2h) f(y2) with 2h exact; y3 = y + (k1 + k2)/6 + 2/3 k3 written as
    // y + (k1 + k2)/2 + (2 k3 - (k1 + k2))/3
    const double h2 = twice_nn(h);
    Trial t;
    t.eR = fma(h2, y2V, -sR);
    t.eV = fma(h2, a3, -sV);
    t.R = fma(1.0 / 3.0, t.eR, fma(0.5, sR, R));
    t.V = fma(1.0 / 3.0, t.eV, fma(0.5, sV, V));
    t.ok = gt0(y1R) && gt0(y2R) && gt0(t.R) && finite64(t.V);
    return t;
}

// The trial with its products on the integer pipe, and again with FP64 products where one of
// them met a subnormal, infinite or NaN value or left the normal range.
__device__ __forceinline__ Trial trial64(const StepConst &K, const BinConst &bc, double B0,
                                         double B0c, double R, double V, double h, GasBase &g,
                                         bool haveG, double G0, double &G0used)
{
    bool ok = true;
    Trial t = trial64_body<true>(K, bc, B0, B0c, R, V, h, g, haveG, G0, G0used, ok);
    if (!ok)
        t = trial64_body<false>(K, bc, B0, B0c, R, V, h, g, haveG, G0, G0used, ok);
    return t;
}

__device__ __forceinline__ Trial trial64(const StepConst &K, const BinConst &bc, double B0,
                                         double B0c, double R, double V, double h, GasBase &g)
{
    double G0;
    return trial64(K, bc, B0, B0c, R, V, h, g, false, 0.0, G0);
}

// The trial with FP64 products: the mixed path's FP64 trials near collapse, too few to repay
// the integer form's registers in kernels held to 64 of them.
__device__ __forceinline__ Trial trial64_fp64(const StepConst &K, const BinConst &bc, double B0,
                                              double B0c, double R, double V, double h, GasBase &g)
{
    double G0;
    bool ok = true;
    return trial64_body<false>(K, bc, B0, B0c, R, V, h, g, false, 0.0, G0, ok);
}

// The embedded difference 2 k3 - (k1 + k2) of FP32 increments, from exact
// parts: k1 + k2 = s + e_s and 2 k3 - s = d + e_d by FP32 TwoSum (2 k3 is
// exact), so the difference is d + (e_d - e_s) exactly.  The two rounding
// errors are combined in FP32 (e_d - e_s rounded once, an error of at most
// 2^-48 (|d| + |s|)) and added to d in FP64: the difference to within 2^-47 of
// the increments at one FP64 addition, where promoting the k's and subtracting
// in FP64 takes three (and keeps a relative error of 2^-53 of the increments).
// For finite |k| < 2^100 (the parts then stay inside f2d_fin's range); a
// trial's increments are many orders below that, and a non-finite one fails
// the trial.
__device__ __forceinline__ double embedded_diff(float k1, float k2, float k3, float &d)
{
    float s, es, ed;
    two_sum(k1, k2, s, es);
    two_sum(__fmul_rn(2.0f, k3), -s, d, ed);
    return f2d_fin(d) + f2d_fin(__fsub_rn(ed, es));
}

// The accept test on one component, |2 k3 - (k1 + k2)| <= T with the difference formed as
// embedded_diff forms it (and d, its FP32 part), deciding in FP32 where the parts' bound settles
// it.  The correction e = e_d - e_s is at most 2^-24 (|d| + |s|) (1 + 2^-24) (each TwoSum error is
// at most half an ulp of its sum, and the FP32 subtraction rounds once), so b = 2^-22 (|d| + |s|)
// bounds it with room for the roundings of the comparisons: |d| + b <= T (1 - 2^-20) means the
// FP64 sum is below T, |d| - b > T (1 + 2^-20) that it is above.  Only differences inside that
// bracket (or non-finite operands) take the FP64 addition of the exact test; the decision is the
// exact test's either way.
__device__ __forceinline__ bool embedded_within(float k1, float k2, float k3, float T, float &d)
{
    float s, es, ed;
    two_sum(k1, k2, s, es);
    two_sum(__fmul_rn(2.0f, k3), -s, d, ed);
    const float e = __fsub_rn(ed, es);
    const float ad = fabsf(d);
    const float b = __fmul_rn(0x1p-22f, __fadd_rn(ad, fabsf(s)));
    if (T <= FLT_MAX) {
        if (__fadd_rn(ad, b) <= __fmul_rn(T, 1.0f - 0x1p-20f))
            return true;
        if (__fsub_rn(ad, b) > __fmul_rn(T, 1.0f + 0x1p-20f))
            return false;
    }
    return le(abs_nn(f2d_fin(d) + f2d_fin(e)), f2d_fin(T));
}

// The three FP32 right-hand sides of one trial, on increments from the state
// (xi = R - R0, v) with k_j = h f(stage j):
//   stage 2 = y + k1,  stage 3 = y + (k1 + k2)/4,  y3 - y = (k1 + k2)/6 + 2/3 k3.
// ok: both inner stage radii positive and every right-hand side finite.
struct Incr32 {
    float k1R, k2R, k3R, k1V, k2V, k3V;
    float d3R, d3V;  // y3 - y
    bool ok;
};
template <class BC>
__device__ __forceinline__ Incr32 incr32(const StepConst &K, const BC &bc, float A, float xi,
                                         float v, float hf)
{
    Incr32 t;
    const float a1 = accel32(K, bc, A, xi, v);
    t.k1R = __fmul_rn(hf, v);
    t.k1V = __fmul_rn(hf, a1);
    const float x1 = __fadd_rn(xi, t.k1R), v1 = __fadd_rn(v, t.k1V);
    const float a2 = accel32(K, bc, A, x1, v1);
    t.k2R = __fmul_rn(hf, v1);
    t.k2V = __fmul_rn(hf, a2);
    const float sR = __fadd_rn(t.k1R, t.k2R), sV = __fadd_rn(t.k1V, t.k2V);
    const float x2 = __fmaf_rn(0.25f, sR, xi), v2 = __fmaf_rn(0.25f, sV, v);
    const float a3 = accel32(K, bc, A, x2, v2);
    t.k3R = __fmul_rn(hf, v2);
    t.k3V = __fmul_rn(hf, a3);
    t.d3R = __fmaf_rn(2.0f / 3.0f, t.k3R, __fmul_rn(1.0f / 6.0f, sR));
    t.d3V = __fmaf_rn(2.0f / 3.0f, t.k3V, __fmul_rn(1.0f / 6.0f, sV));
    t.ok = (__fadd_rn(bc.R0f, x1) > 0.0f) && (__fadd_rn(bc.R0f, x2) > 0.0f)
        && isfinite(__fadd_rn(__fadd_rn(a1, a2), a3));
    return t;
}

// The trial with the three right-hand sides in FP32.  The embedded difference
// y3 - z = (2 k3 - k1 - k2)/3 is formed in FP64 from the k's, so the error
// estimate suffers no FP32 cancellation.  The new state is y plus the FP32
// increment, added in FP64.
__device__ __forceinline__ Trial trial32(const StepConst &K, const BinConst &bc, float A, double R,
                                         double V, double h)
{
    const Incr32 in = incr32(K, bc, A, d2f(R - bc.R0), d2f(V), d2f(h));
    Trial t;
    t.R = R + f2d_fin(in.d3R);
    t.V = V + f2d_fin(in.d3V);
    float dR, dV;
    t.eR = embedded_diff(in.k1R, in.k2R, in.k3R, dR);
    t.eV = embedded_diff(in.k1V, in.k2V, in.k3V, dV);
    t.ok = in.ok && gt0(t.R) && finite64(t.V);
    return t;
}

// Growth factor of the controller, clamp(0.9 (tol/err)^(1/3), 0.2, 5), in FP32
// (a heuristic whose product is stored in FP32 between calls): 0.2 after a
// failed trial or an error past the FP32 range, 5 for a zero error.
__device__ __forceinline__ float growth_factor(const StepConst &K, float errf, bool ok)
{
    if (!ok || !(errf <= FLT_MAX))
        return 0.2f;
    if (errf == 0.0f)
        return 5.0f;
    return fminf(fmaxf(0.9f * K.cbrt_tolf * rcbrtf(errf), 0.2f), 5.0f);
}

// Accept test and growth factor of an FP64 trial.  err <= tol is written
// without a division, |eR| <= tol |R3| and |eRdot| <= tol max(|Rdot3|, v_floor)
// (two FP64 products and integer compares on the threefold differences the
// trial carries, against 3 tol; when ok holds R3 is positive and finite).  The
// factor takes err from the FP32 images of the same quantities.
struct Decision {
    bool accept;
    float fac;
    float errf;  // the FP32 error estimate the factor was taken from
};
// The FP32 estimate errf is within 1e-6 (relative) of err: each image rounds once (2^-24), the
// approximate quotient is within 2 ulp for the normal denominators required here, and the
// product by 1/3 rounds once.  Outside err = tol (1 -/+ 2^-16) it therefore decides as the exact
// test does, which then runs only for estimates in that bracket (or for denominators, error
// images and estimates outside the FP32 range, NaNs included): the same decisions, without its
// two FP64 products.  (For
// tol below 1e-7, where an error image flushed to zero could matter, the bracket is closed.)
__device__ __forceinline__ Decision decide64(const StepConst &K, const Trial &t)
{
    const double aR = abs_nn(t.R);
    const double vs = max_nn(abs_nn(t.V), K.v_floor);
    const float aRf = d2f(aR), vsf = d2f(vs);
    const float eRf = d2f(abs_nn(t.eR)), eVf = d2f(abs_nn(t.eV));
    const float errf = (1.0f / 3.0f) * fmaxf(__fdividef(eRf, aRf), __fdividef(eVf, vsf));
    Decision v;
    // (fmaxf drops a NaN operand: the bracket needs both error images finite)
    const bool sure = aRf >= 0x1p-100f && aRf <= 0x1p100f && vsf >= 0x1p-100f && vsf <= 0x1p100f &&
                      eRf <= FLT_MAX && eVf <= FLT_MAX &&
                      (errf <= K.tol_lof || (errf > K.tol_hif && errf <= FLT_MAX));
    if (!t.ok)
        v.accept = false;
    else if (sure)
        v.accept = errf <= K.tol_lof;
    else
        v.accept = le(abs_nn(t.eR), K.tol3 * aR) && le(abs_nn(t.eV), K.tol3 * vs);
    v.fac = growth_factor(K, errf, t.ok);
    v.errf = errf;
    return v;
}

// ---------------------------------------------------------------------------
// Adaptive advance of one bin over dt with the carried proposal hc:
//   h = min(hc, dt) (dt when hc is not a positive number); the trial size is
//   min(h, rem) with rem the time left of the flow step, and the trial that
//   reaches dt is marked last, so the call ends exactly at dt; accepted:
//   rem -= h_try, proposal h_try * fac (on the last trial the unclipped h is
//   kept when it was clipped and fac >= 1); rejected: h = h_try * fac; at most
//   max_attempts trials.
// FP64 trials throughout (the mixed mode has its own loop, advance_mixed).
// ---------------------------------------------------------------------------
// A cell's pressure terms, the same for all its bins: B0 = (pv - p_inf)/rho and B0/c (FP64
// trials), the FP32 image of p0 - p_inf (mixed trials).
struct CellTerms {
    double B0, B0c;
    float A0;
};
template <bool MIXED>
__device__ __forceinline__ CellTerms cell_terms(const StepConst &K, double p_inf)
{
    CellTerms t;
    t.B0 = (K.pv - p_inf) * K.inv_rho;
    t.B0c = t.B0 * K.inv_c;
    t.A0 = MIXED ? d2f(K.p0 - p_inf) : 0.0f;
    return t;
}

__device__ __forceinline__ uint32_t advance_adaptive(const StepConst &K, const BinConst &bc,
                                                     double B0, double B0c, double dt, double &R,
                                                     double &V, float &hc, int &n_att, GasBase &g)
{
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
        const Trial tr = trial64(K, bc, B0, B0c, R, V, ht, g);
        ++n;
        const Decision vd = decide64(K, tr);
        const double fac = f2d_fin(vd.fac);
        if (vd.accept) {
            R = tr.R;
            V = tr.V;
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

// The FP64 trial of a bin near collapse in the mixed mode, with the FP64 kernel's accept
// test and error estimate (decide64).  (Kept inline: out of line, to spare the FP32 loop its
// registers, it measured 2 % slower.)
struct Trial64Out {
    double R, V;
    bool ok, accept;
    float errf;
};
__device__ __forceinline__ Trial64Out collapse_trial64(const StepConst &K, const BinConst &bc,
                                                       double p_inf, double R, double V, double h)
{
    GasBase g;
    g.reset();
    const double B0 = (K.pv - p_inf) * K.inv_rho;
    const Trial tr = trial64_fp64(K, bc, B0, B0 * K.inv_c, R, V, h, g);
    const Decision vd = decide64(K, tr);
    return {tr.R, tr.V, tr.ok, vd.accept, vd.errf};
}

// ---------------------------------------------------------------------------
// Mixed-precision adaptive advance.  Same controller as advance_adaptive, with
// the trial's three right-hand sides in FP32 (deviation form) on increments
// k_j = h f(stage j) from the accepted state:
//   y3 - y = (k1 + k2)/6 + 2/3 k3,   y3 - z = (2 k3 - k1 - k2)/3.
// FP64 holds the state (inside the loop the radius as its offset R - R0 from
// the bin's equilibrium, so the FP32 image needs no subtraction per step), the
// embedded error estimate (exact parts combined in FP64), its norm and the
// accept decision, and the controller's time bookkeeping (the time left of
// the flow step, counted down, and landing on dt).  The growth factor is formed in
// FP32: the proposal it scales is stored in FP32 between calls anyway.  The
// FP32 images of the state (xi = R - R0, Rdot) change only when a trial is
// accepted: by the same FP32 increments after an FP32 trial, from the state
// after an FP64 one.  Bins near collapse (R < r_collapse R0 or |Rdot| > v_collapse)
// take the FP64 trial.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t advance_mixed(const StepConst &K, const BinConst &bc,
                                                  double p_inf, float A, double dt, double &R,
                                                  double &V, float &hc, int &n_att, int &n64,
                                                  float &xi, float &v)
{
    double h = start_h(hc, dt);
    double rem = dt;  // time left of the flow step
    uint32_t flags = 0;
    int n = 0;
    double xi64 = R - bc.R0;  // the radius offset is the FP64 state inside the loop
    xi = d2f(xi64);
    v = d2f(V);
    const float xi_collapse = (K.r_collapsef - 1.0f) * bc.R0f;
    for (;;) {
        if (n >= K.max_attempts) {
            flags |= PAB_FLAG_STEP_LIMIT;
            break;
        }
        const bool last = le(rem, h);
        const double ht = last ? rem : h;
        const float htf = d2f(ht);
        double nR = 0.0, nV = 0.0;
        float d3R = 0.0f, d3V = 0.0f, errf;
        bool ok, accept, full64;
        if (xi < xi_collapse || fabsf(v) > K.v_collapsef) {
            const Trial64Out tr = collapse_trial64(K, bc, p_inf, bc.R0 + xi64, V, ht);
            ++n64;
            ok = tr.ok;
            accept = tr.accept;
            errf = tr.errf;
            nR = tr.R;
            nV = tr.V;
            full64 = true;
        } else {
            const Incr32 in = incr32(K, bc, A, xi, v, htf);
            d3R = in.d3R;
            d3V = in.d3V;
            float dR, dV;
            const float R3f = __fadd_rn(bc.R0f, __fadd_rn(xi, d3R));
            const float aRf = fabsf(R3f);
            const float aVf = fmaxf(fabsf(__fadd_rn(v, d3V)), K.v_floorf);
            ok = in.ok && (R3f > 0.0f);
            // err <= tol as |e_R| <= 3 tol |R3| and |e_Rdot| <= 3 tol max(|Rdot3|, v_floor):
            // the embedded estimate (FP64 where the FP32 bracket does not settle it) against
            // thresholds formed in FP32 (a relative rounding of 6e-8 on tol, no FP64 product);
            // the growth factor takes err from the FP32 differences d (they differ from the
            // estimate only where it is tiny, and the factor is 5 there either way) and the
            // FP32 images of R3, Rdot3
            const bool wR = embedded_within(in.k1R, in.k2R, in.k3R, __fmul_rn(K.tol3f, aRf), dR);
            const bool wV = embedded_within(in.k1V, in.k2V, in.k3V, __fmul_rn(K.tol3f, aVf), dV);
            accept = ok && wR && wV;
            errf = fmaxf(__fmul_rn(fabsf(dR), rcp32(__fmul_rn(3.0f, aRf))),
                         __fmul_rn(fabsf(dV), rcp32(__fmul_rn(3.0f, aVf))));
            full64 = false;
        }
        ++n;
        const float fac = growth_factor(K, errf, ok);
        // the next proposal, kept in FP32 between calls anyway: an exact FP32 product
        const double hn = f2d_fin(__fmul_rn(htf, fac));
        if (accept) {
            if (full64) {
                xi64 = nR - bc.R0;
                V = nV;
                xi = d2f(xi64);
                v = d2f(V);
            } else {
                // the FP32 images move by the same increments: within an ulp or two of
                // the state's own images until the next flow step derives them afresh
                xi64 += f2d_fin(d3R);
                V += f2d_fin(d3V);
                xi = __fadd_rn(xi, d3R);
                v = __fadd_rn(v, d3V);
            }
            if (last) {
                const bool clipped = !le(h, rem);
                h = (clipped && fac >= 1.0f) ? h : hn;
                break;
            }
            rem -= ht;
            h = hn;
        } else {
            h = hn;
        }
    }
    R = bc.R0 + xi64;
    hc = d2f(h);
    n_att = n;
    return flags;
}

// Fixed mode: n equal trials of dt/n, no error estimate (MIXED: FP64 trials
// only for bins near collapse, as in the adaptive mode).
// h = dt / n_fixed comes from the host (a division here would be hoisted out
// of the bin loop and run in every thread, adaptive mode included).
template <bool MIXED>
__device__ __forceinline__ void advance_fixed(const StepConst &K, const BinConst &bc, double p_inf,
                                              float A, double h, double &R, double &V, GasBase &g)
{
    const double B0 = (K.pv - p_inf) * K.inv_rho;
    const double B0c = B0 * K.inv_c;
    for (int i = 0; i < K.n_fixed; ++i) {
        Trial tr;
        if (MIXED && !((R < K.r_collapse * bc.R0) || (fabs(V) > K.v_collapse)))
            tr = trial32(K, bc, A, R, V, h);
        else
            tr = MIXED ? trial64_fp64(K, bc, B0, B0c, R, V, h, g) : trial64(K, bc, B0, B0c, R, V, h, g);
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
                                                const CellTerms &ct, bool p_ok, double dt, double dt_sub,
                                                double &R, double &V, float &hc, int &na, int &n64,
                                                GasBase &g)
{
    na = 0;
    n64 = 0;
    if (!p_ok || !finite64(R) || !finite64(V))
        return PAB_FLAG_NONFINITE;
    uint32_t fl = 0;
    const float A = MIXED ? bc.dpeqf + ct.A0 : 0.0f;
    if (K.n_fixed > 0) {
        advance_fixed<MIXED>(K, bc, p_inf, A, dt_sub, R, V, g);
        na = K.n_fixed;
    } else if (MIXED) {
        float xi, v;
        fl = advance_mixed(K, bc, p_inf, A, dt, R, V, hc, na, n64, xi, v);
    } else {
        fl = advance_adaptive(K, bc, ct.B0, ct.B0c, dt, R, V, hc, na, g);
    }
    if (!finite64(R) || !finite64(V))
        fl |= PAB_FLAG_NONFINITE;
    else if (!gt0(R))
        fl |= PAB_FLAG_NONPOS;
    if (abs_ge(V, K.c))
        fl |= PAB_FLAG_SUPERSONIC;
    return fl;
}

// Quadrature terms of one bin at (R, Rdot), FP64: w R^3, w R^2 Rdot,
// w R^3 p_bw / rho (= w R^3 p_b/rho - w R^2 s/rho with p_b/rho = pv/rho + A1 G: no division),
// w R^3 Rdot^2.  Every product
// is rounded explicitly, so a sum of the terms comes out the same whether the
// caller stores them first or adds them as they come.
// (G returns the gas factor at R the terms used, the value the next flow step starts from.)
// (The terms with FP64 products: out of line, for the states whose products the integer form
// below does not take; returned by value, so that the caller's terms stay in registers.)
struct Terms4 {
    double t0, t1, t2, t3;
};
static __device__ __noinline__ Terms4 quad_terms64_fp64(const BinConst &bc, double R, double V,
                                                        double G, double pv_rho, double fmu_rho,
                                                        double tsig_rho)
{
    const double wr2 = __dmul_rn(__dmul_rn(bc.w, R), R);
    const double wr3 = __dmul_rn(wr2, R);
    return Terms4{wr3, __dmul_rn(wr2, V),
                  fma(wr3, fma(bc.A1, G, pv_rho), -__dmul_rn(wr2, fma(fmu_rho, V, tsig_rho))),
                  __dmul_rn(__dmul_rn(wr3, V), V)};
}

// The products formed from the significands on the integer pipe (pab_intmul.cuh, each within
// 1 ulp of the FP64 product), GB300's FP64 pipe being the bound of the FP64 step; where one of
// them meets a subnormal, infinite or NaN value the terms are formed again with FP64 products.
__device__ __forceinline__ void quad_terms64(const StepConst &K, const BinConst &bc, double R, double V,
                                             double t[4], GasBase &g, double &G)
{
    G = gas_G(K, bc, R, g);
    bool ok = true;
    const IntFactor fR = int_factor(R);
    const double wr2 = mul_int(mul_int(bc.w, fR, ok), fR, ok);
    const double wr3 = mul_int(wr2, fR, ok);
    t[0] = wr3;
    t[1] = mul2_int(wr2, V, ok);
    t[2] = fma(wr3, fma(bc.A1, G, K.pv_rho), -mul2_int(wr2, fma(K.fmu_rho, V, K.tsig_rho), ok));
    t[3] = mul2_int(mul2_int(wr3, V, ok), V, ok);
    if (!ok) {
        const Terms4 f = quad_terms64_fp64(bc, R, V, G, K.pv_rho, K.fmu_rho, K.tsig_rho);
        t[0] = f.t0;
        t[1] = f.t1;
        t[2] = f.t2;
        t[3] = f.t3;
    }
}
__device__ __forceinline__ void quad_terms64(const StepConst &K, const BinConst &bc, double R, double V,
                                             double t[4], GasBase &g)
{
    double G;
    quad_terms64(K, bc, R, V, t, g, G);
}

// The same terms in mixed precision: w R^3 in FP64 (for the compensated alpha
// sum), and in FP32 w R^2 Rdot, w R^3 (p_bw - p0) (the wall pressure in
// deviation form; p0 sum w R^3 is added once per cell) and w R^3 Rdot^2, with
// explicit roundings as above.
__device__ __forceinline__ double quad_terms_mixed(const StepConst &K, const BinConst &bc, double R,
                                                   double V, float tf[3])
{
    const double wr3 = __dmul_rn(__dmul_rn(__dmul_rn(bc.w, R), R), R);
    const float xi = d2f(R - bc.R0);
    const float u = __fmul_rn(xi, bc.invR0f);
    const float Rf = __fadd_rn(bc.R0f, xi), Vf = d2f(V);
    const float pgdev = (K.gas_mode == PAB_GAS_POLYTROPIC) ? gas_dev32(K, bc, u) : 0.0f;
    const float iRf = rcp32(Rf);
    const float st = __fmaf_rn(K.two_sigmaf, u, __fmul_rn(-K.four_muf, Vf));  // 2 sigma u - 4 mu Rdot
    const float dev = __fadd_rn(__fadd_rn(bc.dpeqf, pgdev), __fmul_rn(st, iRf));
    const float wr3f = d2f(wr3), wr2f = __fmul_rn(wr3f, iRf);  // w R^2 = w R^3 / R
    tf[0] = __fmul_rn(wr2f, Vf);
    tf[1] = __fmul_rn(wr3f, dev);
    tf[2] = __fmul_rn(__fmul_rn(wr3f, Vf), Vf);
    return wr3;
}

}  // namespace pab
