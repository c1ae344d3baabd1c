/*
 * Plain FP64 CPU oracle for the ensemble-averaged (Euler-Euler) bubble-dynamics
 * source update of "Hardware-Accelerated Phase-Averaging for Cavitating Bubbly
 * Flows" (arXiv 2511.21031).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check, and the CPU-baseline
 * leg and the reference arm of the benchmark may load this library.  The product path (the CUDA
 * library) shares no code, header, table or helper with it.
 *
 * Every function follows the paper's statement of the method in the paper's
 * order and notation, with no blocking, fusion or reordering:
 *   - Sec. 2, Eq. (keller_miksis): Keller-Miksis radial ODE, p_bw = p_b - 4 mu Rdot/R - 2 sigma/R.
 *   - Sec. 2, Ando bubble-pressure ODE with the transfer terms set to zero,
 *     which integrates to the polytropic closed form p_b = p_v + p_g0 (R0/R)^(3 gamma).
 *   - Sec. 2.2: lognormal R0 distribution in Nb bins, Simpson quadrature,
 *     Eq. (e:ndf) alpha = (4/3) pi n_b <R^3>, Eq. (e:alpha) source 3 alpha <R^2 Rdot>/<R^3>,
 *     Eq. (e:pressure) moments <R^3 p_bw>/<R^3> and <R^3 Rdot^2>/<R^3>.
 *   - Sec. 3: third-order TVD (SSP) Runge-Kutta with the embedded second-order
 *     TVD pair; a sub-step is accepted when the relative errors in R and Rdot
 *     stay below the tolerance (1e-4 in the paper).
 *
 * Readings of points the paper leaves open (error norm, controller, bin span,
 * weight normalisation, initial state) are stated where they are used.
 *
 * Parity status: every function here is pinned by tests/test_oracle_pins.py
 * against closed forms, invariants or brute force; none is "parity unpinned".
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fopenmp -fPIC -shared (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the OpenMP regions below run with (1 without OpenMP): the core count reported
 * beside the oracle's timings.  A query only; no arithmetic of the method. */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Parameters of the liquid, the gas and the stepper.                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    double rho;      /* liquid density */
    double c;        /* liquid sound speed; INFINITY -> incompressible limit */
    double mu;       /* liquid viscosity mu_l */
    double sigma;    /* surface tension */
    double p0;       /* ambient (equilibrium) pressure */
    double gamma;    /* polytropic exponent of the gas */
    double pv;       /* vapour pressure (constant) */
    int32_t gas_mode;     /* 0: polytropic gas in equilibrium at p0; 1: empty cavity (p_b = p_v) */
    int32_t max_attempts; /* bound on sub-step attempts per bin per call */
    double tol;      /* acceptance tolerance of the embedded error (Sec. 3: 1e-4) */
    double v_floor;  /* floor of the Rdot scale in the relative error norm */
} orc_params;

/* Status bits per bin (OR-ed over one call). */
#define ORC_FLAG_STEP_LIMIT 1u  /* attempts exhausted before the flow step was covered */
#define ORC_FLAG_NONFINITE  2u  /* non-finite input or state */
#define ORC_FLAG_SUPERSONIC 4u  /* |Rdot| >= c after the call */
#define ORC_FLAG_NONPOS     8u  /* R <= 0 after the call */

/* ------------------------------------------------------------------------ */
/* a1. Lognormal bins with Simpson weights (Sec. 2.2).                       */
/* ------------------------------------------------------------------------ */
/*
 * The equilibrium radius R0 is lognormal with median R0ref and shape s:
 * phi = ln(R0/R0ref) ~ N(0, s^2).  The phi axis is cut to [-K s, +K s] and
 * sampled at B equally spaced nodes (B odd).  Composite Simpson coefficients
 * 1,4,2,4,...,4,1 (times dphi/3) multiply the normal density; the weights are
 * normalised to sum to one, so n_b is the number density of all bins together
 * (reading: normalisation over the truncated span).  B = 1 is the monodisperse
 * case: R0 = R0ref, w = 1.
 * Returns 0, or -1 for an invalid request.
 */
int orc_bins(int32_t B, double R0ref, double s, double K, double *R0, double *w)
{
    if (B == 1) {
        R0[0] = R0ref;
        w[0] = 1.0;
        return 0;
    }
    if (B < 3 || (B % 2) == 0 || !(s > 0.0) || !(K > 0.0) || !(R0ref > 0.0))
        return -1;
    double dphi = 2.0 * K * s / (double)(B - 1);
    double total = 0.0;
    for (int32_t i = 0; i < B; ++i) {
        double phi = -K * s + (double)i * dphi;
        double simpson;
        if (i == 0 || i == B - 1)
            simpson = 1.0;
        else if (i % 2 == 1)
            simpson = 4.0;
        else
            simpson = 2.0;
        simpson *= dphi / 3.0;
        double density = exp(-0.5 * phi * phi / (s * s)) / (s * sqrt(2.0 * M_PI));
        R0[i] = R0ref * exp(phi);
        w[i] = simpson * density;
        total += w[i];
    }
    for (int32_t i = 0; i < B; ++i)
        w[i] = w[i] / total;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* a3. Keller-Miksis right-hand side, Eq. (keller_miksis).                   */
/* ------------------------------------------------------------------------ */
/*
 * State y = (R, Rdot).  Bin constant R0, cell pressure p_inf.
 *   p_g0  = p0 + 2 sigma/R0 - p_v                    (gas in equilibrium at p0)
 *   p_b   = p_v + p_g0 (R0/R)^(3 gamma)              (Ando's ODE, no transfer)
 *   dp_b  = -3 gamma (p_b - p_v) Rdot / R
 *   p_bw  = p_b - 4 mu Rdot/R - 2 sigma/R
 *   d/dt p_bw = dp_b + 4 mu Rdot^2/R^2 - 4 mu Rddot/R + 2 sigma Rdot/R^2
 * The Rddot inside d/dt p_bw is kept and the equation, linear in Rddot, is
 * solved exactly (reading):
 *   Rddot [R (1 - Rdot/c) + 4 mu/(rho c)] =
 *        (p_bw - p_inf)/rho (1 + Rdot/c) + R/(rho c) (d/dt p_bw without the Rddot term)
 *        - 3/2 Rdot^2 (1 - Rdot/(3c)).
 * With 1/c = 0 this is the Rayleigh-Plesset equation.
 * Writes f = (Rdot, Rddot) and, if pbw_out is not NULL, p_bw.
 */
void orc_rhs(const orc_params *P, double R0, double p_inf, const double y[2],
             double f[2], double *pbw_out)
{
    double R = y[0];
    double Rdot = y[1];
    double inv_c = 1.0 / P->c;
    double p_b, dp_b;
    if (P->gas_mode == 0) {
        double p_g0 = P->p0 + 2.0 * P->sigma / R0 - P->pv;
        double p_gas = p_g0 * pow(R0 / R, 3.0 * P->gamma);
        p_b = P->pv + p_gas;
        dp_b = -3.0 * P->gamma * p_gas * Rdot / R;
    } else {
        p_b = P->pv;
        dp_b = 0.0;
    }
    double p_bw = p_b - 4.0 * P->mu * Rdot / R - 2.0 * P->sigma / R;
    double dp_bw_explicit = dp_b + 4.0 * P->mu * Rdot * Rdot / (R * R)
                          + 2.0 * P->sigma * Rdot / (R * R);
    double rhs = (p_bw - p_inf) / P->rho * (1.0 + Rdot * inv_c)
               + R * inv_c / P->rho * dp_bw_explicit
               - 1.5 * Rdot * Rdot * (1.0 - Rdot * inv_c / 3.0);
    double lhs_coef = R * (1.0 - Rdot * inv_c) + 4.0 * P->mu * inv_c / P->rho;
    f[0] = Rdot;
    f[1] = rhs / lhs_coef;
    if (pbw_out)
        *pbw_out = p_bw;
}

/* ------------------------------------------------------------------------ */
/* a4. One SSP-RK3 trial with the embedded SSP-RK2 (Sec. 3).                 */
/* ------------------------------------------------------------------------ */
/* A right-hand side with its context, so the same stepper can be checked on
 * a linear ODE with a known solution. */
typedef void (*orc_rhs_fn)(const void *ctx, const double y[2], double f[2]);

typedef struct {
    const orc_params *P;
    double R0;
    double p_inf;
} km_ctx;

static void km_rhs_fn(const void *ctx, const double y[2], double f[2])
{
    const km_ctx *k = (const km_ctx *)ctx;
    orc_rhs(k->P, k->R0, k->p_inf, y, f, NULL);
}

/*
 * Shu-Osher form of the third-order TVD Runge-Kutta scheme (Gottlieb & Shu):
 *   y1 = y + h f(y)
 *   y2 = 3/4 y + 1/4 (y1 + h f(y1))
 *   y3 = 1/3 y + 2/3 (y2 + h f(y2))
 * The second-order TVD scheme (Heun) shares the first two evaluations:
 *   z  = 1/2 y + 1/2 (y1 + h f(y1)).
 * Writes y3 (third order), z (second order) and the stage radii y1[0], y2[0].
 */
void orc_ssprk3_trial(orc_rhs_fn fn, const void *ctx, const double y[2], double h,
                      double y3[2], double z[2], double stage_R[2])
{
    double f[2], y1[2], y2[2];
    fn(ctx, y, f);
    for (int k = 0; k < 2; ++k)
        y1[k] = y[k] + h * f[k];
    fn(ctx, y1, f);
    for (int k = 0; k < 2; ++k) {
        z[k] = 0.5 * y[k] + 0.5 * (y1[k] + h * f[k]);
        y2[k] = 0.75 * y[k] + 0.25 * (y1[k] + h * f[k]);
    }
    fn(ctx, y2, f);
    for (int k = 0; k < 2; ++k)
        y3[k] = y[k] / 3.0 + 2.0 / 3.0 * (y2[k] + h * f[k]);
    stage_R[0] = y1[0];
    stage_R[1] = y2[0];
}

/*
 * Relative error of the trial (reading of "relative errors in R and Rdot"):
 *   err = max(|R3 - R2| / |R3|, |V3 - V2| / max(|V3|, v_floor)).
 * The floor keeps the Rdot term defined at Rdot = 0.
 */
double orc_error_norm(const double y3[2], const double z[2], double v_floor)
{
    double eR = fabs(y3[0] - z[0]) / fabs(y3[0]);
    double vscale = fabs(y3[1]);
    if (vscale < v_floor)
        vscale = v_floor;
    double eV = fabs(y3[1] - z[1]) / vscale;
    return eR > eV ? eR : eV;
}

/*
 * Step-size factor after a trial with error err (reading):
 *   fac = clamp(0.9 (tol/err)^(1/3), 0.2, 5),
 * the exponent 1/3 because err measures the local error of the second-order
 * member, O(h^3).  err = 0 gives the upper clamp; a non-finite err gives 0.2.
 */
double orc_step_factor(double err, double tol)
{
    if (!(err == err) || isinf(err))
        return 0.2;
    if (err == 0.0)
        return 5.0;
    double fac = 0.9 * cbrt(tol / err);
    if (fac < 0.2)
        fac = 0.2;
    if (fac > 5.0)
        fac = 5.0;
    return fac;
}

/*
 * Adaptive advance of one bin over the flow (sub-)step dt with the carried
 * step proposal *h (stored in FP32 between calls).  Reading of the controller:
 *   - h starts as min(h_carried, dt); a non-positive or non-finite carried h means dt;
 *   - h_try = min(h, dt - t); when h >= dt - t the trial is the last one and
 *     lands exactly on dt (t is not accumulated for it);
 *   - a trial is accepted iff err <= tol and R stays positive at every stage;
 *   - accepted: t += h_try, the proposal becomes h_try * fac; on the last trial
 *     the carried proposal is h_try * fac, except when h_try had been clipped to
 *     land on dt and fac >= 1, where the unclipped h is kept;
 *   - rejected: h = h_try * fac (fac < 1) and the trial is repeated;
 *   - more than max_attempts trials: ORC_FLAG_STEP_LIMIT, the bin keeps its last
 *     accepted state.
 * Returns the flags; *n_attempts gets the number of trials.
 */
static uint32_t advance_adaptive(orc_rhs_fn fn, const void *ctx, double y[2],
                                 float *h_carry, double dt, double tol, double v_floor,
                                 int32_t max_attempts, int32_t *n_attempts)
{
    double h = (double)(*h_carry);
    if (!(h > 0.0) || isinf(h) || h > dt)
        h = dt;
    double t = 0.0;
    int32_t attempts = 0;
    uint32_t flags = 0;
    for (;;) {
        if (attempts >= max_attempts) {
            flags |= ORC_FLAG_STEP_LIMIT;
            break;
        }
        double remaining = dt - t;
        int last = (h >= remaining);
        double h_try = last ? remaining : h;
        double y3[2], z[2], stage_R[2];
        orc_ssprk3_trial(fn, ctx, y, h_try, y3, z, stage_R);
        ++attempts;
        double err = orc_error_norm(y3, z, v_floor);
        int positive = stage_R[0] > 0.0 && stage_R[1] > 0.0 && y3[0] > 0.0;
        double fac = orc_step_factor(err, tol);
        if (err <= tol && positive) {
            y[0] = y3[0];
            y[1] = y3[1];
            if (last) {
                int clipped = remaining < h;
                h = (clipped && fac >= 1.0) ? h : h_try * fac;
                break;
            }
            t += h_try;
            h = h_try * fac;
        } else {
            if (!positive && fac > 0.2)
                fac = 0.2;
            h = h_try * fac;
        }
    }
    *h_carry = (float)h;
    *n_attempts = attempts;
    return flags;
}

/* Fixed mode: n equal SSP-RK3 sub-steps of dt/n, no error estimate. */
static void advance_fixed(orc_rhs_fn fn, const void *ctx, double y[2], double dt, int32_t n)
{
    double h = dt / (double)n;
    for (int32_t i = 0; i < n; ++i) {
        double y3[2], z[2], stage_R[2];
        orc_ssprk3_trial(fn, ctx, y, h, y3, z, stage_R);
        y[0] = y3[0];
        y[1] = y3[1];
    }
}

/* ------------------------------------------------------------------------ */
/* a2-a5, a7. Advance every (cell, bin) pair over one flow step.             */
/* ------------------------------------------------------------------------ */
/*
 * Layout: R, Rdot, h, flags and attempts are [B][C] (bin-major); p_inf is [C];
 * R0 is [B].  p_inf is held constant over the call (the carrier is frozen
 * during the bubble half of the Strang split, Sec. 3).
 * n_fixed > 0 selects fixed mode with n_fixed sub-steps; n_fixed == 0 is adaptive.
 * flags and attempts may be NULL.  Cells are independent (no atomics, Sec. 4),
 * so the loop over cells runs with OpenMP.
 */
void orc_step(const orc_params *P, int64_t C, int32_t B, const double *R0,
              const double *p_inf, double dt, int32_t n_fixed,
              double *R, double *Rdot, float *h, uint32_t *flags, int32_t *attempts)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < C; ++c) {
        for (int32_t b = 0; b < B; ++b) {
            size_t k = (size_t)b * (size_t)C + (size_t)c;
            uint32_t fl = 0;
            int32_t na = 0;
            double y[2] = {R[k], Rdot[k]};
            if (!isfinite(p_inf[c]) || !isfinite(y[0]) || !isfinite(y[1])) {
                fl |= ORC_FLAG_NONFINITE;
            } else {
                km_ctx ctx = {P, R0[b], p_inf[c]};
                if (n_fixed > 0) {
                    advance_fixed(km_rhs_fn, &ctx, y, dt, n_fixed);
                    na = n_fixed;
                } else {
                    fl |= advance_adaptive(km_rhs_fn, &ctx, y, &h[k], dt, P->tol,
                                           P->v_floor, P->max_attempts, &na);
                }
                if (!isfinite(y[0]) || !isfinite(y[1]))
                    fl |= ORC_FLAG_NONFINITE;
                else if (!(y[0] > 0.0))
                    fl |= ORC_FLAG_NONPOS;
                if (fabs(y[1]) >= P->c)
                    fl |= ORC_FLAG_SUPERSONIC;
                R[k] = y[0];
                Rdot[k] = y[1];
            }
            if (flags)
                flags[k] = fl;
            if (attempts)
                attempts[k] = na;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* a6. Quadrature moments per cell (Eqs. e:ndf, e:alpha, e:pressure).        */
/* ------------------------------------------------------------------------ */
/*
 * Plain left-to-right FP64 sums over the bins i = 1..B of each cell:
 *   M3 = sum w R^3, M2V = sum w R^2 Rdot, M3P = sum w R^3 p_bw, M3V2 = sum w R^3 Rdot^2.
 * out is [7][C]:
 *   0: n_b                       (input, constant over the source step)
 *   1: alpha = 4/3 pi n_b M3      (Eq. e:ndf)
 *   2: <R^3> = M3
 *   3: <R^2 Rdot> = M2V
 *   4: 3 alpha <R^2 Rdot>/<R^3>   (source of Eq. e:alpha)
 *   5: <R^3 p_bw>/<R^3>           (Eq. e:pressure)
 *   6: <R^3 Rdot^2>/<R^3>         (Eq. e:pressure)
 * p_bw comes from the Keller-Miksis wall-pressure definition (p_inf does not
 * enter it).  alpha_ld, if not NULL, receives alpha summed in long double,
 * which the tests use to judge a compensated FP64 sum.
 */
void orc_moments(const orc_params *P, int64_t C, int32_t B, const double *R0,
                 const double *w, const double *n_b, const double *R, const double *Rdot,
                 double *out, long double *alpha_ld)
{
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < C; ++c) {
        double M3 = 0.0, M2V = 0.0, M3P = 0.0, M3V2 = 0.0;
        long double M3_ld = 0.0L;
        for (int32_t b = 0; b < B; ++b) {
            size_t k = (size_t)b * (size_t)C + (size_t)c;
            double y[2] = {R[k], Rdot[k]};
            double f[2], p_bw;
            orc_rhs(P, R0[b], P->p0, y, f, &p_bw);
            double r = y[0];
            double v = y[1];
            double r3 = r * r * r;
            M3 += w[b] * r3;
            M2V += w[b] * r * r * v;
            M3P += w[b] * r3 * p_bw;
            M3V2 += w[b] * r3 * v * v;
            M3_ld += (long double)w[b] * (long double)r * (long double)r * (long double)r;
        }
        double alpha = 4.0 / 3.0 * M_PI * n_b[c] * M3;
        out[0 * C + c] = n_b[c];
        out[1 * C + c] = alpha;
        out[2 * C + c] = M3;
        out[3 * C + c] = M2V;
        out[4 * C + c] = 3.0 * alpha * M2V / M3;
        out[5 * C + c] = M3P / M3;
        out[6 * C + c] = M3V2 / M3;
        if (alpha_ld)
            alpha_ld[c] = 4.0L / 3.0L * (long double)M_PI * (long double)n_b[c] * M3_ld;
    }
}

/* ------------------------------------------------------------------------ */
/* Hooks for the pins: the same stepper on a linear ODE y' = A y.            */
/* ------------------------------------------------------------------------ */
typedef struct {
    double a[4];
} lin_ctx;

static void lin_rhs_fn(const void *ctx, const double y[2], double f[2])
{
    const lin_ctx *L = (const lin_ctx *)ctx;
    f[0] = L->a[0] * y[0] + L->a[1] * y[1];
    f[1] = L->a[2] * y[0] + L->a[3] * y[1];
}

/* One trial of the stepper on y' = A y (A row-major 2x2). */
void orc_linear_trial(const double A[4], const double y[2], double h, double y3[2], double z[2])
{
    lin_ctx L = {{A[0], A[1], A[2], A[3]}};
    double stage_R[2];
    orc_ssprk3_trial(lin_rhs_fn, &L, y, h, y3, z, stage_R);
}

/* The adaptive driver on y' = A y over dt; returns flags, writes attempts. */
uint32_t orc_linear_advance(const double A[4], double y[2], float *h, double dt,
                            double tol, double v_floor, int32_t max_attempts,
                            int32_t *n_attempts)
{
    lin_ctx L = {{A[0], A[1], A[2], A[3]}};
    return advance_adaptive(lin_rhs_fn, &L, y, h, dt, tol, v_floor, max_attempts, n_attempts);
}

/* ------------------------------------------------------------------------ */
/* Carrier-facing forms (Sec. 2.2, Listing 2): conservative bubble variables */
/* ------------------------------------------------------------------------ */
/*
 * The transported bubble variables are n_b phi (Eq. for d(n_b phi)/dt), stored
 * per bin as qR_i = n_b R_i and qV_i = n_b Rdot_i (Listing 2 writes nbub*R).
 * Primitive -> conservative is that product.  Conservative -> primitive needs
 * n_b: from alpha = 4/3 pi n_b sum w R^3 (Eq. e:ndf) with R_i = qR_i / n_b,
 *   alpha = 4/3 pi sum w qR^3 / n_b^2  =>  n_b = sqrt(4/3 pi sum w qR^3 / alpha).
 * Layout [B][C]; alpha, n_b per cell [C].
 */
void orc_cons_from_prim(int64_t C, int32_t B, const double *n_b, const double *R,
                        const double *Rdot, double *qR, double *qV)
{
    for (int32_t b = 0; b < B; ++b)
        for (int64_t c = 0; c < C; ++c) {
            size_t k = (size_t)b * (size_t)C + (size_t)c;
            qR[k] = n_b[c] * R[k];
            qV[k] = n_b[c] * Rdot[k];
        }
}

void orc_prim_from_cons(int64_t C, int32_t B, const double *w, const double *alpha,
                        const double *qR, const double *qV, double *R, double *Rdot, double *n_b)
{
    for (int64_t c = 0; c < C; ++c) {
        double s = 0.0;
        for (int32_t b = 0; b < B; ++b) {
            double q = qR[(size_t)b * (size_t)C + (size_t)c];
            s += w[b] * q * q * q;
        }
        double nb = sqrt(4.0 / 3.0 * M_PI * s / alpha[c]);
        n_b[c] = nb;
        for (int32_t b = 0; b < B; ++b) {
            size_t k = (size_t)b * (size_t)C + (size_t)c;
            R[k] = qR[k] / nb;
            Rdot[k] = qV[k] / nb;
        }
    }
}

/*
 * Mixture pressure, Eq. (e:pressure):
 *   p = (1 - alpha) p_l + alpha (<R^3 p_bw>/<R^3> - rho <R^3 Rdot^2>/<R^3>),
 * with alpha and the two ratios taken from the moments rows 1, 5 and 6 and rho
 * the liquid density (rho_l per cell, or rho_default when rho_l is NULL).
 * moments is [7][C].
 */
void orc_mixture_pressure(int64_t C, const double *moments, const double *p_l, const double *rho_l,
                          double rho_default, double *p)
{
    for (int64_t c = 0; c < C; ++c) {
        double alpha = moments[1 * C + c];
        double rho = rho_l ? rho_l[c] : rho_default;
        p[c] = (1.0 - alpha) * p_l[c] + alpha * (moments[5 * C + c] - rho * moments[6 * C + c]);
    }
}

/* Stiffened-gas liquid pressure, Eq. (eos_liquid): p_l = (gamma_l - 1) rho_l e_l - gamma_l pi_inf. */
void orc_stiffened_gas(int64_t n, const double *rho_l, const double *e_l, double gamma_l,
                       double pi_inf, double *p_l)
{
    for (int64_t i = 0; i < n; ++i)
        p_l[i] = (gamma_l - 1.0) * rho_l[i] * e_l[i] - gamma_l * pi_inf;
}

/* ------------------------------------------------------------------------ */
/* Volume-averaged (Euler-Lagrange) model, Sec. 2.1                          */
/* ------------------------------------------------------------------------ */
/*
 * N bubbles at fixed positions x_n (no translation, Sec. 2.1) on a grid of
 * nx x ny x nz cells of size dx (cell (i,j,k) centred at ((i+1/2)dx, ...),
 * x fastest in memory).  Each bubble has its own R0_n; its far-field pressure
 * is the carrier pressure of the cell that contains it (reading), held fixed
 * over the step.  The bubble ODE is the same Keller-Miksis equation, advanced
 * by the same adaptive stepper as one bin.  bub_p_cell holds the cell index of
 * every bubble (-1 outside the grid).
 */
void orc_el_advance(const orc_params *P, int64_t N, const double *R0, const int64_t *cell,
                    const double *p_cell, double dt, double *R, double *Rdot, float *h,
                    uint32_t *flags, int32_t *attempts)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t n = 0; n < N; ++n) {
        uint32_t fl = 0;
        int32_t na = 0;
        double y[2] = {R[n], Rdot[n]};
        double p_inf = cell[n] >= 0 ? p_cell[cell[n]] : NAN;
        if (!isfinite(p_inf) || !isfinite(y[0]) || !isfinite(y[1])) {
            fl |= ORC_FLAG_NONFINITE;
        } else {
            km_ctx ctx = {P, R0[n], p_inf};
            fl |= advance_adaptive(km_rhs_fn, &ctx, y, &h[n], dt, P->tol, P->v_floor,
                                   P->max_attempts, &na);
            if (!isfinite(y[0]) || !isfinite(y[1]))
                fl |= ORC_FLAG_NONFINITE;
            else if (!(y[0] > 0.0))
                fl |= ORC_FLAG_NONPOS;
            R[n] = y[0];
            Rdot[n] = y[1];
        }
        if (flags)
            flags[n] = fl;
        if (attempts)
            attempts[n] = na;
    }
}

/*
 * Smearing of the bubbles into the Eulerian void fraction, Eq. (kernel3D):
 *   alpha(x) = sum_n V_n delta(d_n, h_n),   V_n = 4/3 pi R_n^3,
 *   delta(d, h) = exp(-d^2 / (2 h^2)) / (h^3 (2 pi)^{3/2})  for d/h < 3, else 0,
 * with d_n the distance from the cell centre to the bubble and the kernel width
 * h_n = dx when R_n < dx and R_n otherwise (Eq. model_inequality and the rule
 * after it).  The kernel is evaluated at cell centres (Listing 1).  The rate
 *   alpha_dot(x) = sum_n (dV_n/dt) delta(d_n, h_n),  dV_n/dt = 4 pi R_n^2 Rdot_n,
 * is the first term of the d alpha/dt equation; the second, V_n d delta/dt =
 * -V_n u . grad delta, vanishes for fixed bubbles in a liquid at rest and is
 * left to the carrier.  Cells outside the grid are skipped.  Plain loops over
 * bubbles and over every cell of the grid whose centre lies within 3 h_n.
 * alpha_dot may be NULL.
 */
void orc_el_smear(int64_t N, const double *x, const double *y, const double *z, const double *R,
                  const double *Rdot, int32_t nx, int32_t ny, int32_t nz, double dx,
                  double *alpha, double *alpha_dot)
{
    int64_t ncell = (int64_t)nx * ny * nz;
    for (int64_t c = 0; c < ncell; ++c) {
        alpha[c] = 0.0;
        if (alpha_dot)
            alpha_dot[c] = 0.0;
    }
    double norm = pow(2.0 * M_PI, 1.5);
    for (int64_t n = 0; n < N; ++n) {
        double h = R[n] < dx ? dx : R[n];
        double V = 4.0 / 3.0 * M_PI * R[n] * R[n] * R[n];
        double Vdot = 4.0 * M_PI * R[n] * R[n] * Rdot[n];
        for (int32_t k = 0; k < nz; ++k)
            for (int32_t j = 0; j < ny; ++j)
                for (int32_t i = 0; i < nx; ++i) {
                    double cx = (i + 0.5) * dx - x[n];
                    double cy = (j + 0.5) * dx - y[n];
                    double cz = (k + 0.5) * dx - z[n];
                    double d = sqrt(cx * cx + cy * cy + cz * cz);
                    if (!(d / h < 3.0))
                        continue;
                    double delta = exp(-d * d / (2.0 * h * h)) / (h * h * h * norm);
                    int64_t c = ((int64_t)k * ny + j) * nx + i;
                    alpha[c] += V * delta;
                    if (alpha_dot)
                        alpha_dot[c] += Vdot * delta;
                }
    }
}

/* ------------------------------------------------------------------------ */
/* Non-polytropic bubble contents (Sec. 2): gas and vapour with heat and     */
/* mass transfer at the wall, reduced-order form with constant transfer      */
/* coefficients.                                                              */
/* ------------------------------------------------------------------------ */
/*
 * The bubble holds a fixed mass m_g of non-condensable gas (gas constant R_g)
 * and a vapour mass m_v (gas constant R_v); its pressure p_b is a state. The
 * state per bin is y = (R, Rdot, p_b, m_v). The paper fixes:
 *   - Eq. (keller_miksis) with p_bw = p_b - 4 mu Rdot/R - 2 sigma/R;
 *   - Eq. (massVaporRate): mdot_v = D rho_bw / (1 - chi_vw) dchi_v/dr|_R;
 *   - Ando's pressure equation:
 *       dp_b/dt = (3 gamma_b / R) (-Rdot p_b + R_v T_bw mdot_v
 *                                  + (gamma_b - 1)/gamma_b k_bw dT/dr|_R).
 * Readings of what the paper leaves to the cited reduced-order model:
 *   - the wall gradients are constant coefficients times the difference
 *     between wall and bubble mean over R:
 *       dchi_v/dr|_R = beta_c (chi_vw - chi_mean) / R,
 *       dT/dr|_R     = beta_T (T_w - T_mean) / R;
 *   - the wall stays at the liquid temperature T_w (T_bw = T_w) and the vapour
 *     there is saturated at p_v (the handle's vapour pressure);
 *   - T_mean from the ideal-gas mixture: p_b V = (m_g R_g + m_v R_v) T_mean,
 *     V = 4/3 pi R^3; chi_mean = m_v / (m_v + m_g);
 *   - wall vapour mass fraction and density from the partial pressures p_v and
 *     p_b - p_v at T_w: chi_vw = (p_v/R_v) / (p_v/R_v + (p_b - p_v)/R_g),
 *     rho_bw = (p_v/R_v + (p_b - p_v)/R_g) / T_w;
 *   - mdot_v is a flux per unit wall area: dm_v/dt = 4 pi R^2 mdot_v;
 *   - gamma_b is the handle's gamma; m_g follows from equilibrium at R0:
 *     m_g = (p0 + 2 sigma/R0 - p_v) (4/3 pi R0^3) / (R_g T_w);
 *   - the error norm stays the one of R and Rdot (Sec. 3 names those two).
 * With beta_T = beta_c = 0 the pressure equation reduces to
 * dp_b/dt = -3 gamma_b Rdot p_b / R, whose solution is the polytropic law.
 */
typedef struct {
    double R_g, R_v;     /* gas constants of the gas and of the vapour */
    double T_w;          /* wall (liquid) temperature */
    double k_bw;         /* thermal conductivity of the contents at the wall */
    double D;            /* binary diffusion coefficient of vapour in gas */
    double beta_T;       /* heat transfer coefficient (dimensionless) */
    double beta_c;       /* mass transfer coefficient (dimensionless) */
} orc_transfer;

/* Gas mass of a bubble of equilibrium radius R0. */
double orc_transfer_gas_mass(const orc_params *P, const orc_transfer *T, double R0)
{
    double V0 = 4.0 / 3.0 * M_PI * R0 * R0 * R0;
    return (P->p0 + 2.0 * P->sigma / R0 - P->pv) * V0 / (T->R_g * T->T_w);
}

/* Equilibrium state of bin R0: R = R0, Rdot = 0, p_b = p0 + 2 sigma/R0,
 * m_v = p_v V0 / (R_v T_w) (saturated vapour at the wall temperature). */
void orc_transfer_init(const orc_params *P, const orc_transfer *T, double R0, double y[4])
{
    double V0 = 4.0 / 3.0 * M_PI * R0 * R0 * R0;
    y[0] = R0;
    y[1] = 0.0;
    y[2] = P->p0 + 2.0 * P->sigma / R0;
    y[3] = P->pv * V0 / (T->R_v * T->T_w);
}

/* dp_b/dt and dm_v/dt at (R, Rdot, p_b, m_v) for the gas mass m_g. */
void orc_transfer_rates(const orc_params *P, const orc_transfer *T, double m_g,
                        const double y[4], double *dpb, double *dmv)
{
    double R = y[0], Rdot = y[1], p_b = y[2], m_v = y[3];
    double V = 4.0 / 3.0 * M_PI * R * R * R;
    double T_mean = p_b * V / (m_g * T->R_g + m_v * T->R_v);
    double chi_mean = m_v / (m_v + m_g);
    double rho_v_w = P->pv / (T->R_v * T->T_w);
    double rho_g_w = (p_b - P->pv) / (T->R_g * T->T_w);
    double rho_bw = rho_v_w + rho_g_w;
    double chi_vw = rho_v_w / rho_bw;
    double dchi_dr = T->beta_c * (chi_vw - chi_mean) / R;
    double dT_dr = T->beta_T * (T->T_w - T_mean) / R;
    double mdot_v = T->D * rho_bw / (1.0 - chi_vw) * dchi_dr;
    double gb = P->gamma;
    *dpb = 3.0 * gb / R * (-Rdot * p_b + T->R_v * T->T_w * mdot_v + (gb - 1.0) / gb * T->k_bw * dT_dr);
    *dmv = 4.0 * M_PI * R * R * mdot_v;
}

/* Keller-Miksis (Eq. keller_miksis) with the bubble pressure as a state: the
 * wall-pressure rate dp_bw/dt = dp_b/dt + 4 mu Rdot^2/R^2 + 2 sigma Rdot/R^2
 * - 4 mu Rddot/R, whose Rddot term moves to the left-hand side. */
void orc_transfer_rhs(const orc_params *P, const orc_transfer *T, double m_g, double p_inf,
                      const double y[4], double f[4], double *pbw_out)
{
    double R = y[0], Rdot = y[1], p_b = y[2];
    double inv_c = 1.0 / P->c;
    double dpb, dmv;
    orc_transfer_rates(P, T, m_g, y, &dpb, &dmv);
    double p_bw = p_b - 4.0 * P->mu * Rdot / R - 2.0 * P->sigma / R;
    double dp_bw_explicit = dpb + 4.0 * P->mu * Rdot * Rdot / (R * R)
                          + 2.0 * P->sigma * Rdot / (R * R);
    double rhs = (p_bw - p_inf) / P->rho * (1.0 + Rdot * inv_c)
               + R * inv_c / P->rho * dp_bw_explicit
               - 1.5 * Rdot * Rdot * (1.0 - Rdot * inv_c / 3.0);
    double lhs_coef = R * (1.0 - Rdot * inv_c) + 4.0 * P->mu * inv_c / P->rho;
    f[0] = Rdot;
    f[1] = rhs / lhs_coef;
    f[2] = dpb;
    f[3] = dmv;
    if (pbw_out)
        *pbw_out = p_bw;
}

/* The SSP-RK3 trial with the embedded Heun member (as orc_ssprk3_trial), on
 * the four components. */
static void transfer_trial(const orc_params *P, const orc_transfer *T, double m_g, double p_inf,
                           const double y[4], double h, double y3[4], double z[4],
                           double stage_R[2])
{
    double f[4], y1[4], y2[4];
    orc_transfer_rhs(P, T, m_g, p_inf, y, f, NULL);
    for (int k = 0; k < 4; ++k)
        y1[k] = y[k] + h * f[k];
    orc_transfer_rhs(P, T, m_g, p_inf, y1, f, NULL);
    for (int k = 0; k < 4; ++k) {
        z[k] = 0.5 * y[k] + 0.5 * (y1[k] + h * f[k]);
        y2[k] = 0.75 * y[k] + 0.25 * (y1[k] + h * f[k]);
    }
    orc_transfer_rhs(P, T, m_g, p_inf, y2, f, NULL);
    for (int k = 0; k < 4; ++k)
        y3[k] = y[k] / 3.0 + 2.0 / 3.0 * (y2[k] + h * f[k]);
    stage_R[0] = y1[0];
    stage_R[1] = y2[0];
}

/* The adaptive controller of advance_adaptive on the four components (the
 * error norm reads R and Rdot only). */
static uint32_t transfer_advance(const orc_params *P, const orc_transfer *T, double m_g,
                                 double p_inf, double y[4], float *h_carry, double dt,
                                 int32_t n_fixed, int32_t *n_attempts)
{
    double y3[4], z[4], stage_R[2];
    if (n_fixed > 0) {
        double hf = dt / (double)n_fixed;
        for (int32_t i = 0; i < n_fixed; ++i) {
            transfer_trial(P, T, m_g, p_inf, y, hf, y3, z, stage_R);
            for (int k = 0; k < 4; ++k)
                y[k] = y3[k];
        }
        *n_attempts = n_fixed;
        return 0;
    }
    double h = (double)(*h_carry);
    if (!(h > 0.0) || isinf(h) || h > dt)
        h = dt;
    double t = 0.0;
    int32_t attempts = 0;
    uint32_t flags = 0;
    for (;;) {
        if (attempts >= P->max_attempts) {
            flags |= ORC_FLAG_STEP_LIMIT;
            break;
        }
        double remaining = dt - t;
        int last = (h >= remaining);
        double h_try = last ? remaining : h;
        transfer_trial(P, T, m_g, p_inf, y, h_try, y3, z, stage_R);
        ++attempts;
        double err = orc_error_norm(y3, z, P->v_floor);
        int positive = stage_R[0] > 0.0 && stage_R[1] > 0.0 && y3[0] > 0.0;
        double fac = orc_step_factor(err, P->tol);
        if (err <= P->tol && positive) {
            for (int k = 0; k < 4; ++k)
                y[k] = y3[k];
            if (last) {
                int clipped = remaining < h;
                h = (clipped && fac >= 1.0) ? h : h_try * fac;
                break;
            }
            t += h_try;
            h = h_try * fac;
        } else {
            if (!positive && fac > 0.2)
                fac = 0.2;
            h = h_try * fac;
        }
    }
    *h_carry = (float)h;
    *n_attempts = attempts;
    return flags;
}

/* orc_step for the transfer model: the state adds p_b and m_v ([B][C] each). */
void orc_transfer_step(const orc_params *P, const orc_transfer *T, int64_t C, int32_t B,
                       const double *R0, const double *p_inf, double dt, int32_t n_fixed,
                       double *R, double *Rdot, double *pb, double *mv, float *h,
                       uint32_t *flags, int32_t *attempts)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < C; ++c) {
        for (int32_t b = 0; b < B; ++b) {
            size_t k = (size_t)b * (size_t)C + (size_t)c;
            uint32_t fl = 0;
            int32_t na = 0;
            double y[4] = {R[k], Rdot[k], pb[k], mv[k]};
            int finite = isfinite(p_inf[c]);
            for (int i = 0; i < 4; ++i)
                finite = finite && isfinite(y[i]);
            if (!finite) {
                fl |= ORC_FLAG_NONFINITE;
            } else {
                double m_g = orc_transfer_gas_mass(P, T, R0[b]);
                fl |= transfer_advance(P, T, m_g, p_inf[c], y, &h[k], dt, n_fixed, &na);
                if (!isfinite(y[0]) || !isfinite(y[1]) || !isfinite(y[2]) || !isfinite(y[3]))
                    fl |= ORC_FLAG_NONFINITE;
                else if (!(y[0] > 0.0))
                    fl |= ORC_FLAG_NONPOS;
                if (fabs(y[1]) >= P->c)
                    fl |= ORC_FLAG_SUPERSONIC;
                R[k] = y[0];
                Rdot[k] = y[1];
                pb[k] = y[2];
                mv[k] = y[3];
            }
            if (flags)
                flags[k] = fl;
            if (attempts)
                attempts[k] = na;
        }
    }
}

/* orc_moments with p_bw = p_b - 4 mu Rdot/R - 2 sigma/R from the state p_b. */
void orc_transfer_moments(const orc_params *P, int64_t C, int32_t B, const double *w,
                          const double *n_b, const double *R, const double *Rdot,
                          const double *pb, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < C; ++c) {
        double M3 = 0.0, M2V = 0.0, M3P = 0.0, M3V2 = 0.0;
        for (int32_t b = 0; b < B; ++b) {
            size_t k = (size_t)b * (size_t)C + (size_t)c;
            double r = R[k];
            double v = Rdot[k];
            double p_bw = pb[k] - 4.0 * P->mu * v / r - 2.0 * P->sigma / r;
            double r3 = r * r * r;
            M3 += w[b] * r3;
            M2V += w[b] * r * r * v;
            M3P += w[b] * r3 * p_bw;
            M3V2 += w[b] * r3 * v * v;
        }
        double alpha = 4.0 / 3.0 * M_PI * n_b[c] * M3;
        out[0 * C + c] = n_b[c];
        out[1 * C + c] = alpha;
        out[2 * C + c] = M3;
        out[3 * C + c] = M2V;
        out[4 * C + c] = 3.0 * alpha * M2V / M3;
        out[5 * C + c] = M3P / M3;
        out[6 * C + c] = M3V2 / M3;
    }
}
