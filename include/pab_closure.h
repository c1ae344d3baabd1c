/*
 * pab_closure.h - carrier-facing forms of the bubble source update (sm_103a).
 *
 * These entry points connect a handle of pab.h to a compressible flow solver:
 *   - Strang splitting (Sec. 3): the bubble ODEs are advanced for half a flow
 *     step before and after the carrier's step;
 *   - conservative bubble variables (Sec. 2.2, Listing 2): the transported
 *     quantities are n_b R_i and n_b Rdot_i per bin, and n_b follows from the
 *     void fraction by Eq. (e:ndf);
 *   - the mixture pressure of Eq. (e:pressure) from the quadrature moments and
 *     the liquid pressure of the stiffened-gas equation of state, Eq. (eos_liquid).
 * Conventions are those of pab.h (caller-owned device pointers, bin-major
 * [Nb][C] state, [7][C] moments, stream-ordered calls, no traps).
 */
#ifndef PAB_CLOSURE_H
#define PAB_CLOSURE_H

#include <stdint.h>

#include "pab.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * One bubble half of a Strang-split flow step (Sec. 3): pab_bubble_step with
 * dt_flow / 2.  A flow step is strang_half, carrier step over dt_flow,
 * strang_half, with p_inf_dev the carrier pressure at the start (first half)
 * and at the end (second half) of the carrier step.
 * Errors: as pab_bubble_step.
 */
pab_status pab_strang_half(pab_t *h, const double *p_inf_dev, const double *nb_dev, double dt_flow,
                           double *moments_dev, void *stream);

/*
 * Conservative bubble variables of the current state (the transported n_b R_i and
 * n_b Rdot_i of Sec. 2.2 and Listing 2): qR_dev[i][c] = n_b[c] R,
 * qV_dev[i][c] = n_b[c] Rdot ([Nb][C], device).  nb_dev [C] or NULL for the
 * handle's default n_b.  Errors: PAB_EINVAL (NULL outputs), PAB_ECUDA.
 */
pab_status pab_get_conservative(pab_t *h, const double *nb_dev, double *qR_dev, double *qV_dev,
                                void *stream);

/*
 * Set the state from conservative variables and the void fraction alpha_dev
 * [C]: n_b = sqrt(4/3 pi sum_i w_i qR_i^3 / alpha) (Eq. e:ndf with R = qR/n_b),
 * then R = qR / n_b, Rdot = qV / n_b.  The cubes and the products by 1/n_b are
 * formed from the significands on the integer pipe, each within 1 ulp of the
 * FP64 result (FP64 instructions for a cell with a subnormal, infinite or NaN
 * value).  nb_out_dev [C] receives n_b (may be NULL).  A cell with alpha <= 0
 * or non-finite gets n_b = NaN and is flagged
 * PAB_FLAG_NONFINITE on its next step; the carried sub-step h is kept.
 * Errors: PAB_EINVAL (NULL inputs), PAB_ECUDA.
 */
pab_status pab_set_conservative(pab_t *h, const double *alpha_dev, const double *qR_dev,
                                const double *qV_dev, double *nb_out_dev, void *stream);

/*
 * Mixture pressure, Eq. (e:pressure), per cell:
 *   p = (1 - alpha) p_l + alpha (<R^3 p_bw>/<R^3> - rho_l <R^3 Rdot^2>/<R^3>),
 * alpha and the two ratios from rows 1, 5 and 6 of moments_dev [7][C] (as
 * written by pab_bubble_step or pab_moments), p_l_dev [C] the liquid pressure,
 * rho_l_dev [C] the liquid density or NULL for the handle's rho.
 * Errors: PAB_EINVAL (NULL moments, p_l or output), PAB_ECUDA.
 */
pab_status pab_mixture_pressure(pab_t *h, const double *moments_dev, const double *p_l_dev,
                                const double *rho_l_dev, double *p_dev, void *stream);

/*
 * Stiffened-gas liquid pressure, Eq. (eos_liquid), for n values:
 *   p_l = (gamma_l - 1) rho_l e_l - gamma_l pi_inf
 * (rho_l_dev, e_l_dev, p_l_dev: [n] FP64 device).  No handle is needed.
 * Errors: PAB_EINVAL (n < 0, NULL pointers, gamma_l <= 1), PAB_ECUDA.
 */
pab_status pab_stiffened_gas(int64_t n, const double *rho_l_dev, const double *e_l_dev,
                             double gamma_l, double pi_inf, double *p_l_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PAB_CLOSURE_H */
