/*
 * pab_transfer.h - bubble contents with heat and mass transfer (sm_103a).
 *
 * With gas_mode = PAB_GAS_TRANSFER (pab.h) the bubble pressure p_b and the
 * vapour mass m_v are states of every (bin, cell) beside R and Rdot (Sec. 2):
 *   - Keller-Miksis, Eq. (keller_miksis), with p_bw = p_b - 4 mu Rdot/R - 2 sigma/R;
 *   - Ando's pressure equation
 *       dp_b/dt = (3 gamma/R) (-Rdot p_b + R_v T_w mdot_v + (gamma - 1)/gamma k_bw dT/dr|_R);
 *   - the vapour flux of Eq. (massVaporRate), mdot_v = D rho_bw/(1 - chi_vw) dchi/dr|_R,
 *     and dm_v/dt = 4 pi R^2 mdot_v;
 *   - constant transfer coefficients for the wall gradients (the reduced-order
 *     model the paper adopts): dchi/dr|_R = beta_c (chi_vw - chi_mean)/R and
 *     dT/dr|_R = beta_T (T_w - T_mean)/R, with T_mean from the ideal-gas mixture
 *     p_b V = (m_g R_g + m_v R_v) T_mean, chi_mean = m_v/(m_v + m_g), the wall at
 *     T_w with saturated vapour at pv, and the gas mass m_g of equilibrium at R0.
 * gamma is the handle's gamma; the error norm of the stepper stays the one of R
 * and Rdot.  A handle starts in equilibrium: R = R0, p_b = p0 + 2 sigma/R0,
 * m_v = pv (4/3 pi R0^3)/(R_v T_w) (Rdot as pab_create sets it).
 * Requirements checked by pab_create: precision PAB_FP64, 0 <= pv < p0,
 * R_g, R_v, T_w positive, k_bw, D_vg, beta_T, beta_c >= 0.  The batched,
 * allocation-free and volume-averaged entry points do not take this mode.
 * Moments (pab.h) use the state p_b in <R^3 p_bw>.  Conventions, and the
 * integer-pipe forms of the trial's products and reciprocals (within 1 ulp of
 * FP64; see precision), are those of pab.h.
 */
#ifndef PAB_TRANSFER_H
#define PAB_TRANSFER_H

#include <stdint.h>

#include "pab.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Copy the contents p_b [Nb][C] and m_v [Nb][C] (FP64, device, bin-major) out
 * of / into the handle, stream-ordered.  Either pointer may be NULL to skip it.
 * Errors: PAB_EINVAL (handle without PAB_GAS_TRANSFER), PAB_ECUDA.
 */
pab_status pab_get_contents(pab_t *h, double *pb_dev, double *mv_dev, void *stream);
pab_status pab_set_contents(pab_t *h, const double *pb_dev, const double *mv_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PAB_TRANSFER_H */
