/*
 * pab_el.h - the volume-averaged (Euler-Lagrange) subgrid model on sm_103a.
 *
 * Sec. 2.1 of "Hardware-Accelerated Phase-Averaging for Cavitating Bubbly
 * Flows" (arXiv 2511.21031): discrete bubbles at fixed positions, each obeying
 * the Keller-Miksis equation of pab.h under the carrier pressure of the cell
 * that contains it, and their volumes smeared into the Eulerian void fraction
 * with the truncated Gaussian kernel of Eq. (kernel3D):
 *   alpha(x) = sum_n V_n delta(d_n, h_n),  V_n = 4/3 pi R_n^3,
 *   delta(d, h) = exp(-d^2/(2 h^2)) / (h^3 (2 pi)^{3/2}) for d/h < 3, else 0,
 * with h_n = dx while R_n < dx and R_n otherwise (Eq. model_inequality and the
 * rule after it), evaluated at cell centres as Listing 1 does, and the bubble
 * growth part of its rate, alpha_dot(x) = sum_n 4 pi R_n^2 Rdot_n delta(d_n, h_n).
 *
 * Grid: nx x ny x nz cells of size dx, cell (i,j,k) centred at
 * ((i+1/2) dx, (j+1/2) dx, (k+1/2) dx), index (k ny + j) nx + i.  A bubble
 * outside the grid has no pressure: its step is skipped and flagged
 * PAB_FLAG_NONFINITE.  Conventions are those of pab.h.
 */
#ifndef PAB_EL_H
#define PAB_EL_H

#include <stdint.h>

#include "pab.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pab_el_s pab_el_t;

/*
 * Create the bubble population on the current device.  liquid: the fluid, gas
 * and stepper fields of a pab_config (rho, c, mu, sigma, p0, gamma, pv,
 * gas_mode, tol, v_floor, max_attempts; the bin and cell fields are ignored;
 * adaptive FP64 stepping).  pos_host: [3][N] positions (x row, y row, z row);
 * R0_host: [N] equilibrium radii; the bubbles start at rest at R = R0.
 * Errors: PAB_EINVAL (N < 0 or above PAB_MAX_CELLS, non-positive sizes or radii,
 * nx * ny * nz above PAB_MAX_CELLS, non-finite positions),
 * PAB_ENOMEM, PAB_ECUDA.
 */
pab_status pab_el_create(const pab_config *liquid, int64_t n_bubbles, const double *pos_host,
                         const double *R0_host, int32_t nx, int32_t ny, int32_t nz, double dx,
                         void *stream, pab_el_t **out);

/*
 * Advance every bubble over dt under p_cell_dev [nx ny nz] (device), then, if
 * alpha_dev is not NULL, write the smeared void fraction of the new state into
 * alpha_dev [nx ny nz] and, if alpha_dot_dev is not NULL, its growth rate.
 * Errors: PAB_EINVAL (NULL p_cell_dev, dt <= 0 or non-finite), PAB_ECUDA.
 */
pab_status pab_el_step(pab_el_t *e, const double *p_cell_dev, double dt, double *alpha_dev,
                       double *alpha_dot_dev, void *stream);

/* Smear the current state only (alpha_dev required, alpha_dot_dev optional).  A
 * bubble whose radius is NaN (one flagged non-finite by a step) adds nothing. */
pab_status pab_el_smear(pab_el_t *e, double *alpha_dev, double *alpha_dot_dev, void *stream);

/* Synchronise `stream`, read and reset the status as pab_status_flags does. */
pab_status pab_el_status(pab_el_t *e, uint32_t *flags, int64_t *n_flagged, int64_t *n_attempts,
                         void *stream);

/* Bubble state [N] (device buffers); h_dev may be NULL on set. */
pab_status pab_el_get_state(pab_el_t *e, double *R_dev, double *Rdot_dev, float *h_dev, void *stream);
pab_status pab_el_set_state(pab_el_t *e, const double *R_dev, const double *Rdot_dev,
                            const float *h_dev, void *stream);

void pab_el_destroy(pab_el_t *e);
const char *pab_el_last_error(const pab_el_t *e);

#ifdef __cplusplus
}
#endif

#endif /* PAB_EL_H */
