/*
 * pab.h - C ABI of the phase-averaged bubble-dynamics library (sm_103a).
 *
 * The library advances the ensemble-averaged (Euler-Euler) bubble state of
 * "Hardware-Accelerated Phase-Averaging for Cavitating Bubbly Flows"
 * (arXiv 2511.21031) over one flow step and reduces it into the source terms
 * of the carrier equations:
 *   - every grid cell carries Nb equilibrium-radius bins R0_i drawn from a
 *     lognormal distribution with Simpson quadrature weights w_i (Sec. 2.2);
 *   - each bin's radius obeys the Keller-Miksis equation, Eq. (keller_miksis),
 *     with a polytropic gas (Ando's pressure ODE without transfer terms),
 *     surface tension, viscosity and liquid compressibility (Sec. 2);
 *   - the bins of a cell advance under that cell's pressure p_inf with
 *     adaptive third-order TVD Runge-Kutta sub-steps, accepted when the
 *     relative error against the embedded second-order member stays below a
 *     tolerance (1e-4 in the paper, Sec. 3);
 *   - the bins are reduced by the quadrature weights into n_b, the void
 *     fraction alpha = 4/3 pi n_b <R^3> (Eq. e:ndf), the alpha source
 *     3 alpha <R^2 Rdot>/<R^3> (Eq. e:alpha) and the pressure moments
 *     <R^3 p_bw>/<R^3>, <R^3 Rdot^2>/<R^3> (Eq. e:pressure).
 *
 * Conventions (all entry points):
 *   - Device pointers are caller-owned, contiguous, resident on the device
 *     that was current at pab_create, and must stay valid until the stream
 *     work that uses them has completed.  The handle owns only its state and
 *     its scratch (status counters, staging for the host entry point, and for
 *     small grids the quadrature terms of pab_create below).
 *   - State layout is bin-major structure-of-arrays: element (bin i, cell c)
 *     is at index i * n_cells + c.  Moments are [7][n_cells], row k at k * n_cells.
 *   - Calls are stream-ordered and asynchronous unless stated.  `stream` is a
 *     cudaStream_t (NULL = legacy default stream).  Device-side problems are
 *     recorded in the handle's status word and per-bin flags, never by trapping;
 *     pab_status_flags reads them.
 *   - No exceptions cross the ABI.  A handle is not thread-safe; separate
 *     handles are.  Every call returns PAB_EINVAL for a NULL handle.
 *   - On a non-OK return, pab_last_error(handle) describes the failure.
 */
#ifndef PAB_H
#define PAB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pab_s pab_t;

typedef enum {
    PAB_OK = 0,
    PAB_EINVAL = 1,        /* invalid argument or configuration; nothing launched */
    PAB_ENOMEM = 2,        /* device or host allocation failed */
    PAB_ECUDA = 3,         /* a CUDA runtime call failed */
    PAB_ESTEP_LIMIT = 4,   /* some bin exhausted max_attempts (pab_status_flags) */
    PAB_ENONFINITE = 5,    /* non-finite input or state met (pab_status_flags) */
    PAB_ESTATE = 6         /* call not valid in the handle's state */
} pab_status;

/* precision: PAB_FP64 computes every step in FP64: FP64 state and FP64
 * operations, where the plain products and reciprocals of the trial and of the
 * moment terms are formed from the 53-bit significands on the integer pipe and
 * rounded once, each within 1 ulp of the IEEE FP64 result (a trial meeting a
 * subnormal, infinite or NaN value is formed again with FP64 instructions).
 * PAB_MIXED evaluates the
 * Keller-Miksis right-hand sides in FP32, written in deviations from
 * equilibrium, and keeps in FP64 the state, the embedded error estimate and the
 * accept decision, the time bookkeeping and a compensated alpha sum; bins near
 * collapse (R < 0.2 R0 or |Rdot| > c/20) take whole FP64 trials. */
enum { PAB_FP64 = 0, PAB_MIXED = 1 };
/* stepper */
enum { PAB_ADAPTIVE = 0, PAB_FIXED = 1 };
/* gas_mode */
enum { PAB_GAS_POLYTROPIC = 0, PAB_GAS_EMPTY = 1, PAB_GAS_TRANSFER = 2 };

/* Per-bin status bits (OR-ed into the handle's status word). */
#define PAB_FLAG_STEP_LIMIT 1u   /* attempts exhausted; the bin keeps its last accepted state */
#define PAB_FLAG_NONFINITE 2u    /* non-finite pressure or state; the bin is left unchanged */
#define PAB_FLAG_SUPERSONIC 4u   /* |Rdot| >= c after the step */
#define PAB_FLAG_NONPOS 8u       /* R <= 0 after the step */

#define PAB_MAX_BINS 63
/* Largest cell count any entry point accepts (3.4e10 cells, far beyond what HBM holds at
 * any Nb): every size, index and grid product of a handle stays inside 64-bit and
 * launch limits. */
#define PAB_MAX_CELLS (1LL << 35)

/*
 * Configuration of one handle.  pab_config_default fills water (Sec. 5):
 * rho 1000, c 1500, mu 1e-3, sigma 0.072, p0 101325, gamma 1.4, pv 0; bins
 * R0ref 10e-6, s 0.3, span 5 s; adaptive FP64, tol 1e-4 (Sec. 3),
 * v_floor 1e-3 sqrt(p0/rho), max_attempts 100000; alpha0 4e-5; equilibrium start.
 */
typedef struct {
    int64_t n_cells;        /* C: 1..PAB_MAX_CELLS */
    int32_t n_bins;         /* Nb: 1, or odd 3..PAB_MAX_BINS (Simpson needs odd Nb) */
    int32_t gas_mode;       /* PAB_GAS_POLYTROPIC: p_b = pv + p_g0 (R0/R)^(3 gamma),
                               p_g0 = p0 + 2 sigma/R0 - pv; PAB_GAS_EMPTY: p_b = pv;
                               PAB_GAS_TRANSFER: p_b and the vapour mass are states with
                               heat and mass transfer at the wall (pab_transfer.h) */
    double rho, c, mu, sigma, p0, gamma, pv;   /* c = INFINITY: incompressible (RP) limit */
    double R0ref;           /* median equilibrium radius of the lognormal */
    double s_lognormal;     /* shape s of the lognormal (> 0 when Nb > 1) */
    double span_K;          /* bins cover ln(R0/R0ref) in [-K s, K s] */
    const double *R0_host;  /* optional explicit table [n_bins] (host, copied at create); */
    const double *w_host;   /*   both non-NULL overrides the lognormal table */
    int32_t precision;      /* PAB_FP64 or PAB_MIXED */
    int32_t stepper;        /* PAB_ADAPTIVE or PAB_FIXED */
    int32_t n_fixed_sub;    /* sub-steps per call in PAB_FIXED mode (>= 1) */
    int32_t max_attempts;   /* bound on trials per bin per call (>= 1) */
    double tol;             /* acceptance tolerance of the embedded error */
    double v_floor;         /* floor of the Rdot scale in the error norm; < 0: default */
    double alpha0;          /* default n_b = alpha0 / (4/3 pi sum_i w_i R0_i^3) */
    double Rdot0_ref;       /* initial Rdot_i = Rdot0_ref * R0_i / R0ref (0: rest) */
    int32_t record_attempts;/* non-zero: keep per-bin trial counts of the last call */
    int32_t block_warps;    /* warps per CTA, 1..16 (0: the default, 4); a CTA of w warps
                               owns 32 w cells (32 when a small grid is split by bins) */
    /* Contents with heat and mass transfer (gas_mode PAB_GAS_TRANSFER; FP64 only;
     * pab_transfer.h): gas constants of the gas and of the vapour, wall (liquid)
     * temperature, thermal conductivity of the contents, vapour-gas diffusion
     * coefficient, and the constant heat and mass transfer coefficients.
     * Defaults: air and water vapour at 20 C, beta_T = beta_c = 5. */
    double R_g, R_v, T_w, k_bw, D_vg, beta_T, beta_c;
} pab_config;

/* Fill *cfg with the defaults above (n_cells = 1, n_bins = 21). */
void pab_config_default(pab_config *cfg);

/*
 * Create a handle: validates cfg, builds the bin table (R0_i, w_i) in FP64 on
 * the host (Sec. 2.2; lognormal nodes equally spaced in ln R0 over +-K s,
 * composite Simpson coefficients times the normal density, normalised to sum
 * one), allocates the state R, Rdot (FP64 [Nb][C]) and the carried sub-step
 * h (FP32 [Nb][C]) on the current device, and initialises R = R0_i,
 * Rdot = Rdot0_ref R0_i/R0ref, h = 0 (first call uses dt) on `stream`.
 * An FP64 polytropic handle also holds each bin's gas factor at its radius
 * (FP64 [Nb][C]), which a step that writes moments leaves for the next step.
 * A grid of fewer 32-cell tiles than the device has SMs is stepped split by
 * bins over more CTAs; its handle also holds 4 doubles per bin-state for the
 * quadrature terms and one counter per tile (under 10 MB on 152 SMs), so that
 * the step writes the moments in one launch.
 * Errors: PAB_EINVAL (bad cfg, even Nb, NULL out), PAB_ENOMEM, PAB_ECUDA.
 */
pab_status pab_create(const pab_config *cfg, void *stream, pab_t **out);

/*
 * Advance every (cell, bin) over one flow step dt (Sec. 3; the bubble half
 * of the Strang split: p_inf is held constant over the call), then, if
 * moments_dev is not NULL, reduce the new state into moments_dev [7][C]:
 *   0 n_b, 1 alpha, 2 <R^3>, 3 <R^2 Rdot>, 4 3 alpha <R^2 Rdot>/<R^3>,
 *   5 <R^3 p_bw>/<R^3>, 6 <R^3 Rdot^2>/<R^3>.
 * p_inf_dev: [C] FP64 cell pressure (device).  nb_dev: [C] FP64 number
 * density (device) or NULL for the handle's default n_b.
 * Errors: PAB_EINVAL (NULL p_inf_dev, dt <= 0 or non-finite), PAB_ECUDA.
 * Non-finite p_inf in a cell is not an error return: its bins are left
 * unchanged and flagged PAB_FLAG_NONFINITE.
 */
pab_status pab_bubble_step(pab_t *h, const double *p_inf_dev, const double *nb_dev,
                           double dt, double *moments_dev, void *stream);

/* Reduce the current state into moments_dev [7][C] (same rows as above:
 * Eqs. e:ndf, e:alpha and e:pressure of Sec. 2.2) without advancing it.
 * nb_dev as in pab_bubble_step.  Errors: PAB_EINVAL (NULL moments_dev), PAB_ECUDA. */
pab_status pab_moments(pab_t *h, const double *nb_dev, double *moments_dev, void *stream);

/*
 * End-to-end form for host buffers: copies p_inf_host [C] (and nb_host [C]
 * when not NULL) to the device, runs pab_bubble_step, copies the moments to
 * moments_host [7][C] (when not NULL) and synchronises `stream`.  Pinned host
 * memory makes the copies asynchronous DMA.  Staging buffers are allocated on
 * first use and owned by the handle.  The step is the one of pab_bubble_step;
 * the host buffering has no counterpart in the paper.
 */
pab_status pab_bubble_step_host(pab_t *h, const double *p_inf_host, const double *nb_host,
                                double dt, double *moments_host, void *stream);

/*
 * Pipelined form of pab_bubble_step_host: enqueues the copy of p_inf_host (and
 * nb_host) to the device, the step on `stream`, and the copy of the moments
 * to moments_host, and returns without waiting.  The copies run on two streams
 * the handle owns, through two sets of device staging buffers, so the input
 * copy of one call and the output copy of the previous call overlap the
 * steps; the steps themselves stay in call order on `stream`.  At most two
 * calls are in flight: a call first waits until the call two before it has
 * finished.  A call's host buffers must stay valid and unchanged, and its
 * moments_host is not ready, until pab_host_wait returns (or until the second
 * call after it has returned).  Pinned host memory is required for overlap.
 * On an error return nothing of the failed call is still in flight.
 * Errors: as pab_bubble_step_host.
 */
pab_status pab_bubble_step_host_async(pab_t *h, const double *p_inf_host, const double *nb_host,
                                      double dt, double *moments_host, void *stream);

/* Wait until every pipelined call of the handle has finished (its moments are
 * on the host and its host buffers are free).  Errors: PAB_EINVAL, PAB_ECUDA. */
pab_status pab_host_wait(pab_t *h);

/*
 * Status of the bounded stepper (no counterpart in the paper, which describes
 * no failure handling).  Synchronise `stream`, return the status accumulated
 * since the last call and reset it: *flags = OR of per-bin PAB_FLAG_* bits, *n_flagged = number
 * of bin-steps that set any bit, *n_attempts = total trials, *n_fp64 = trials
 * taken on the FP64 path in PAB_MIXED mode.  Any output pointer may be NULL.
 * Returns PAB_ENONFINITE or PAB_ESTEP_LIMIT when those bits are set, else PAB_OK.
 */
pab_status pab_status_flags(pab_t *h, uint32_t *flags, int64_t *n_flagged, int64_t *n_attempts,
                            int64_t *n_fp64, void *stream);

/* Checkpoint / resume (no counterpart in the paper): copy the state out of /
 * into the handle (device buffers [Nb][C]; h_dev may be NULL to leave h
 * untouched on set).  A carried
 * h that is not a number in (0, dt] (NaN, zero, negative, infinite or above
 * the call's dt) makes the next call start that bin's step at dt.  On get any
 * destination may be NULL to skip it.  Errors: PAB_EINVAL (NULL handle; on set,
 * NULL R_dev or Rdot_dev), PAB_ECUDA. */
pab_status pab_get_state(pab_t *h, double *R_dev, double *Rdot_dev, float *h_dev, void *stream);
pab_status pab_set_state(pab_t *h, const double *R_dev, const double *Rdot_dev, const float *h_dev,
                         void *stream);

/* Per-bin trial counts of the last pab_bubble_step (int32 [Nb][C], device);
 * PAB_ESTATE unless the handle was created with record_attempts. */
pab_status pab_get_attempts(pab_t *h, int32_t *attempts_dev, void *stream);

/* Copy the bin table (host arrays of n_bins) and the default n_b. */
pab_status pab_get_bins(const pab_t *h, double *R0_host, double *w_host, double *nb_default);

/*
 * The bin table and default n_b that pab_create builds for cfg (Sec. 2.2:
 * lognormal R0 in Nb bins with Simpson weights, or the explicit table; n_b =
 * alpha0 / (4/3 pi sum_i w_i R0_i^3), Eq. e:ndf at equilibrium), computed on
 * the host with no handle and no device.  R0_host and w_host receive n_bins
 * values each; nb_default may be NULL.  The values are those pab_get_bins
 * returns for a handle of the same cfg.
 * Errors: PAB_EINVAL (NULL cfg or outputs, cfg refused as pab_create refuses it).
 */
pab_status pab_bin_table(const pab_config *cfg, double *R0_host, double *w_host, double *nb_default);

/* Launch shape: warps per CTA (1..16).  A CTA of w warps owns 32 w cells and
 * its warps take the (bin, cell) items of those cells from one shared pool;
 * the results are the same bits for every value.  Used by the autotuner. */
pab_status pab_set_block_warps(pab_t *h, int32_t block_warps);

/*
 * Allocation-free form of pab_bubble_step.  The paper has no counterpart of
 * this entry point; it exists for callers that may not allocate device memory
 * themselves or have a library allocate behind their back: a flow solver that
 * owns every byte of the GPU through its own pre-sized pools (its memory
 * budget is fixed, and a cudaMalloc from a library would break it or fail on a
 * full device), or a plugin that receives device pointers from a host
 * framework's allocator and must return them untouched in count and size.
 *
 * There is no handle: the caller passes the configuration and owns the whole
 * state.  cfg is validated exactly as in pab_create (record_attempts and
 * block_warps = 0 are ignored; the default warps per CTA then).  The bin table is the one
 * pab_create builds from cfg (R0_i = R0ref exp(-K s + i 2 K s/(Nb-1)) for Nb > 1).
 * R_dev, Rdot_dev: FP64 [Nb][C] state, advanced in place (device).
 * h_dev: FP32 [Nb][C] carried sub-step, in place (device; 0 before the first
 *   call; may be NULL in PAB_FIXED mode only).
 * p_inf_dev, nb_dev, dt, moments_dev: as in pab_bubble_step.
 * status_dev: NULL, or 4 int64 on the device receiving, stream-ordered,
 *   {flags, n_flagged, n_attempts, n_fp64} of this call (see pab_status_flags).
 *
 * The only scratch is one status block kept in a static device array of
 * PAB_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the library holds
 * until the process exits.  The block does not grow with the problem, so the
 * only sizes refused (PAB_EINVAL, nothing launched) are those the kernel
 * cannot take: n_bins outside 1..PAB_MAX_BINS (odd), n_cells outside
 * 1..PAB_MAX_CELLS.  The call
 * clears the block, launches the step kernel and copies the block out; it
 * calls no cudaMalloc, cudaFree or allocating library routine.  Every call
 * shares the block, so calls that overlap on the GPU (other streams, other
 * threads) race on it and may report each other's counts; the state and the
 * moments, which live in caller buffers, are not affected.
 * The first call in each CUDA context (the device's primary context, normally)
 * looks up the block's device address with that context current
 * (cudaGetSymbolAddress) and caches it under the context's id; a context made
 * anew, after cudaDeviceReset for instance, looks it up again on its first
 * call.  Make the first call in a context before any stream capture.
 * Errors: PAB_EINVAL (bad cfg, explicit weights summing to zero, NULL
 * pointers, dt <= 0 or non-finite),
 * PAB_ECUDA (symbol lookup or launch failure).
 */
#define PAB_NOALLOC_SCRATCH_BYTES 256
pab_status pab_bubble_step_noalloc(const pab_config *cfg, const double *p_inf_dev,
                                   const double *nb_dev, double dt, double *R_dev,
                                   double *Rdot_dev, float *h_dev, double *moments_dev,
                                   int64_t *status_dev, void *stream);

/* Release the state on the creation stream (waiting for pipelined host
 * calls first).  NULL-safe. */
void pab_destroy(pab_t *h);

/* Description of the last failure on this handle ("" if none). */
const char *pab_last_error(const pab_t *h);

/* Static name of a status code. */
const char *pab_status_string(pab_status s);

#ifdef __cplusplus
}
#endif

#endif /* PAB_H */
