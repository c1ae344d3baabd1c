/*
 * pab_measure.h - measurement aid shipped with libpab.
 *
 * The paper has no counterpart of these entry points: they serve the
 * roofline of the bubble kernels (how fast this GPU retires fused
 * multiply-adds in FP64 and in FP32) and the tests of the kernels' helper
 * arithmetic and of the host-built gas-term table.
 */
#ifndef PAB_MEASURE_H
#define PAB_MEASURE_H

#include <stdint.h>

#include "pab.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Throughput of dependent-free FMA streams: `blocks` CTAs of `threads`
 * threads each run 8 independent FMA chains of `iters` steps in FP64
 * (precision = PAB_FP64) or FP32 (PAB_MIXED), launched on `stream` and timed
 * with CUDA events.  Writes the kernel time in ms to *ms_out and the FMA
 * count (2 flops each) to *fma_out; the result of the chains goes to the
 * device scratch sink_dev (>= blocks*threads doubles, caller-owned) so that
 * nothing is optimised away.  Synchronises `stream`.
 * Errors: PAB_EINVAL (bad sizes or NULL pointers), PAB_ECUDA.
 */
pab_status pab_peak_fma(int32_t precision, int32_t blocks, int32_t threads, int32_t iters,
                        double *sink_dev, float *ms_out, double *fma_out, void *stream);

/*
 * The FP32 gas term of the mixed right-hand side, (1 + u)^(-a) - 1, for the
 * tests to compare with FP64 references (no counterpart in the paper): for
 * i < n, out_dev[i] = the library's branch-free evaluation at u_dev[i] and
 * lib_dev[i] = expm1f(-a log1pf(u_dev[i])) with CUDA's functions.  All arrays
 * [n] FP32 on the device; 1 + u > 0, a = 3 gamma > 0.
 * Errors: PAB_EINVAL (n < 0, a <= 0 or NULL pointers with n > 0), PAB_ECUDA.
 */
pab_status pab_gas32_check(int64_t n, const float *u_dev, float a, float *out_dev, float *lib_dev,
                           void *stream);

/*
 * Values of the FP64 device helpers, for the tests to compare with
 * high-precision references (no counterpart in the paper):
 *   gas_dev[i]     = the library's (1/R[i])^a reached from the base radius Rb[i]
 *                    (exact value at Rb[i] times the binomial series of
 *                    (1 + d)^(-a), d = (R[i] - Rb[i]) / Rb[i], or the exact value
 *                    when |d| is beyond the series' range);
 *   gas_tab_dev[i] = the same value from the node table a handle uses (nearest
 *                    node x_j = q^j of R[i], node value times the series);
 *   exact_dev[i]   = exp(a log(1/R[i])) with CUDA's exp and log.
 * All arrays [n] FP64 on the device; a = 3 gamma > 0.  Allocates and frees a
 * small table.  Errors: PAB_EINVAL, PAB_ECUDA.
 */
pab_status pab_math_check(int64_t n, const double *R_dev, const double *Rb_dev, double a,
                          double *gas_dev, double *gas_tab_dev, double *exact_dev, void *stream);

/*
 * Values of the helpers that take work off the FP64 pipe, for the tests to
 * compare with the hardware's own conversions, compares and division (no
 * counterpart in the paper).  For i < n:
 *   f2d_dev[i]  = the library's integer float -> double of f_dev[i];
 *   f2d_hw[i]   = (double)f_dev[i] by the conversion instruction;
 *   rcp_dev[i]  = the library's reciprocal of x_dev[i];
 *   div_dev[i]  = 1.0 / x_dev[i] (IEEE division);
 *   seed_dev[i] = the rcp.approx.ftz.f64 estimate the reciprocal starts from;
 *   cmp_dev[i]  = bit k set when the library's k-th predicate disagrees with the
 *                 IEEE one: 0 x > 0, 1 x <= y, 2 isfinite(x), 3 |x| >= y,
 *                 4 fmax(|x|, y) (compared as bit patterns), 5 fmin(|x|, y),
 *                 6 (float)x (bit patterns, with subnormal float results
 *                 flushed to a signed zero; NaN for NaN), 7 the embedded
 *                 difference 2 k3 - (k1 + k2) of k1 = f, k2 = (float)x,
 *                 k3 = (float)y against FP64 within 2^-46 of its terms
 *                 (where |k1|, |k2|, |k3| < 2^100),
 *                 8 2|x| and 2s (s the subnormal or zero with the bits of |x|
 *                 shifted right by 12) against the FP64 additions, 9 the
 *                 library's FP32 quotient f / (float)x and 10 its reciprocal
 *                 1 / (float)x, each within an ulp of the IEEE operation
 *                 where operands and result lie between 2^-100 and 2^100,
 *                 11 the library's short float -> double of a finite f with
 *                 |f| < 2^104 (bit patterns);
 *                 y_dev[i] must be a finite number >= +0.
 * f_dev [n] float; the others [n] double (cmp_dev [n] uint16), all on the device.
 * Errors: PAB_EINVAL (n < 0 or NULL pointers with n > 0), PAB_ECUDA.
 */
pab_status pab_bits_check(int64_t n, const float *f_dev, const double *x_dev, const double *y_dev,
                          double *f2d_dev, double *f2d_hw, double *rcp_dev, double *div_dev,
                          double *seed_dev, uint16_t *cmp_dev, void *stream);

/*
 * The smear's FP64 exponential against the library's (no counterpart in the
 * paper; a test hook): mine_dev[i] = the table-driven e^x the Gaussian kernel
 * of the Euler-Lagrange smear uses, lib_dev[i] = the CUDA math library's exp,
 * for x_dev[i].  All [n] double on the device.
 * Errors: PAB_EINVAL (n < 0 or NULL pointers with n > 0), PAB_ECUDA.
 */
pab_status pab_exp_check(int64_t n, const double *x_dev, double *mine_dev, double *lib_dev,
                         void *stream);

/*
 * The integer-pipe arithmetic against FP64 (no counterpart in the paper; a
 * test hook for the n_b R_i, n_b Rdot_i inversion of Listing 2 and Eq. e:ndf
 * and for the FP64 trial's Keller-Miksis right-hand side, Eq. keller_miksis):
 * prod_dev[i] = x_dev[i] y_dev[i], cube_dev[i] = x_dev[i]^3 and
 * rcp_dev[i] = 1 / x_dev[i], each formed from the significands with integer
 * multiplies (the reciprocal from an FP32 approximate one, refined as an
 * integer) and rounded once; the FP64 operation for zero, subnormal, infinite
 * or NaN operands and results outside the normal range.  Each is within 1 ulp
 * of the correctly rounded value.  All [n] double on the device.
 * Errors: PAB_EINVAL (n < 0 or NULL pointers with n > 0), PAB_ECUDA.
 */
pab_status pab_intmul_check(int64_t n, const double *x_dev, const double *y_dev, double *prod_dev,
                            double *cube_dev, double *rcp_dev, void *stream);

/*
 * The trial accept tests against their exact forms (no counterpart in the
 * paper; a test hook for the controller of Sec. 3).  For each i:
 *   out[4i+0]  the FP64 trial's accept decision (an FP32 error estimate decides
 *              outside tol (1 -/+ 2^-16), the FP64 test inside) on the trial
 *              trial[4i..4i+3] = {R3, Rdot3, e_R, e_Rdot} (e: three times the
 *              embedded difference), the trial taken as valid;
 *   out[4i+1]  the exact FP64 test |e_R| <= 3 tol |R3| and
 *              |e_Rdot| <= 3 tol max(|Rdot3|, v_floor) on the same trial;
 *   out[4i+2]  the mixed trial's test on one component (an FP32 bound on the
 *              TwoSum parts decides outside T (1 -/+ 2^-20), the FP64 sum
 *              inside) for k[4i..4i+3] = {k1, k2, k3, T};
 *   out[4i+3]  the exact form: |d + (e_d - e_s)| <= T with the FP64 sum.
 * trial_dev [4n] double, k_dev [4n] float, out_dev [4n] uint8, on the device;
 * tol > 0 and v_floor >= 0 as in pab_config.
 * Errors: PAB_EINVAL (n < 0, NULL pointers with n > 0, tol or v_floor out of
 * range), PAB_ECUDA.
 */
pab_status pab_accept_check(int64_t n, const double *trial_dev, const float *k_dev, double tol,
                            double v_floor, uint8_t *out_dev, void *stream);

/*
 * The gas-term node table a handle builds for the polytropic exponent gamma,
 * on the host (no handle, no device).  The gas factor (R0/R)^(3 gamma) is
 * x^(-3 gamma) with x = R/R0; the table holds nodes x_j = q^j, j = -J..J
 * (covering 1/25..25), each as *stride doubles {x_j, c_0, .., c_d, 0 ..}
 * with c_k the coefficients of the binomial series of (x_j + delta)^(-3 gamma)
 * in delta, so that x^(-3 gamma) = sum_k c_k (x - x_j)^k for x near x_j.
 * *dmax receives the bound on |x/x_j - 1| within which the first omitted term
 * stays below half an ulp; the nodes are spaced so that the nearest one (in
 * log x) is always within it.  *n_nodes = 2 J + 1.  When tab_host is not NULL
 * it receives the table if capacity (doubles) holds it.
 * Errors: PAB_EINVAL (gamma not positive and finite, NULL counts, capacity
 * too small).
 */
pab_status pab_gas_table(double gamma, double *tab_host, int64_t capacity, int32_t *n_nodes,
                         int32_t *stride, double *dmax);

/*
 * Report of the checked build (no counterpart in the paper).  The library
 * compiled with PAB_CHECKED (libpab_checked.so) tests every global-memory
 * index of its kernels against the length of its buffer before the access,
 * skips the access when the index falls outside, and records the first such
 * index of each source file with its line and the buffer's length.  This call
 * waits for the device, returns that record for the first file with one
 * (unit: 1 step kernels, 2 batch, 3 carrier coupling, 4 Euler-Lagrange, 5
 * transfer contents; *count: how many indices fell outside in that file,
 * 0 and the other outputs 0 when none did) and clears every record.
 * NULL outputs are allowed.
 * Errors: PAB_ESTATE (a library built without PAB_CHECKED; *count = 0),
 * PAB_ECUDA.
 */
pab_status pab_check_report(int64_t *count, int32_t *unit, int32_t *line, int64_t *index, int64_t *bound);

#ifdef __cplusplus
}
#endif

#endif /* PAB_MEASURE_H */
