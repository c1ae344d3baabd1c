// Internal declarations shared by the host API and the kernels of libpab.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "pab.h"

namespace pab {

// Per-bin constants, computed once in FP64 on the host at create time, with
// pg0 = p0 + 2 sigma/R0 - pv the gas pressure at equilibrium (0 for an empty
// cavity) and peq = pv + pg0 - 2 sigma/R0 the wall pressure at rest at R0.
// 56 bytes: 63 of them keep StepConst within the 4 KB of kernel parameters
// that are read like any other constant.
struct BinConst {
    double R0;     // equilibrium radius R0_i
    double w;      // quadrature weight w_i (sums to one over the bins)
    double invR0;  // 1/R0
    double A1;     // pg0 / rho
    double A3;     // (1 - 3 gamma) pg0 / (rho c)
    float R0f;     // R0 in FP32 (mixed path)
    float invR0f;  // 1/R0 in FP32
    float pg0f;    // pg0 in FP32
    float dpeqf;   // peq - p0 in FP32 (0 up to rounding for the polytropic gas)
};

// Warps per CTA of the step kernels when the configuration leaves it open.  A CTA of w warps
// owns w tiles of 32 cells and streams their items from one pool (pab_stream.cuh), parking the
// mixed path's FP64 trials in one lot.  Measured on the 128^3 x 31 line and on the collapse
// window of the 64^3 x 31 stress workload (1, 4 and 8 warps): FP64 4.93/5.00/5.01e9 and
// 4.45/4.46/4.28e9 bin-steps/s; mixed 25.5/26.0/25.7e9 and 8.85/9.27/8.93e9.  4 in both.
constexpr int kDefaultWarps = 4;
constexpr int kDefaultWarpsMixed = 4;
inline int default_warps(int precision) { return precision == PAB_MIXED ? kDefaultWarpsMixed : kDefaultWarps; }

constexpr int kGasTerms = 12;    // binomial series of the gas term: degree 11
constexpr int kGasTabTerms = 4;   // degree 3 around the nodes of a gas table
constexpr int kGasTabStride = 6;  // doubles per node: x_j, the coefficients and a pad

// Liquid, gas and stepper constants.  Passed by value as a kernel parameter,
// so warp-uniform reads come from the constant bank.
struct StepConst {
    int64_t C;            // cells
    int32_t B;            // bins
    int32_t gas_mode;
    int32_t max_attempts;
    int32_t n_fixed;      // > 0: fixed mode with n_fixed sub-steps
    double rho, inv_rho, c, inv_c, pv, p0;
    double three_gamma;   // 3 gamma
    double two_sigma;     // 2 sigma
    double ic_rho;        // (1/c)/rho
    double fmu_ic_rho;    // 4 mu (1/c)/rho
    double fmu_rho;       // 4 mu / rho
    double tsig_rho;      // 2 sigma / rho
    double pv_rho;        // pv / rho
    double m05_inv_c;     // -0.5 / c
    double tol;
    double tol3;          // 3 tol (Trial carries three times the embedded difference)
    double v_floor;
    double v_collapse;    // mixed: |Rdot| above this takes the FP64 path (c/20)
    double r_collapse;    // mixed: R/R0 below this takes the FP64 path (0.2)
    double nb_default;    // n_b when the caller passes no n_b field
    // contents with heat and mass transfer (gas_mode PAB_GAS_TRANSFER)
    double tr_Rg, tr_Rv;  // gas constants of the gas and of the vapour
    double tr_RvTw_4pi;   // R_v T_w / (4 pi)
    double tr_rho_vw;     // pv / (R_v T_w): vapour density at the wall
    double tr_inv_RgTw;   // 1 / (R_g T_w)
    double tr_kT_43pi;    // (4 pi/3) (gamma - 1)/gamma k_bw beta_T
    double tr_kT_Tw;      // (gamma - 1)/gamma k_bw beta_T T_w
    double tr_Dc_4pi;     // 4 pi D beta_c
    // (1 + d)^(-3 gamma) = sum_k gas_c[k] d^k for |d| <= gas_dmax (truncation below half an ulp)
    double gas_c[kGasTerms];
    double gas_dmax;
    double gas_dmax_tab;  // the same bound for the degree kGasTabTerms-1 of the table path
    // optional table of nodes x_j = q^j, j = -gas_J..gas_J, kGasTabStride doubles each,
    // {x_j, c_0 .. c_3, 0}: (R/R0)^(-3 gamma) = sum_k c_k (R/R0 - x_j)^k with
    // c_k = x_j^(-3 gamma) C(-3 gamma, k) x_j^(-k), the binomial series about the node
    // (nullptr: no table)
    const double *gas_tab;
    float gas_inv_log2q;  // 1/log2(q)
    int32_t gas_J;
    float inv_rhof, inv_cf, four_muf, two_sigmaf, three_gammaf, ic_rhof, fmu_ic_rhof, v_floorf;
    float cbrt_tolf, v_collapsef, r_collapsef, cf;
    float tg_ic_rhof;     // 3 gamma (1/c)/rho
    float tol3f;          // 3 tol
    // the FP64 accept test's bracket: an FP32 error estimate below tol_lof is accepted and one
    // above tol_hif rejected without the exact test (tol (1 -/+ 2^-16); -1 and inf, that is never,
    // for tol below 1e-7)
    float tol_lof, tol_hif;
    BinConst bins[PAB_MAX_BINS];
};

static_assert(sizeof(BinConst) == 56, "BinConst layout");
static_assert(sizeof(StepConst) <= 4000, "StepConst must fit the 4 KB kernel-parameter space");

// Device-side status accumulated over calls until pab_status_flags reads it.

struct Counters {
    unsigned int flags_or;
    unsigned int pad;
    unsigned long long n_flagged;
    unsigned long long n_attempts;
    unsigned long long n_fp64;
};

// A mixed-precision item parked in a CTA's lot: the controller state of one (bin, cell) part
// way through its flow step.
struct Parked {
    double xi64, V, h, rem;
    float xi, v;
    int32_t b, n, n64, pad;
    int64_t c;
};

struct StepArgs {
    const double *p_inf;   // [C]
    const double *nb;      // [C] or nullptr
    double dt;
    double *R;             // [B][C]
    double *V;             // [B][C]
    float *h;              // [B][C]
    int32_t *attempts;     // [B][C] or nullptr
    double *out;           // [7][C] or nullptr
    Counters *counters;
    double dt_sub = 0.0;   // dt / n_fixed in fixed mode (formed on the host)
    double *pb = nullptr;  // [B][C] bubble pressure (PAB_GAS_TRANSFER)
    double *mv = nullptr;  // [B][C] vapour mass (PAB_GAS_TRANSFER)
    // A grid split by bins (step_splits_by_bins) ends with its moments when both are given:
    // terms, [4][B][C] doubles for its items' quadrature terms, and tickets, one zeroed counter
    // per 32-cell tile (left zeroed).  Without them its moments come from a second launch.
    double *terms = nullptr;
    unsigned int *tickets = nullptr;
    // FP64: [B][C] the gas factor at the stored radii.  The moment pass writes it (when moments
    // are requested); with G_valid the items start from it instead of evaluating it again.
    double *G = nullptr;
    int G_valid = 0;
};

// The first out-of-bounds index a checked build (PAB_CHECKED, pab_check.cuh) met in one
// translation unit: how many were met, the source line, the index and the buffer's length.
struct CheckRecord {
    unsigned int count;
    int line;
    long long index;
    long long bound;
};
// Readers of each unit's record (zeros in an unchecked build); clear: reset it after reading.
void check_fetch_kernels(CheckRecord *r, bool clear);
void check_fetch_batch(CheckRecord *r, bool clear);
void check_fetch_closure(CheckRecord *r, bool clear);
void check_fetch_el(CheckRecord *r, bool clear);
void check_fetch_transfer(CheckRecord *r, bool clear);

// Configuration helpers (pab_api.cu): validation as pab_create does it, the
// bin table of a configuration, and the kernel constants.
pab_status validate_config(const pab_config *c, char *msg, size_t n);
bool bin_table(const pab_config *c, double *R0, double *w);
void make_const(const pab_config *c, const double *R0, const double *w, StepConst *K);
BinConst make_bin(const pab_config *c, double R0, double w);  // constants of one radius
// Host values of the gas-term table for a = 3 gamma (kGasTabStride * (2 J + 1) doubles) and its
// spacing.
void gas_table(double a, double dmax, std::vector<double> *tab, int *J, double *inv_log2q);

// Launchers (pab_kernels.cu).  Return the launch error.
cudaError_t launch_step(const StepConst &K, int precision, const StepArgs &a, int block_warps,
                        cudaStream_t s);
cudaError_t launch_moments(const StepConst &K, int precision, const double *nb, const double *R,
                           const double *V, double *out, int block_warps, cudaStream_t s);
// True when launch_step splits this grid by bins over more CTAs (fewer 32-cell tiles than the
// current device's SMs, more than one bin): its moments then come from a second launch.
bool step_splits_by_bins(const StepConst &K);
cudaError_t launch_init(const StepConst &K, double Rdot0_ref, double R0ref, double *R, double *V,
                        float *h, cudaStream_t s);
// Contents with transfer (pab_transfer.cu): the step, the moments and the equilibrium
// contents p_b = p0 + 2 sigma/R0, m_v = pv V0/(R_v T_w).
cudaError_t launch_transfer_step(const StepConst &K, const StepArgs &a, int block_warps, cudaStream_t s);
cudaError_t launch_transfer_moments(const StepConst &K, const double *nb, const double *R,
                                    const double *V, const double *pb, double *out, int block_warps,
                                    cudaStream_t s);
cudaError_t launch_transfer_init(const StepConst &K, double *pb, double *mv, cudaStream_t s);

// Launchers of the carrier-facing forms (pab_closure.cu).
cudaError_t launch_cons_from_prim(const StepConst &K, const double *nb, const double *R,
                                  const double *V, double *qR, double *qV, cudaStream_t s);
cudaError_t launch_prim_from_cons(const StepConst &K, const double *alpha, const double *qR,
                                  const double *qV, double *R, double *V, double *nb_out,
                                  cudaStream_t s);
cudaError_t launch_mixture_pressure(long long C, const double *moments, const double *p_l,
                                    const double *rho_l, double rho_default, double *p,
                                    cudaStream_t s);
cudaError_t launch_stiffened_gas(long long n, const double *rho, const double *e, double gamma_l,
                                 double pi_inf, double *p, cudaStream_t s);

}  // namespace pab
