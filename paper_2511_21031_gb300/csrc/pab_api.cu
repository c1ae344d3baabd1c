// Host side of the C ABI declared in include/pab.h: configuration checks,
// the lognormal bin table, device state ownership and the stream-ordered
// entry points.  No compute happens here; every step of the path runs in the
// kernels of pab_kernels.cu.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "pab.h"
#include "pab_transfer.h"
#include "pab_closure.h"
#include "pab_measure.h"
#include "pab_internal.h"

struct pab_s {
    pab_config cfg;
    pab::StepConst K;
    int device = 0;
    cudaStream_t create_stream = nullptr;
    double *R = nullptr;
    double *V = nullptr;
    float *h = nullptr;
    int32_t *attempts = nullptr;
    double *G = nullptr;        // [Nb][C] gas factor at the stored radii (FP64 polytropic)
    int G_valid = 0;            // G holds the factor at the current state
    double *terms = nullptr;    // [4][Nb][C] quadrature terms of a grid split by bins
    unsigned int *tickets = nullptr;  // [tiles] its per-tile counters (zero between steps)
    double *gas_tab = nullptr;  // gas-term nodes (K.gas_tab points here)
    double *pb = nullptr;       // [Nb][C] bubble pressure (PAB_GAS_TRANSFER)
    double *mv = nullptr;       // [Nb][C] vapour mass (PAB_GAS_TRANSFER)
    pab::Counters *counters = nullptr;
    pab::Counters *counters_host = nullptr;  // pinned
    double *stage_p = nullptr;                // host entry point staging [C]
    double *stage_nb = nullptr;               // [C]
    double *stage_out = nullptr;              // [7][C]
    // pipelined host entry point: two staging sets, an input and an output copy stream
    double *pipe_p[2] = {nullptr, nullptr};
    double *pipe_nb[2] = {nullptr, nullptr};
    double *pipe_out[2] = {nullptr, nullptr};
    cudaStream_t pipe_in = nullptr, pipe_outs = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_step[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
    bool pipe_busy[2] = {false, false};
    int pipe_next = 0;
    int block_warps = 8;
    char err[512] = {0};
};

namespace {

// Sub-step size of fixed mode (0 in adaptive mode).
double sub_step(const pab::StepConst &K, double dt) { return K.n_fixed > 0 ? dt / (double)K.n_fixed : 0.0; }

pab_status fail(pab_t *h, pab_status s, const char *fmt, ...)
{
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof(h->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

pab_status cuda_fail(pab_t *h, cudaError_t e, const char *what)
{
    return fail(h, e == cudaErrorMemoryAllocation ? PAB_ENOMEM : PAB_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

size_t n_state(const pab_t *h) { return (size_t)h->cfg.n_bins * (size_t)h->cfg.n_cells; }

// Lognormal bins with composite Simpson weights (Sec. 2.2): nodes equally
// spaced in phi = ln(R0/R0ref) over [-K s, K s]; coefficient 1,4,2,...,4,1
// times the normal density N(phi; 0, s^2); normalised to sum one.
bool lognormal_table(int B, double R0ref, double s, double K, double *R0, double *w)
{
    if (B == 1) {
        R0[0] = R0ref;
        w[0] = 1.0;
        return true;
    }
    if (B < 3 || B % 2 == 0 || !(s > 0.0) || !(K > 0.0))
        return false;
    const double step = 2.0 * K * s / (double)(B - 1);
    double sum = 0.0;
    for (int i = 0; i < B; ++i) {
        const double phi = -K * s + step * (double)i;
        const int coef = (i == 0 || i == B - 1) ? 1 : ((i & 1) ? 4 : 2);
        const double g = std::exp(-phi * phi / (2.0 * s * s));
        R0[i] = R0ref * std::exp(phi);
        w[i] = (double)coef * g;  // dphi/3 and the density's constant cancel
        sum += w[i];
    }
    for (int i = 0; i < B; ++i)
        w[i] /= sum;
    return true;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

pab_status validate(const pab_config *c, char *msg, size_t n)
{
#define BAD(...)                        \
    do {                                \
        snprintf(msg, n, __VA_ARGS__);  \
        return PAB_EINVAL;              \
    } while (0)
    if (c->n_cells < 1 || c->n_cells > PAB_MAX_CELLS)
        BAD("n_cells must be 1..%lld (got %lld)", (long long)PAB_MAX_CELLS, (long long)c->n_cells);
    if (c->n_bins < 1 || c->n_bins > PAB_MAX_BINS || (c->n_bins > 1 && c->n_bins % 2 == 0))
        BAD("n_bins must be 1 or odd in 3..%d (got %d)", PAB_MAX_BINS, c->n_bins);
    if (!finite_pos(c->rho) || !(c->c > 0.0) || !(c->mu >= 0.0) || !(c->sigma >= 0.0) ||
        !finite_pos(c->p0) || !finite_pos(c->gamma) || !(c->pv >= 0.0) || !std::isfinite(c->pv))
        BAD("fluid constants out of range");
    if (c->gas_mode != PAB_GAS_POLYTROPIC && c->gas_mode != PAB_GAS_EMPTY &&
        c->gas_mode != PAB_GAS_TRANSFER)
        BAD("gas_mode must be 0, 1 or 2");
    if (c->gas_mode == PAB_GAS_TRANSFER) {
        if (c->precision != PAB_FP64)
            BAD("gas_mode PAB_GAS_TRANSFER runs in PAB_FP64 only");
        if (!(c->pv < c->p0))
            BAD("gas_mode PAB_GAS_TRANSFER needs pv < p0 (a positive gas partial pressure)");
        if (!finite_pos(c->R_g) || !finite_pos(c->R_v) || !finite_pos(c->T_w))
            BAD("R_g, R_v and T_w must be positive");
        const double nn[] = {c->k_bw, c->D_vg, c->beta_T, c->beta_c};
        for (double x : nn)
            if (!(x >= 0.0) || !std::isfinite(x))
                BAD("k_bw, D_vg, beta_T and beta_c must be finite and >= 0");
    }
    if (c->precision != PAB_FP64 && c->precision != PAB_MIXED)
        BAD("precision must be PAB_FP64 or PAB_MIXED");
    if (c->stepper != PAB_ADAPTIVE && c->stepper != PAB_FIXED)
        BAD("stepper must be PAB_ADAPTIVE or PAB_FIXED");
    if (c->stepper == PAB_FIXED && c->n_fixed_sub < 1)
        BAD("n_fixed_sub must be >= 1 in fixed mode");
    if (c->max_attempts < 1)
        BAD("max_attempts must be >= 1");
    if (!finite_pos(c->tol))
        BAD("tol must be positive");
    if ((c->R0_host == nullptr) != (c->w_host == nullptr))
        BAD("R0_host and w_host must be given together");
    if (c->R0_host) {
        for (int i = 0; i < c->n_bins; ++i)
            if (!finite_pos(c->R0_host[i]) || !(c->w_host[i] >= 0.0) || !std::isfinite(c->w_host[i]))
                BAD("explicit bin table entry %d out of range", i);
    } else {
        if (!finite_pos(c->R0ref))
            BAD("R0ref must be positive");
        if (c->n_bins > 1 && (!finite_pos(c->s_lognormal) || !finite_pos(c->span_K)))
            BAD("s_lognormal and span_K must be positive when n_bins > 1");
    }
    if (!std::isfinite(c->Rdot0_ref) || !(c->alpha0 >= 0.0) || !std::isfinite(c->alpha0))
        BAD("Rdot0_ref / alpha0 out of range");
    if (c->block_warps < 0 || c->block_warps > 16)
        BAD("block_warps must be 0..16");
    return PAB_OK;
#undef BAD
}

void build_const(const pab_config *c, const double *R0, const double *w, pab::StepConst *K)
{
    std::memset(K, 0, sizeof(*K));
    K->C = c->n_cells;
    K->B = c->n_bins;
    K->gas_mode = c->gas_mode;
    K->max_attempts = c->max_attempts;
    K->n_fixed = c->stepper == PAB_FIXED ? c->n_fixed_sub : 0;
    K->rho = c->rho;
    K->inv_rho = 1.0 / c->rho;
    K->c = c->c;
    K->inv_c = 1.0 / c->c;
    K->pv = c->pv;
    K->p0 = c->p0;
    K->three_gamma = 3.0 * c->gamma;
    K->two_sigma = 2.0 * c->sigma;
    K->ic_rho = K->inv_c / c->rho;
    K->fmu_ic_rho = 4.0 * c->mu * K->inv_c / c->rho;
    K->fmu_rho = 4.0 * c->mu / c->rho;
    K->tsig_rho = 2.0 * c->sigma / c->rho;
    K->pv_rho = c->pv / c->rho;
    K->m05_inv_c = -0.5 * K->inv_c;
    K->tol = c->tol;
    K->tol3 = 3.0 * c->tol;
    K->v_floor = c->v_floor >= 0.0 ? c->v_floor : 1e-3 * std::sqrt(c->p0 / c->rho);
    K->v_collapse = c->c / 20.0;
    K->r_collapse = 0.2;
    K->inv_rhof = (float)K->inv_rho;
    K->inv_cf = (float)K->inv_c;
    K->four_muf = (float)(4.0 * c->mu);
    K->two_sigmaf = (float)K->two_sigma;
    K->three_gammaf = (float)K->three_gamma;
    K->ic_rhof = (float)K->ic_rho;
    K->tg_ic_rhof = (float)(K->three_gamma * K->ic_rho);
    K->fmu_ic_rhof = (float)K->fmu_ic_rho;
    K->v_floorf = (float)K->v_floor;
    K->cbrt_tolf = (float)std::cbrt(c->tol);
    K->tol3f = (float)K->tol3;
    K->tol_lof = c->tol >= 1e-7 ? (float)(c->tol * (1.0 - 0x1p-16)) : -1.0f;
    K->tol_hif = c->tol >= 1e-7 ? (float)(c->tol * (1.0 + 0x1p-16)) : INFINITY;
    K->v_collapsef = (float)K->v_collapse;
    K->r_collapsef = (float)K->r_collapse;
    K->cf = (float)c->c;
    K->tr_Rg = c->R_g;
    K->tr_Rv = c->R_v;
    K->tr_RvTw_4pi = c->R_v * c->T_w / (4.0 * M_PI);
    K->tr_rho_vw = c->gas_mode == PAB_GAS_TRANSFER ? c->pv / (c->R_v * c->T_w) : 0.0;
    K->tr_inv_RgTw = c->gas_mode == PAB_GAS_TRANSFER ? 1.0 / (c->R_g * c->T_w) : 0.0;
    const double kT = (c->gamma - 1.0) / c->gamma * c->k_bw * c->beta_T;
    K->tr_kT_43pi = 4.0 / 3.0 * M_PI * kT;
    K->tr_kT_Tw = kT * c->T_w;
    K->tr_Dc_4pi = 4.0 * M_PI * c->D_vg * c->beta_c;
    double m3 = 0.0;
    for (int i = 0; i < c->n_bins; ++i) {
        pab::BinConst &b = K->bins[i];
        b.R0 = R0[i];
        b.w = w[i];
        const double pg0 =
            c->gas_mode == PAB_GAS_POLYTROPIC ? c->p0 + 2.0 * c->sigma / R0[i] - c->pv : 0.0;
        const double peq = c->pv + pg0 - 2.0 * c->sigma / R0[i];
        b.R0f = (float)R0[i];
        b.invR0f = (float)(1.0 / R0[i]);
        b.pg0f = (float)pg0;
        b.dpeqf = (float)(peq - c->p0);
        b.invR0 = 1.0 / R0[i];
        b.A1 = pg0 / c->rho;
        b.A3 = (1.0 - 3.0 * c->gamma) * pg0 / c->rho * K->inv_c;
        m3 += w[i] * R0[i] * R0[i] * R0[i];
    }
    K->nb_default = m3 > 0.0 ? c->alpha0 / (4.0 / 3.0 * M_PI * m3) : 0.0;
    // binomial series (1 + d)^(-a) = sum_k C(-a, k) d^k, a = 3 gamma, truncated after
    // degree kGasTerms-1; the series is used where the first omitted term is below
    // 1.1e-16 (half an ulp of the result)
    const double a = 3.0 * c->gamma;
    double ck = 1.0;
    for (int k = 0; k < pab::kGasTerms; ++k) {
        K->gas_c[k] = ck;
        ck *= (-a - (double)k) / (double)(k + 1);
        if (k + 1 == pab::kGasTabTerms)
            K->gas_dmax_tab = std::pow(1.1e-16 / std::fabs(ck), 1.0 / (double)pab::kGasTabTerms);
    }
    K->gas_dmax = std::pow(1.1e-16 / std::fabs(ck), 1.0 / (double)pab::kGasTerms);
    K->gas_tab = nullptr;  // the handle attaches its table after allocating it
    K->gas_inv_log2q = 0.0f;
    K->gas_J = 0;
}

}  // namespace

namespace pab {

pab_status validate_config(const pab_config *c, char *msg, size_t n) { return validate(c, msg, n); }

bool bin_table(const pab_config *c, double *R0, double *w)
{
    if (c->R0_host) {
        double sum = 0.0;
        for (int i = 0; i < c->n_bins; ++i) {
            R0[i] = c->R0_host[i];
            w[i] = c->w_host[i];
            sum += w[i];
        }
        return sum > 0.0;
    }
    return lognormal_table(c->n_bins, c->R0ref, c->s_lognormal, c->span_K, R0, w);
}

void make_const(const pab_config *c, const double *R0, const double *w, StepConst *K)
{
    build_const(c, R0, w, K);
}

// Nodes x_j = q^j with (sqrt(q) - 1) = 0.9 d_max, so that the nearest node of any
// x in [q^-J, q^J] lies within the series' range; J covers R/R0 from 1/25 to 25.
void gas_table(double a, double dmax, std::vector<double> *tab, int *J, double *inv_log2q)
{
    const double sq = 1.0 + 0.9 * dmax;
    const double q = sq * sq;
    const double lq = std::log(q);
    *J = (int)std::ceil(std::log(25.0) / lq);
    *inv_log2q = 1.0 / std::log2(q);
    tab->resize((size_t)kGasTabStride * (2 * *J + 1));
    for (int j = -*J; j <= *J; ++j) {
        const double x = std::exp((double)j * lq);
        double *e = tab->data() + kGasTabStride * (size_t)(j + *J);
        e[0] = x;
        // c_k = x^(-a) C(-a, k) x^(-k): the binomial series of (x + delta)^(-a) in delta
        double ck = std::pow(x, -a);
        for (int k = 0; k < kGasTabTerms; ++k) {
            e[1 + k] = ck;
            ck *= (-a - (double)k) / ((double)(k + 1) * x);
        }
        for (int k = 1 + kGasTabTerms; k < kGasTabStride; ++k)
            e[k] = 0.0;
    }
}

BinConst make_bin(const pab_config *c, double R0, double w)
{
    StepConst K;
    pab_config one = *c;
    one.n_bins = 1;
    build_const(&one, &R0, &w, &K);
    return K.bins[0];
}

}  // namespace pab

extern "C" {

void pab_config_default(pab_config *c)
{
    if (!c)
        return;
    std::memset(c, 0, sizeof(*c));
    c->n_cells = 1;
    c->n_bins = 21;
    c->gas_mode = PAB_GAS_POLYTROPIC;
    c->rho = 1000.0;
    c->c = 1500.0;
    c->mu = 1e-3;
    c->sigma = 0.072;
    c->p0 = 101325.0;
    c->gamma = 1.4;
    c->pv = 0.0;
    c->R0ref = 10e-6;
    c->s_lognormal = 0.3;
    c->span_K = 5.0;
    c->precision = PAB_FP64;
    c->stepper = PAB_ADAPTIVE;
    c->n_fixed_sub = 1;
    c->max_attempts = 100000;
    c->tol = 1e-4;
    c->v_floor = -1.0;
    c->alpha0 = 4e-5;
    c->Rdot0_ref = 0.0;
    c->R_g = 287.05;
    c->R_v = 461.5;
    c->T_w = 293.15;
    c->k_bw = 0.0257;
    c->D_vg = 2.42e-5;
    c->beta_T = 5.0;
    c->beta_c = 5.0;
    c->record_attempts = 0;
    c->block_warps = 0;
}

const char *pab_status_string(pab_status s)
{
    switch (s) {
    case PAB_OK: return "PAB_OK";
    case PAB_EINVAL: return "PAB_EINVAL";
    case PAB_ENOMEM: return "PAB_ENOMEM";
    case PAB_ECUDA: return "PAB_ECUDA";
    case PAB_ESTEP_LIMIT: return "PAB_ESTEP_LIMIT";
    case PAB_ENONFINITE: return "PAB_ENONFINITE";
    case PAB_ESTATE: return "PAB_ESTATE";
    }
    return "PAB_UNKNOWN";
}

const char *pab_last_error(const pab_t *h) { return h ? h->err : "NULL handle"; }

pab_status pab_create(const pab_config *cfg, void *stream, pab_t **out)
{
    if (!out)
        return PAB_EINVAL;
    *out = nullptr;
    if (!cfg)
        return PAB_EINVAL;
    char msg[256];
    if (validate(cfg, msg, sizeof(msg)) != PAB_OK) {
        fprintf(stderr, "pab_create: %s\n", msg);
        return PAB_EINVAL;
    }
    double R0[PAB_MAX_BINS], w[PAB_MAX_BINS];
    if (cfg->R0_host) {
        double sum = 0.0;
        for (int i = 0; i < cfg->n_bins; ++i) {
            R0[i] = cfg->R0_host[i];
            w[i] = cfg->w_host[i];
            sum += w[i];
        }
        if (!(sum > 0.0)) {
            fprintf(stderr, "pab_create: explicit weights sum to zero\n");
            return PAB_EINVAL;
        }
    } else if (!lognormal_table(cfg->n_bins, cfg->R0ref, cfg->s_lognormal, cfg->span_K, R0, w)) {
        fprintf(stderr, "pab_create: invalid bin table request\n");
        return PAB_EINVAL;
    }
    pab_t *h = new (std::nothrow) pab_t();
    if (!h)
        return PAB_ENOMEM;
    h->cfg = *cfg;
    h->cfg.R0_host = nullptr;
    h->cfg.w_host = nullptr;
    h->create_stream = (cudaStream_t)stream;
    h->block_warps = cfg->block_warps > 0 ? cfg->block_warps : pab::default_warps(cfg->precision);
    build_const(cfg, R0, w, &h->K);
    cudaError_t e = cudaGetDevice(&h->device);
    const size_t n = n_state(h);
    cudaStream_t s = h->create_stream;
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&h->R, n * sizeof(double), s);
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&h->V, n * sizeof(double), s);
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&h->h, n * sizeof(float), s);
    if (e == cudaSuccess && cfg->record_attempts)
        e = cudaMallocAsync((void **)&h->attempts, n * sizeof(int32_t), s);
    // a small grid's step is split by bins over more CTAs, which store their items' quadrature
    // terms and count off each tile (at most 32 x SMs cells x 63 bins x 32 bytes, under 10 MB on
    // 152 SMs)
    // FP64 polytropic steps carry each bin's gas factor from one flow step's moment pass to the
    // next step's first right-hand side (8 bytes per bin-state)
    if (e == cudaSuccess && cfg->precision == PAB_FP64 && cfg->gas_mode == PAB_GAS_POLYTROPIC)
        e = cudaMallocAsync((void **)&h->G, n * sizeof(double), s);
    const bool split = cfg->gas_mode != PAB_GAS_TRANSFER && pab::step_splits_by_bins(h->K);
    const size_t n_tiles = (size_t)((cfg->n_cells + 31) / 32);
    if (e == cudaSuccess && split)
        e = cudaMallocAsync((void **)&h->terms, 4 * n * sizeof(double), s);
    if (e == cudaSuccess && split)
        e = cudaMallocAsync((void **)&h->tickets, n_tiles * sizeof(unsigned int), s);
    if (e == cudaSuccess && split)
        e = cudaMemsetAsync(h->tickets, 0, n_tiles * sizeof(unsigned int), s);
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&h->counters, sizeof(pab::Counters), s);
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&h->counters_host, sizeof(pab::Counters));
    std::vector<double> tab;
    int J = 0;
    double il2q = 0.0;
    pab::gas_table(3.0 * cfg->gamma, h->K.gas_dmax_tab, &tab, &J, &il2q);
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&h->gas_tab, tab.size() * sizeof(double), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->gas_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);  // tab is a host temporary
    if (e == cudaSuccess) {
        h->K.gas_tab = h->gas_tab;
        h->K.gas_J = J;
        h->K.gas_inv_log2q = (float)il2q;
    }
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->counters, 0, sizeof(pab::Counters), s);
    if (e == cudaSuccess && h->attempts)
        e = cudaMemsetAsync(h->attempts, 0, n * sizeof(int32_t), s);
    if (e == cudaSuccess)
        e = pab::launch_init(h->K, cfg->Rdot0_ref, cfg->R0ref, h->R, h->V, h->h, s);
    if (e == cudaSuccess && cfg->gas_mode == PAB_GAS_TRANSFER) {
        e = cudaMallocAsync((void **)&h->pb, n * sizeof(double), s);
        if (e == cudaSuccess)
            e = cudaMallocAsync((void **)&h->mv, n * sizeof(double), s);
        if (e == cudaSuccess)
            e = pab::launch_transfer_init(h->K, h->pb, h->mv, s);
    }
    if (e != cudaSuccess) {
        pab_status st = e == cudaErrorMemoryAllocation ? PAB_ENOMEM : PAB_ECUDA;
        fprintf(stderr, "pab_create: %s\n", cudaGetErrorString(e));
        cudaGetLastError();
        pab_destroy(h);
        return st;
    }
    *out = h;
    return PAB_OK;
}

void pab_destroy(pab_t *h)
{
    if (!h)
        return;
    cudaStream_t s = h->create_stream;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != h->device)
        cudaSetDevice(h->device);
    for (int i = 0; i < 2; ++i) {
        if (h->ev_out[i])
            cudaEventSynchronize(h->ev_out[i]);
    }
    void *bufs[] = {h->R, h->V, h->h, h->attempts, h->G, h->terms, h->tickets, h->gas_tab, h->pb, h->mv, h->counters, h->stage_p,
                    h->stage_nb, h->stage_out, h->pipe_p[0], h->pipe_p[1], h->pipe_nb[0], h->pipe_nb[1],
                    h->pipe_out[0], h->pipe_out[1]};
    for (void *b : bufs)
        if (b)
            cudaFreeAsync(b, s);
    cudaStreamSynchronize(s);
    for (int i = 0; i < 2; ++i) {
        cudaEvent_t evs[] = {h->ev_in[i], h->ev_step[i], h->ev_out[i]};
        for (cudaEvent_t ev : evs)
            if (ev)
                cudaEventDestroy(ev);
    }
    if (h->pipe_in)
        cudaStreamDestroy(h->pipe_in);
    if (h->pipe_outs)
        cudaStreamDestroy(h->pipe_outs);
    if (h->counters_host)
        cudaFreeHost(h->counters_host);
    if (cur != h->device)
        cudaSetDevice(cur);
    delete h;
}

pab_status pab_bubble_step(pab_t *h, const double *p_inf_dev, const double *nb_dev, double dt,
                           double *moments_dev, void *stream)
{
    if (!h)
        return PAB_EINVAL;
    if (!p_inf_dev)
        return fail(h, PAB_EINVAL, "pab_bubble_step: p_inf_dev is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt))
        return fail(h, PAB_EINVAL, "pab_bubble_step: dt must be positive and finite (got %g)", dt);
    pab::StepArgs a;
    a.p_inf = p_inf_dev;
    a.nb = nb_dev;
    a.dt = dt;
    a.dt_sub = sub_step(h->K, dt);
    a.R = h->R;
    a.V = h->V;
    a.h = h->h;
    a.attempts = h->attempts;
    a.terms = h->terms;
    a.tickets = h->tickets;
    a.G = h->G;
    a.G_valid = h->G_valid;
    a.out = moments_dev;
    a.counters = h->counters;
    a.pb = h->pb;
    a.mv = h->mv;
    cudaError_t e = h->cfg.gas_mode == PAB_GAS_TRANSFER
                        ? pab::launch_transfer_step(h->K, a, h->block_warps, (cudaStream_t)stream)
                        : pab::launch_step(h->K, h->cfg.precision, a, h->block_warps, (cudaStream_t)stream);
    // the moment pass wrote the factors at the new state; without moments they are stale
    h->G_valid = (h->G && moments_dev && e == cudaSuccess) ? 1 : 0;
    if (e != cudaSuccess)
        return cuda_fail(h, e, "pab_bubble_step launch");
    return PAB_OK;
}

pab_status pab_moments(pab_t *h, const double *nb_dev, double *moments_dev, void *stream)
{
    if (!h)
        return PAB_EINVAL;
    if (!moments_dev)
        return fail(h, PAB_EINVAL, "pab_moments: moments_dev is NULL");
    cudaError_t e = h->cfg.gas_mode == PAB_GAS_TRANSFER
                        ? pab::launch_transfer_moments(h->K, nb_dev, h->R, h->V, h->pb, moments_dev,
                                                       h->block_warps, (cudaStream_t)stream)
                        : pab::launch_moments(h->K, h->cfg.precision, nb_dev, h->R, h->V, moments_dev,
                                              h->block_warps, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "pab_moments launch");
    return PAB_OK;
}

pab_status pab_bubble_step_host(pab_t *h, const double *p_inf_host, const double *nb_host, double dt,
                                double *moments_host, void *stream)
{
    if (!h)
        return PAB_EINVAL;
    if (!p_inf_host)
        return fail(h, PAB_EINVAL, "pab_bubble_step_host: p_inf_host is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt))
        return fail(h, PAB_EINVAL, "pab_bubble_step_host: dt must be positive and finite");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t C = (size_t)h->cfg.n_cells;
    cudaError_t e = cudaSuccess;
    if (!h->stage_p)
        e = cudaMallocAsync((void **)&h->stage_p, C * sizeof(double), s);
    if (e == cudaSuccess && nb_host && !h->stage_nb)
        e = cudaMallocAsync((void **)&h->stage_nb, C * sizeof(double), s);
    if (e == cudaSuccess && moments_host && !h->stage_out)
        e = cudaMallocAsync((void **)&h->stage_out, 7 * C * sizeof(double), s);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "pab_bubble_step_host staging");
    e = cudaMemcpyAsync(h->stage_p, p_inf_host, C * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nb_host)
        e = cudaMemcpyAsync(h->stage_nb, nb_host, C * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "pab_bubble_step_host H2D");
    pab_status st = pab_bubble_step(h, h->stage_p, nb_host ? h->stage_nb : nullptr, dt,
                                    moments_host ? h->stage_out : nullptr, stream);
    if (st != PAB_OK)
        return st;
    if (moments_host) {
        e = cudaMemcpyAsync(moments_host, h->stage_out, 7 * C * sizeof(double),
                            cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess)
            return cuda_fail(h, e, "pab_bubble_step_host D2H");
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "pab_bubble_step_host sync");
    return PAB_OK;
}

pab_status pab_status_flags(pab_t *h, uint32_t *flags, int64_t *n_flagged, int64_t *n_attempts,
                            int64_t *n_fp64, void *stream)
{
    if (!h)
        return PAB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h->counters_host, h->counters, sizeof(pab::Counters),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->counters, 0, sizeof(pab::Counters), s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "pab_status_flags");
    const pab::Counters c = *h->counters_host;
    if (flags)
        *flags = c.flags_or;
    if (n_flagged)
        *n_flagged = (int64_t)c.n_flagged;
    if (n_attempts)
        *n_attempts = (int64_t)c.n_attempts;
    if (n_fp64)
        *n_fp64 = (int64_t)c.n_fp64;
    if (c.flags_or & PAB_FLAG_NONFINITE)
        return fail(h, PAB_ENONFINITE, "non-finite pressure or state in %llu bin-steps",
                    (unsigned long long)c.n_flagged);
    if (c.flags_or & PAB_FLAG_STEP_LIMIT)
        return fail(h, PAB_ESTEP_LIMIT, "max_attempts exhausted (%llu flagged bin-steps)",
                    (unsigned long long)c.n_flagged);
    return PAB_OK;
}

pab_status pab_get_state(pab_t *h, double *R_dev, double *Rdot_dev, float *h_dev, void *stream)
{
    if (!h)
        return PAB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = n_state(h);
    cudaError_t e = cudaSuccess;
    if (R_dev)
        e = cudaMemcpyAsync(R_dev, h->R, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && Rdot_dev)
        e = cudaMemcpyAsync(Rdot_dev, h->V, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && h_dev)
        e = cudaMemcpyAsync(h_dev, h->h, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? PAB_OK : cuda_fail(h, e, "pab_get_state");
}

pab_status pab_set_state(pab_t *h, const double *R_dev, const double *Rdot_dev, const float *h_dev,
                         void *stream)
{
    if (!h)
        return PAB_EINVAL;
    if (!R_dev || !Rdot_dev)
        return fail(h, PAB_EINVAL, "pab_set_state: R_dev and Rdot_dev are required");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = n_state(h);
    h->G_valid = 0;  // the carried gas factors belong to the old radii
    cudaError_t e = cudaMemcpyAsync(h->R, R_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->V, Rdot_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && h_dev)
        e = cudaMemcpyAsync(h->h, h_dev, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? PAB_OK : cuda_fail(h, e, "pab_set_state");
}

pab_status pab_get_attempts(pab_t *h, int32_t *attempts_dev, void *stream)
{
    if (!h)
        return PAB_EINVAL;
    if (!h->attempts)
        return fail(h, PAB_ESTATE, "handle was created without record_attempts");
    if (!attempts_dev)
        return fail(h, PAB_EINVAL, "pab_get_attempts: NULL destination");
    cudaError_t e = cudaMemcpyAsync(attempts_dev, h->attempts, n_state(h) * sizeof(int32_t),
                                    cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? PAB_OK : cuda_fail(h, e, "pab_get_attempts");
}

pab_status pab_bin_table(const pab_config *cfg, double *R0_host, double *w_host, double *nb_default)
{
    if (!cfg || !R0_host || !w_host)
        return PAB_EINVAL;
    char msg[256];
    if (validate(cfg, msg, sizeof(msg)) != PAB_OK) {
        fprintf(stderr, "pab_bin_table: %s\n", msg);
        return PAB_EINVAL;
    }
    double R0[PAB_MAX_BINS], w[PAB_MAX_BINS];
    if (!pab::bin_table(cfg, R0, w)) {
        fprintf(stderr, "pab_bin_table: invalid bin table request\n");
        return PAB_EINVAL;
    }
    // the constants a handle of this cfg would hold, so the values are the handle's own
    pab::StepConst K;
    build_const(cfg, R0, w, &K);
    for (int i = 0; i < K.B; ++i) {
        R0_host[i] = K.bins[i].R0;
        w_host[i] = K.bins[i].w;
    }
    if (nb_default)
        *nb_default = K.nb_default;
    return PAB_OK;
}

pab_status pab_gas_table(double gamma, double *tab_host, int64_t capacity, int32_t *n_nodes,
                         int32_t *stride, double *dmax)
{
    if (!finite_pos(gamma) || !n_nodes || !stride || !dmax || capacity < 0)
        return PAB_EINVAL;
    // the bound a handle of this gamma derives, from the same constants builder
    pab_config cfg;
    pab_config_default(&cfg);
    cfg.gamma = gamma;
    double R0[PAB_MAX_BINS], w[PAB_MAX_BINS];
    if (!pab::bin_table(&cfg, R0, w))
        return PAB_EINVAL;
    pab::StepConst K;
    build_const(&cfg, R0, w, &K);
    std::vector<double> tab;
    int J = 0;
    double il2q = 0.0;
    pab::gas_table(3.0 * gamma, K.gas_dmax_tab, &tab, &J, &il2q);
    *n_nodes = 2 * J + 1;
    *stride = pab::kGasTabStride;
    *dmax = K.gas_dmax_tab;
    if (tab_host) {
        if ((size_t)capacity < tab.size())
            return PAB_EINVAL;
        std::memcpy(tab_host, tab.data(), tab.size() * sizeof(double));
    }
    return PAB_OK;
}

pab_status pab_get_bins(const pab_t *h, double *R0_host, double *w_host, double *nb_default)
{
    if (!h)
        return PAB_EINVAL;
    for (int i = 0; i < h->K.B; ++i) {
        if (R0_host)
            R0_host[i] = h->K.bins[i].R0;
        if (w_host)
            w_host[i] = h->K.bins[i].w;
    }
    if (nb_default)
        *nb_default = h->K.nb_default;
    return PAB_OK;
}

pab_status pab_set_block_warps(pab_t *h, int32_t block_warps)
{
    if (!h)
        return PAB_EINVAL;
    if (block_warps < 1 || block_warps > 16)
        return fail(h, PAB_EINVAL, "block_warps must be 1..16");
    h->block_warps = block_warps;
    return PAB_OK;
}

// ---- carrier-facing forms (pab_closure.h) ---------------------------------

pab_status pab_strang_half(pab_t *h, const double *p_inf_dev, const double *nb_dev, double dt_flow,
                           double *moments_dev, void *stream)
{
    if (!h)
        return PAB_EINVAL;
    if (!(dt_flow > 0.0) || !std::isfinite(dt_flow))
        return fail(h, PAB_EINVAL, "pab_strang_half: dt_flow must be positive and finite");
    return pab_bubble_step(h, p_inf_dev, nb_dev, 0.5 * dt_flow, moments_dev, stream);
}

pab_status pab_get_conservative(pab_t *h, const double *nb_dev, double *qR_dev, double *qV_dev,
                                void *stream)
{
    if (!h)
        return PAB_EINVAL;
    if (!qR_dev || !qV_dev)
        return fail(h, PAB_EINVAL, "pab_get_conservative: NULL output");
    cudaError_t e = pab::launch_cons_from_prim(h->K, nb_dev, h->R, h->V, qR_dev, qV_dev,
                                               (cudaStream_t)stream);
    return e == cudaSuccess ? PAB_OK : cuda_fail(h, e, "pab_get_conservative");
}

pab_status pab_set_conservative(pab_t *h, const double *alpha_dev, const double *qR_dev,
                                const double *qV_dev, double *nb_out_dev, void *stream)
{
    if (!h)
        return PAB_EINVAL;
    if (!alpha_dev || !qR_dev || !qV_dev)
        return fail(h, PAB_EINVAL, "pab_set_conservative: NULL input");
    h->G_valid = 0;  // new radii: the carried gas factors are stale
    cudaError_t e = pab::launch_prim_from_cons(h->K, alpha_dev, qR_dev, qV_dev, h->R, h->V, nb_out_dev,
                                               (cudaStream_t)stream);
    return e == cudaSuccess ? PAB_OK : cuda_fail(h, e, "pab_set_conservative");
}

pab_status pab_mixture_pressure(pab_t *h, const double *moments_dev, const double *p_l_dev,
                                const double *rho_l_dev, double *p_dev, void *stream)
{
    if (!h)
        return PAB_EINVAL;
    if (!moments_dev || !p_l_dev || !p_dev)
        return fail(h, PAB_EINVAL, "pab_mixture_pressure: NULL pointer");
    cudaError_t e = pab::launch_mixture_pressure(h->K.C, moments_dev, p_l_dev, rho_l_dev, h->K.rho,
                                                 p_dev, (cudaStream_t)stream);
    return e == cudaSuccess ? PAB_OK : cuda_fail(h, e, "pab_mixture_pressure");
}

pab_status pab_stiffened_gas(int64_t n, const double *rho_l_dev, const double *e_l_dev, double gamma_l,
                             double pi_inf, double *p_l_dev, void *stream)
{
    if (n < 0 || !(gamma_l > 1.0) || !std::isfinite(gamma_l) || !std::isfinite(pi_inf))
        return PAB_EINVAL;
    if (n == 0)
        return PAB_OK;
    if (!rho_l_dev || !e_l_dev || !p_l_dev)
        return PAB_EINVAL;
    cudaError_t e = pab::launch_stiffened_gas(n, rho_l_dev, e_l_dev, gamma_l, pi_inf, p_l_dev,
                                              (cudaStream_t)stream);
    return e == cudaSuccess ? PAB_OK : PAB_ECUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entry point.  Its only scratch, the status block of the
// step kernel, lives in this static device array instead of a handle's
// cudaMalloc'ed memory.  Host code cannot use the array's name as a device
// address, so its address is looked up (cudaGetSymbolAddress) once per CUDA
// context, with that context current, and cached under the context's id: a
// context created anew (after cudaDeviceReset, say) reloads the module, and its
// first call looks the address up again instead of reusing a stale one.
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PAB_NOALLOC_SCRATCH_BYTES];
static_assert(sizeof(pab::Counters) <= PAB_NOALLOC_SCRATCH_BYTES, "status block exceeds the scratch");

constexpr int kNoallocCacheSlots = 64;
struct NoallocSlot {
    unsigned long long ctx_id;
    void *addr;
};
std::mutex g_noalloc_mu;
NoallocSlot g_noalloc_cache[kNoallocCacheSlots] = {};
int g_noalloc_next = 0;
CUresult (*g_cu_ctx_get_current)(CUcontext *) = nullptr;
CUresult (*g_cu_ctx_get_id)(CUcontext, unsigned long long *) = nullptr;

// The current context's id, through the driver entry points the runtime hands out (the
// library links no driver library of its own).  A thread with no current context yet gets
// the device's primary context from the runtime first (the symbol lookup does that).
cudaError_t current_context_id(unsigned long long *id)
{
    if (!g_cu_ctx_get_current || !g_cu_ctx_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                         cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess)
            return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorNotSupported;
        g_cu_ctx_get_current = (CUresult(*)(CUcontext *))f1;
        g_cu_ctx_get_id = (CUresult(*)(CUcontext, unsigned long long *))f2;
    }
    CUcontext ctx = nullptr;
    if (g_cu_ctx_get_current(&ctx) != CUDA_SUCCESS)
        return cudaErrorDeviceUninitialized;
    if (!ctx) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return e;
        if (g_cu_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx)
            return cudaErrorDeviceUninitialized;
    }
    return g_cu_ctx_get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

cudaError_t noalloc_scratch(pab::Counters **out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess)
        return e;
    for (int i = 0; i < kNoallocCacheSlots; ++i)
        if (g_noalloc_cache[i].addr && g_noalloc_cache[i].ctx_id == id) {
            *out = (pab::Counters *)g_noalloc_cache[i].addr;
            return cudaSuccess;
        }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
        return e;
    g_noalloc_cache[g_noalloc_next] = NoallocSlot{id, p};
    g_noalloc_next = (g_noalloc_next + 1) % kNoallocCacheSlots;
    *out = (pab::Counters *)p;
    return cudaSuccess;
}

}  // namespace

extern "C" pab_status pab_bubble_step_noalloc(const pab_config *cfg, const double *p_inf_dev,
                                              const double *nb_dev, double dt, double *R_dev,
                                              double *Rdot_dev, float *h_dev, double *moments_dev,
                                              int64_t *status_dev, void *stream)
{
    if (!cfg || !p_inf_dev || !R_dev || !Rdot_dev)
        return PAB_EINVAL;
    if (!h_dev && cfg->stepper != PAB_FIXED)
        return PAB_EINVAL;
    if (!(dt > 0.0) || !std::isfinite(dt))
        return PAB_EINVAL;
    char msg[256];
    if (validate(cfg, msg, sizeof(msg)) != PAB_OK) {
        fprintf(stderr, "pab_bubble_step_noalloc: %s\n", msg);
        return PAB_EINVAL;
    }
    if (cfg->gas_mode == PAB_GAS_TRANSFER) {
        fprintf(stderr, "pab_bubble_step_noalloc: gas_mode PAB_GAS_TRANSFER needs a handle\n");
        return PAB_EINVAL;
    }
    double R0[PAB_MAX_BINS], w[PAB_MAX_BINS];
    if (!pab::bin_table(cfg, R0, w)) {
        fprintf(stderr, "pab_bubble_step_noalloc: invalid bin table (explicit weights summing to zero?)\n");
        return PAB_EINVAL;
    }
    pab::StepConst K;
    build_const(cfg, R0, w, &K);
    pab::Counters *scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) {
        fprintf(stderr, "pab_bubble_step_noalloc: scratch lookup: %s\n", cudaGetErrorString(e));
        return PAB_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(scratch, 0, sizeof(pab::Counters), s);
    pab::StepArgs a;
    a.p_inf = p_inf_dev;
    a.nb = nb_dev;
    a.dt = dt;
    a.dt_sub = sub_step(K, dt);
    a.R = R_dev;
    a.V = Rdot_dev;
    a.h = h_dev;
    a.attempts = nullptr;
    a.out = moments_dev;
    a.counters = scratch;
    if (e == cudaSuccess)
        e = pab::launch_step(K, cfg->precision, a,
                             cfg->block_warps > 0 ? cfg->block_warps : pab::default_warps(cfg->precision), s);
    if (e == cudaSuccess && status_dev)
        e = cudaMemcpyAsync(status_dev, scratch, sizeof(pab::Counters), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        fprintf(stderr, "pab_bubble_step_noalloc: %s\n", cudaGetErrorString(e));
        return PAB_ECUDA;
    }
    return PAB_OK;
}

extern "C" pab_status pab_check_report(int64_t *count, int32_t *unit, int32_t *line, int64_t *index,
                                       int64_t *bound)
{
    if (count)
        *count = 0;
    if (unit)
        *unit = 0;
    if (line)
        *line = 0;
    if (index)
        *index = 0;
    if (bound)
        *bound = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
        return PAB_ECUDA;
    void (*fetch[])(pab::CheckRecord *, bool) = {pab::check_fetch_kernels, pab::check_fetch_batch,
                                                 pab::check_fetch_closure, pab::check_fetch_el,
                                                 pab::check_fetch_transfer};
    bool reported = false;
    for (int u = 0; u < 5; ++u) {
        pab::CheckRecord r = {0u, 0, 0, 0};
        fetch[u](&r, true);
        if (r.count && !reported) {
            reported = true;
            if (count)
                *count = r.count;
            if (unit)
                *unit = u + 1;
            if (line)
                *line = r.line;
            if (index)
                *index = r.index;
            if (bound)
                *bound = r.bound;
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return PAB_ECUDA;
#ifdef PAB_CHECKED
    return PAB_OK;
#else
    return PAB_ESTATE;
#endif
}

extern "C" pab_status pab_get_contents(pab_t *h, double *pb_dev, double *mv_dev, void *stream)
{
    if (!h)
        return PAB_EINVAL;
    if (h->cfg.gas_mode != PAB_GAS_TRANSFER)
        return fail(h, PAB_EINVAL, "pab_get_contents: the handle has no PAB_GAS_TRANSFER contents");
    const size_t n = n_state(h) * sizeof(double);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (pb_dev)
        e = cudaMemcpyAsync(pb_dev, h->pb, n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && mv_dev)
        e = cudaMemcpyAsync(mv_dev, h->mv, n, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? PAB_OK : cuda_fail(h, e, "pab_get_contents");
}

extern "C" pab_status pab_set_contents(pab_t *h, const double *pb_dev, const double *mv_dev,
                                       void *stream)
{
    if (!h)
        return PAB_EINVAL;
    if (h->cfg.gas_mode != PAB_GAS_TRANSFER)
        return fail(h, PAB_EINVAL, "pab_set_contents: the handle has no PAB_GAS_TRANSFER contents");
    const size_t n = n_state(h) * sizeof(double);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (pb_dev)
        e = cudaMemcpyAsync(h->pb, pb_dev, n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && mv_dev)
        e = cudaMemcpyAsync(h->mv, mv_dev, n, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? PAB_OK : cuda_fail(h, e, "pab_set_contents");
}

extern "C" pab_status pab_host_wait(pab_t *h)
{
    if (!h)
        return PAB_EINVAL;
    for (int i = 0; i < 2; ++i) {
        if (!h->pipe_busy[i])
            continue;
        cudaError_t e = cudaEventSynchronize(h->ev_out[i]);
        if (e != cudaSuccess)
            return cuda_fail(h, e, "pab_host_wait");
        h->pipe_busy[i] = false;
    }
    return PAB_OK;
}

extern "C" pab_status pab_bubble_step_host_async(pab_t *h, const double *p_inf_host, const double *nb_host,
                                                 double dt, double *moments_host, void *stream)
{
    if (!h)
        return PAB_EINVAL;
    if (!p_inf_host)
        return fail(h, PAB_EINVAL, "pab_bubble_step_host_async: p_inf_host is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt))
        return fail(h, PAB_EINVAL, "pab_bubble_step_host_async: dt must be positive and finite");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t C = (size_t)h->cfg.n_cells;
    const int k = h->pipe_next;
    cudaError_t e = cudaSuccess;
    if (!h->pipe_in)
        e = cudaStreamCreateWithFlags(&h->pipe_in, cudaStreamNonBlocking);
    if (e == cudaSuccess && !h->pipe_outs)
        e = cudaStreamCreateWithFlags(&h->pipe_outs, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        if (!h->ev_in[i])
            e = cudaEventCreateWithFlags(&h->ev_in[i], cudaEventDisableTiming);
        if (e == cudaSuccess && !h->ev_step[i])
            e = cudaEventCreateWithFlags(&h->ev_step[i], cudaEventDisableTiming);
        if (e == cudaSuccess && !h->ev_out[i])
            e = cudaEventCreateWithFlags(&h->ev_out[i], cudaEventDisableTiming);
    }
    // the call two before this one used the same staging set and host-side slot
    if (e == cudaSuccess && h->pipe_busy[k]) {
        e = cudaEventSynchronize(h->ev_out[k]);
        h->pipe_busy[k] = false;
    }
    if (e == cudaSuccess && !h->pipe_p[k])
        e = cudaMalloc((void **)&h->pipe_p[k], C * sizeof(double));
    if (e == cudaSuccess && nb_host && !h->pipe_nb[k])
        e = cudaMalloc((void **)&h->pipe_nb[k], C * sizeof(double));
    if (e == cudaSuccess && moments_host && !h->pipe_out[k])
        e = cudaMalloc((void **)&h->pipe_out[k], 7 * C * sizeof(double));
    if (e != cudaSuccess)
        return cuda_fail(h, e, "pab_bubble_step_host_async setup");
    // after a failure past this point nothing of this call may still touch the caller's
    // buffers: wait for whatever of it the copy streams already hold
    auto drain = [h]() {
        cudaStreamSynchronize(h->pipe_in);
        cudaStreamSynchronize(h->pipe_outs);
    };
    e = cudaMemcpyAsync(h->pipe_p[k], p_inf_host, C * sizeof(double), cudaMemcpyHostToDevice, h->pipe_in);
    if (e == cudaSuccess && nb_host)
        e = cudaMemcpyAsync(h->pipe_nb[k], nb_host, C * sizeof(double), cudaMemcpyHostToDevice, h->pipe_in);
    if (e == cudaSuccess)
        e = cudaEventRecord(h->ev_in[k], h->pipe_in);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(s, h->ev_in[k], 0);
    if (e != cudaSuccess) {
        drain();
        return cuda_fail(h, e, "pab_bubble_step_host_async H2D");
    }
    pab_status st = pab_bubble_step(h, h->pipe_p[k], nb_host ? h->pipe_nb[k] : nullptr, dt,
                                    moments_host ? h->pipe_out[k] : nullptr, stream);
    if (st != PAB_OK) {
        drain();
        return st;
    }
    e = cudaEventRecord(h->ev_step[k], s);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(h->pipe_outs, h->ev_step[k], 0);
    if (e == cudaSuccess && moments_host)
        e = cudaMemcpyAsync(moments_host, h->pipe_out[k], 7 * C * sizeof(double), cudaMemcpyDeviceToHost,
                            h->pipe_outs);
    if (e == cudaSuccess)
        e = cudaEventRecord(h->ev_out[k], h->pipe_outs);
    if (e != cudaSuccess) {
        drain();
        return cuda_fail(h, e, "pab_bubble_step_host_async D2H");
    }
    h->pipe_busy[k] = true;
    h->pipe_next = 1 - k;
    return PAB_OK;
}
