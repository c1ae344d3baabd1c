// Batched form of the bubble source update: many independent instances in one
// persistent kernel fed by a device work queue (include/pab_batch.h).
//
// Per step:
//   order kernel   one CTA sorts the active slots by the average cost of their
//                  tiles in the previous step (trials / tiles, stiffest first)
//                  and writes the queue layout: order[j], start[j] (first item
//                  of the j-th slot), the item total, and resets the head;
//   batch kernel   ctas_per_sm x 152 CTAs loop: take the next item (slot,
//                  32-cell tile) from the head counter, stage the slot's
//                  constants in shared memory (only when the slot changes),
//                  then let the warps take bins from a shared counter
//                  (bins_per_grab at a time).  Each bin's four quadrature terms
//                  go to shared memory at its bin index and one warp sums them
//                  in bin order after the CTA barrier, so the moments do not
//                  depend on which warp took which bin.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "pab.h"
#include "pab_batch.h"
#include "pab_check.cuh"
#include "pab_device.cuh"
#include "pab_internal.h"
#include "pab_stream.cuh"

namespace pab {
namespace {

constexpr int kTile = 32;
constexpr int kMaxSlots = 4096;
constexpr int kOrderThreads = 1024;

struct SlotDesc {
    const StepConst *K;  // device copy of the slot's constants
    const double *p_inf;
    const double *nb;
    double *R;
    double *V;
    float *h;
    double *out;
    double dt;
    double dt_sub;       // dt / n_fixed in fixed mode (formed on the host)
    long long C;
    long long n_tiles;
    int B;
    int active;          // admitted and bound
};

struct SlotCounters {
    unsigned int flags_or;
    unsigned int pad;
    unsigned long long n_flagged;
    unsigned long long n_attempts;
    unsigned long long n_fp64;
    unsigned long long step_attempts;  // trials of the step in progress (ordering of the next)
    unsigned long long prev_attempts;  // trials of the previous step
};

struct Queue {
    unsigned long long head;
    long long total;
    int n_order;
    int pad;
};

__host__ __device__ constexpr size_t const_bytes() { return (sizeof(StepConst) + 15) & ~(size_t)15; }

// ---------------------------------------------------------------------------
// Order kernel: bitonic sort of the slots by decreasing tile cost.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kOrderThreads)
    batch_order_kernel(const SlotDesc *__restrict__ slots, SlotCounters *cnt, int max_slots,
                       int *order, long long *start, Queue *q)
{
    __shared__ unsigned int key[kMaxSlots];
    __shared__ int idx[kMaxSlots];
    int n = 1;
    while (n < max_slots)
        n <<= 1;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        unsigned int k = 0;
        if (i < max_slots && slots[i].active) {
            const unsigned long long prev = cnt[i].step_attempts;
            cnt[i].prev_attempts = prev;
            cnt[i].step_attempts = 0;
            const unsigned long long tiles = (unsigned long long)slots[i].n_tiles;
            // average trials per tile (x16); untried slots count one trial per bin-step
            unsigned long long cost =
                prev ? (prev << 4) / tiles : ((unsigned long long)slots[i].B * kTile << 4);
            if (cost > 0xfffffff0ull)
                cost = 0xfffffff0ull;
            k = (unsigned int)cost + 1u;
        }
        key[i] = k;
        idx[i] = i;
    }
    __syncthreads();
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const bool swap = desc ? (key[i] < key[j]) : (key[i] > key[j]);
                    if (swap) {
                        const unsigned int tk = key[i];
                        key[i] = key[j];
                        key[j] = tk;
                        const int ti = idx[i];
                        idx[i] = idx[j];
                        idx[j] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        long long acc = 0;
        int m = 0;
        for (int j = 0; j < n && key[j] != 0; ++j) {
            PAB_ST(order, m, max_slots, idx[j]);
            PAB_ST(start, m, max_slots + 1, acc);
            acc += slots[idx[j]].n_tiles;
            ++m;
        }
        PAB_ST(start, m, max_slots + 1, acc);
        q->head = 0;
        q->total = acc;
        q->n_order = m;
    }
}

// ---------------------------------------------------------------------------
// Pieces of the persistent batch kernel.
// ---------------------------------------------------------------------------
// Advance bin b of cell c over the slot's flow step, store the state and count.
template <bool MIXED>
__device__ __forceinline__ void advance_one(const StepConst &K, const BinConst &bc, const SlotDesc &d,
                                            int b, long long c, double p_inf, const CellTerms &ct,
                                            bool p_ok, double &R, double &V, GasBase &g, uint32_t &fl_or,
                                            uint32_t &n_flag, uint32_t &n_att, uint32_t &n64)
{
    const size_t k = (size_t)b * (size_t)d.C + (size_t)c;
    const long long ns = (long long)d.B * d.C;
    R = PAB_LD(d.R, k, ns);
    V = PAB_LD(d.V, k, ns);
    float hc = PAB_LD(d.h, k, ns);
    int na = 0, nd = 0;
    g.reset();
    const uint32_t fl = advance_bin<MIXED>(K, bc, p_inf, ct, p_ok, d.dt, d.dt_sub, R, V, hc, na, nd, g);
    PAB_ST(d.R, k, ns, R);  // unchanged when the input was not finite
    PAB_ST(d.V, k, ns, V);
    PAB_ST(d.h, k, ns, hc);
    fl_or |= fl;
    n_flag += (fl != 0);
    n_att += na;
    n64 += nd;
}

// One tile's status counts into the slot's counters.
__device__ __forceinline__ void flush_slot(SlotCounters *sc, uint32_t f, unsigned long long a,
                                           unsigned long long t, unsigned long long e)
{
    if (f)
        atomicOr(&sc->flags_or, f);
    if (a)
        atomicAdd(&sc->n_flagged, a);
    if (t) {
        atomicAdd(&sc->n_attempts, t);
        atomicAdd(&sc->step_attempts, t);
    }
    if (e)
        atomicAdd(&sc->n_fp64, e);
}

// ---------------------------------------------------------------------------
// Persistent batch kernel.  A CTA of one warp sums its tile's terms itself and
// needs only the slot's constants in shared memory; wider CTAs stage the terms.
// ---------------------------------------------------------------------------
// ONE_WARP: CTAs of one warp (the autotuner's usual choice) stream the tile's items lane by
// lane; wider CTAs take bins from a shared counter and stage the terms.  Each is its own
// instantiation with its own registers.  At most 72 registers: one-warp CTAs are bounded by
// registers alone (28 fit on an SM at 72); wider CTAs stage the per-bin terms in shared memory
// (about 37 KB per CTA at Nb = 51), which leaves room for 6 CTAs of 4 warps per SM.
#ifndef PAB_BATCH_MAXNREG
#define PAB_BATCH_MAXNREG 72
#endif

template <bool MIXED, bool ONE_WARP>
__global__ void __maxnreg__(PAB_BATCH_MAXNREG)
    batch_kernel(const SlotDesc *__restrict__ slots, const int *__restrict__ order,
                 const long long *__restrict__ start, Queue *q, SlotCounters *cnt,
                 int bins_per_grab, int max_bins, int max_slots)
{
    extern __shared__ __align__(16) unsigned char smem[];
    StepConst &K = *reinterpret_cast<StepConst *>(smem);
    // per-bin quadrature terms in bin order: [max_bins][32] FP64 w R^3, then the other
    // three as [3][max_bins][32], FP32 in MIXED (their sums are FP32 there) and FP64 otherwise
    double *terms = reinterpret_cast<double *>(smem + const_bytes());
    float *terms_f = reinterpret_cast<float *>(terms + (size_t)max_bins * kTile);
    double *terms_d = terms + (size_t)max_bins * kTile;
    __shared__ long long s_item;
    __shared__ int s_j;
    __shared__ int s_next;
    __shared__ unsigned int s_cnt[4][16];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const long long total = q->total;
    const int n_order = q->n_order;
    int staged = -1;

    for (;;) {
        if (threadIdx.x == 0) {
            const long long it = (long long)atomicAdd(&q->head, 1ULL);
            s_item = it;
            if (it < total) {
                int lo = 0, hi = n_order - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (PAB_LD(start, mid, max_slots + 1) <= it)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                s_j = lo;
            }
            s_next = 0;
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= total)
            break;
        const int slot = PAB_LD(order, s_j, max_slots);
        const SlotDesc d = PAB_LD(slots, slot, max_slots);
        if (slot != staged) {
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(d.K);
            unsigned long long *dst = reinterpret_cast<unsigned long long *>(smem);
            for (int i = threadIdx.x; i < (int)(sizeof(StepConst) / 8); i += blockDim.x)
                dst[i] = src[i];
            staged = slot;
            __syncthreads();
        }
        const long long tile = item - PAB_LD(start, s_j, max_slots + 1);
        const long long c = tile * kTile + lane;
        const bool valid = c < d.C;
        const double p_inf = valid ? PAB_LD(d.p_inf, c, d.C) : K.p0;
        const bool p_ok = finite64(p_inf);
        const CellTerms ct = cell_terms<MIXED>(K, p_inf);  // once per cell, not per bin
        uint32_t fl_or = 0, n_flag = 0, n_att = 0, n64 = 0;
        TermSums S;

        if constexpr (ONE_WARP) {
            // one warp: the tile's bins in order, each bin's terms summed as they come, in the
            // order and with the arithmetic of the staged sum below and of the step kernel's
            // closing pass (the same results for every launch shape).  (Streaming the items lane
            // by lane, as the step kernel does, measured slower here: 16.0e9 against 17.6e9
            // bin-steps/s on the 512-instance line, and 11.2e9 with each lane walking its own
            // cell's bins.)
            TileCounts tc;
            for (int b = 0; b < d.B && valid; ++b) {
                const BinConst &bc = K.bins[b];
                double R, V;
                GasBase g;
                advance_one<MIXED>(K, bc, d, b, c, p_inf, ct, p_ok, R, V, g, tc.fl_or, tc.n_flag, tc.n_att, tc.n64);
                if (d.out)
                    add_bin_terms<MIXED>(K, b, R, V, S);
            }
            fl_or = __reduce_or_sync(0xffffffffu, tc.fl_or);
            n_flag = __reduce_add_sync(0xffffffffu, tc.n_flag);
            n_att = __reduce_add_sync(0xffffffffu, tc.n_att);
            n64 = __reduce_add_sync(0xffffffffu, tc.n64);
            if (d.out && valid)
                write_moments<MIXED>(K, d.nb ? PAB_LD(d.nb, c, d.C) : K.nb_default, d.C, c, S, d.out);
            if (lane == 0)
                flush_slot(PAB_AT(cnt, slot, max_slots), fl_or, n_flag, n_att, n64);
            __syncwarp();
            continue;
        }

        for (;;) {
            int b0 = 0;
            if (lane == 0)
                b0 = atomicAdd(&s_next, bins_per_grab);
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            if (b0 >= d.B)
                break;
            const int b1 = min(b0 + bins_per_grab, d.B);
            for (int b = b0; b < b1; ++b) {
                if (!valid)
                    continue;
                const BinConst &bc = K.bins[b];
                double R, V;
                GasBase g;
                advance_one<MIXED>(K, bc, d, b, c, p_inf, ct, p_ok, R, V, g, fl_or, n_flag, n_att, n64);
                if (d.out) {
                    if (MIXED) {
                        float tf[3];
                        terms[(size_t)b * kTile + lane] = quad_terms_mixed(K, bc, R, V, tf);
                        for (int m = 0; m < 3; ++m)
                            terms_f[((size_t)m * max_bins + b) * kTile + lane] = tf[m];
                    } else {
                        double t[4];
                        quad_terms64(K, bc, R, V, t, g);
                        terms[(size_t)b * kTile + lane] = t[0];
                        for (int m = 0; m < 3; ++m)
                            terms_d[((size_t)m * max_bins + b) * kTile + lane] = t[m + 1];
                    }
                }
            }
        }
        fl_or = __reduce_or_sync(0xffffffffu, fl_or);
        n_flag = __reduce_add_sync(0xffffffffu, n_flag);
        n_att = __reduce_add_sync(0xffffffffu, n_att);
        n64 = __reduce_add_sync(0xffffffffu, n64);
        if (lane == 0) {
            s_cnt[0][warp] = fl_or;
            s_cnt[1][warp] = n_flag;
            s_cnt[2][warp] = n_att;
            s_cnt[3][warp] = n64;
        }
        __syncthreads();
        if (warp == 0 && d.out && valid) {
            for (int b = 0; b < d.B; ++b) {
                const double x = terms[(size_t)b * kTile + lane];
                if (MIXED) {
                    const float tf[3] = {terms_f[((size_t)0 * max_bins + b) * kTile + lane],
                                         terms_f[((size_t)1 * max_bins + b) * kTile + lane],
                                         terms_f[((size_t)2 * max_bins + b) * kTile + lane]};
                    add_terms<MIXED>(S, x, tf, nullptr);
                } else {
                    const double td[3] = {terms_d[((size_t)0 * max_bins + b) * kTile + lane],
                                          terms_d[((size_t)1 * max_bins + b) * kTile + lane],
                                          terms_d[((size_t)2 * max_bins + b) * kTile + lane]};
                    add_terms<MIXED>(S, x, nullptr, td);
                }
            }
            write_moments<MIXED>(K, d.nb ? PAB_LD(d.nb, c, d.C) : K.nb_default, d.C, c, S, d.out);
        }
        if (threadIdx.x == 0) {
            uint32_t f = 0;
            unsigned long long a = 0, t = 0, e = 0;
            for (int w = 0; w < nw; ++w) {
                f |= s_cnt[0][w];
                a += s_cnt[1][w];
                t += s_cnt[2][w];
                e += s_cnt[3][w];
            }
            flush_slot(PAB_AT(cnt, slot, max_slots), f, a, t, e);
        }
        __syncthreads();
    }
}

template <bool MIXED>
cudaError_t set_smem_limit(size_t bytes)
{
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<MIXED, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_kernel<MIXED, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes);
    return e;
}

// The batch kernel of a precision and CTA width.
typedef void (*BatchKernelFn)(const SlotDesc *, const int *, const long long *, Queue *, SlotCounters *,
                              int, int, int);
inline BatchKernelFn batch_kernel_fn(bool mixed, bool one_warp)
{
    if (mixed)
        return one_warp ? batch_kernel<true, true> : batch_kernel<true, false>;
    return one_warp ? batch_kernel<false, true> : batch_kernel<false, false>;
}

}  // namespace
}  // namespace pab

PAB_CHECK_UNIT(batch)

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct pab_batch_s {
    pab_batch_config cfg;
    int device = 0;
    cudaStream_t create_stream = nullptr;
    double *R = nullptr;  // arenas [capacity]
    double *V = nullptr;
    float *h = nullptr;
    pab::StepConst *K_dev = nullptr;        // [max_slots]
    pab::StepConst *K_host = nullptr;       // pinned mirror
    pab::SlotDesc *desc_dev = nullptr;      // [max_slots]
    pab::SlotDesc *desc_host = nullptr;     // pinned mirror
    pab::SlotCounters *cnt_dev = nullptr;   // [max_slots]
    pab::SlotCounters *cnt_host = nullptr;  // pinned, one entry
    int *order = nullptr;                   // [max_slots]
    long long *start = nullptr;             // [max_slots + 1]
    pab::Queue *queue = nullptr;
    std::vector<int> admitted;              // 1 if the slot holds an instance
    std::vector<long long> offset;          // arena offset of each slot
    std::vector<long long> size;            // bin-states of each slot
    std::map<long long, long long> free_ranges;  // offset -> length
    // gas-term node tables shared by the slots of one 3 gamma (keyed by its bit
    // pattern), kept until the batch is destroyed
    struct GasTab {
        double *dev;
        int J;
        double inv_log2q;
    };
    std::map<unsigned long long, GasTab> gas_tabs;
    long long used = 0;
    size_t smem_bytes = 0;
    int block_warps = 8;
    int ctas_per_sm = 0;
    int bins_per_grab = 1;
    int n_sm = 152;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t capture_stream = nullptr;  // the legacy default stream cannot be captured
    // A step copies the slot table from desc_host when it runs, not when it is enqueued, so
    // the table may be rewritten only after the last enqueued step has finished: each step
    // records ev_step, and whatever rewrites the table waits for it first.
    cudaEvent_t ev_step = nullptr;
    bool step_pending = false;
    char err[512] = {0};
};

namespace {

pab_status bfail(pab_batch_t *b, pab_status s, const char *fmt, ...)
{
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

pab_status bcuda(pab_batch_t *b, cudaError_t e, const char *what)
{
    return bfail(b, e == cudaErrorMemoryAllocation ? PAB_ENOMEM : PAB_ECUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

void drop_graph(pab_batch_t *b)
{
    if (b->graph_exec)
        cudaGraphExecDestroy(b->graph_exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
}

// First fit in the free list; returns -1 when nothing fits.
long long arena_take(pab_batch_t *b, long long n)
{
    for (auto it = b->free_ranges.begin(); it != b->free_ranges.end(); ++it) {
        if (it->second >= n) {
            const long long off = it->first;
            const long long rest = it->second - n;
            b->free_ranges.erase(it);
            if (rest > 0)
                b->free_ranges[off + n] = rest;
            b->used += n;
            return off;
        }
    }
    return -1;
}

void arena_give(pab_batch_t *b, long long off, long long n)
{
    auto it = b->free_ranges.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != b->free_ranges.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        b->free_ranges.erase(nx);
    }
    if (it != b->free_ranges.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            b->free_ranges.erase(it);
        }
    }
    b->used -= n;
}

// Dynamic shared memory of a launch: the slot's constants, and for CTAs of more
// than one warp the per-bin terms of a tile too.
size_t launch_smem(const pab_batch_t *b)
{
    if (b->block_warps == 1)
        return pab::const_bytes();
    return b->smem_bytes;
}

int resident_ctas(const pab_batch_t *b)
{
    int per_sm = 0;
    const int threads = b->block_warps * 32;
    cudaError_t e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, pab::batch_kernel_fn(b->cfg.precision == PAB_MIXED, b->block_warps == 1), threads,
        launch_smem(b));
    if (e != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int want = b->ctas_per_sm > 0 ? b->ctas_per_sm : 4;
    return std::min(want, per_sm) * b->n_sm;
}

cudaError_t enqueue_step(pab_batch_t *b, cudaStream_t s, int grid)
{
    const int ms = b->cfg.max_slots;
    cudaError_t e = cudaMemcpyAsync(b->desc_dev, b->desc_host, sizeof(pab::SlotDesc) * ms,
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return e;
    pab::batch_order_kernel<<<1, pab::kOrderThreads, 0, s>>>(b->desc_dev, b->cnt_dev, ms, b->order,
                                                               b->start, b->queue);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const int threads = b->block_warps * 32;
    const int maxb = b->cfg.max_bins;
    pab::batch_kernel_fn(b->cfg.precision == PAB_MIXED, b->block_warps == 1)<<<grid, threads,
                                                                              launch_smem(b), s>>>(
        b->desc_dev, b->order, b->start, b->queue, b->cnt_dev, b->bins_per_grab, maxb, b->cfg.max_slots);
    return cudaGetLastError();
}

bool valid_slot(const pab_batch_t *b, int slot)
{
    return slot >= 0 && slot < b->cfg.max_slots && b->admitted[slot];
}

// Wait until the last enqueued step has finished (it reads the slot tables when it runs).
cudaError_t wait_last_step(pab_batch_t *b)
{
    if (!b->step_pending)
        return cudaSuccess;
    const cudaError_t e = cudaEventSynchronize(b->ev_step);
    if (e == cudaSuccess)
        b->step_pending = false;
    return e;
}

// Mark a step enqueued on s.  A step enqueued into the caller's own stream capture is not
// marked: it runs when the caller launches that graph, which the caller orders.
cudaError_t mark_step(pab_batch_t *b, cudaStream_t s)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return e;
    e = cudaEventRecord(b->ev_step, s);
    if (e == cudaSuccess)
        b->step_pending = true;
    return e;
}

}  // namespace

extern "C" {

void pab_batch_config_default(pab_batch_config *c)
{
    if (!c)
        return;
    std::memset(c, 0, sizeof(*c));
    c->max_slots = 512;
    c->precision = PAB_MIXED;
    c->capacity_bins = 0;
    c->block_warps = 8;
    c->ctas_per_sm = 0;
    c->bins_per_grab = 1;
    c->max_bins = PAB_MAX_BINS;
}

const char *pab_batch_last_error(const pab_batch_t *b) { return b ? b->err : "NULL batch"; }

pab_status pab_batch_create(const pab_batch_config *cfg, void *stream, pab_batch_t **out)
{
    if (!out)
        return PAB_EINVAL;
    *out = nullptr;
    if (!cfg || cfg->max_slots < 1 || cfg->max_slots > pab::kMaxSlots ||
        (cfg->precision != PAB_FP64 && cfg->precision != PAB_MIXED) || cfg->capacity_bins < 0 ||
        cfg->capacity_bins > PAB_MAX_CELLS * PAB_MAX_BINS ||
        cfg->block_warps < 0 || cfg->block_warps > 16 || cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > 32 ||
        cfg->bins_per_grab < 0 || cfg->bins_per_grab > 8 || cfg->max_bins < 0 ||
        cfg->max_bins > PAB_MAX_BINS) {
        fprintf(stderr, "pab_batch_create: invalid batch configuration\n");
        return PAB_EINVAL;
    }
    pab_batch_t *b = new (std::nothrow) pab_batch_t();
    if (!b)
        return PAB_ENOMEM;
    b->cfg = *cfg;
    if (b->cfg.max_bins == 0)
        b->cfg.max_bins = PAB_MAX_BINS;
    b->block_warps = cfg->block_warps > 0 ? cfg->block_warps : 8;
    b->ctas_per_sm = cfg->ctas_per_sm;
    b->bins_per_grab = cfg->bins_per_grab > 0 ? cfg->bins_per_grab : 1;
    b->create_stream = (cudaStream_t)stream;
    cudaStream_t s = b->create_stream;
    const int ms = b->cfg.max_slots;
    b->admitted.assign(ms, 0);
    b->offset.assign(ms, 0);
    b->size.assign(ms, 0);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device);
    long long cap = b->cfg.capacity_bins;
    if (e == cudaSuccess && cap == 0) {
        size_t free_b = 0, total_b = 0;
        e = cudaMemGetInfo(&free_b, &total_b);
        cap = (long long)((double)free_b * 0.8 / 20.0);
    }
    b->cfg.capacity_bins = cap;
    if (e == cudaSuccess && cap < 1)
        e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&b->R, (size_t)cap * sizeof(double), s);
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&b->V, (size_t)cap * sizeof(double), s);
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&b->h, (size_t)cap * sizeof(float), s);
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&b->K_dev, sizeof(pab::StepConst) * ms, s);
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&b->desc_dev, sizeof(pab::SlotDesc) * ms, s);
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&b->cnt_dev, sizeof(pab::SlotCounters) * ms, s);
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&b->order, sizeof(int) * ms, s);
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&b->start, sizeof(long long) * (ms + 1), s);
    if (e == cudaSuccess)
        e = cudaMallocAsync((void **)&b->queue, sizeof(pab::Queue), s);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&b->ev_step, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&b->K_host, sizeof(pab::StepConst) * ms);
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&b->desc_host, sizeof(pab::SlotDesc) * ms);
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&b->cnt_host, sizeof(pab::SlotCounters));
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->cnt_dev, 0, sizeof(pab::SlotCounters) * ms, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->queue, 0, sizeof(pab::Queue), s);
    if (e == cudaSuccess) {
        std::memset(b->desc_host, 0, sizeof(pab::SlotDesc) * ms);
        b->free_ranges[0] = cap;
        b->smem_bytes = pab::const_bytes() + (size_t)b->cfg.max_bins * pab::kTile * sizeof(double) +
                        (size_t)3 * b->cfg.max_bins * pab::kTile *
                            (cfg->precision == PAB_MIXED ? sizeof(float) : sizeof(double));
        const size_t limit = b->smem_bytes;
        e = cfg->precision == PAB_MIXED ? pab::set_smem_limit<true>(limit)
                                        : pab::set_smem_limit<false>(limit);
    }
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        fprintf(stderr, "pab_batch_create: %s\n", cudaGetErrorString(e));
        pab_status st = e == cudaErrorMemoryAllocation ? PAB_ENOMEM : PAB_ECUDA;
        cudaGetLastError();
        pab_batch_destroy(b);
        return st;
    }
    *out = b;
    return PAB_OK;
}

void pab_batch_destroy(pab_batch_t *b)
{
    if (!b)
        return;
    drop_graph(b);
    cudaStream_t s = b->create_stream;
    cudaStreamSynchronize(s);
    void *dev[] = {b->R, b->V, b->h, b->K_dev, b->desc_dev, b->cnt_dev, b->order, b->start, b->queue};
    for (void *p : dev)
        if (p)
            cudaFreeAsync(p, s);
    for (auto &kv : b->gas_tabs)
        cudaFreeAsync(kv.second.dev, s);
    cudaStreamSynchronize(s);
    void *host[] = {b->K_host, b->desc_host, b->cnt_host};
    for (void *p : host)
        if (p)
            cudaFreeHost(p);
    if (b->capture_stream)
        cudaStreamDestroy(b->capture_stream);
    if (b->ev_step)
        cudaEventDestroy(b->ev_step);
    delete b;
}

pab_status pab_batch_admit(pab_batch_t *b, const pab_config *cfg, void *stream, int32_t *slot)
{
    if (!b || !cfg || !slot)
        return PAB_EINVAL;
    char msg[256];
    if (pab::validate_config(cfg, msg, sizeof(msg)) != PAB_OK)
        return bfail(b, PAB_EINVAL, "pab_batch_admit: %s", msg);
    if (cfg->gas_mode == PAB_GAS_TRANSFER)
        return bfail(b, PAB_EINVAL, "pab_batch_admit: gas_mode PAB_GAS_TRANSFER is not batched");
    if (cfg->n_bins > b->cfg.max_bins)
        return bfail(b, PAB_EINVAL, "pab_batch_admit: n_bins %d above the batch's max_bins %d",
                     cfg->n_bins, b->cfg.max_bins);
    double R0[PAB_MAX_BINS], w[PAB_MAX_BINS];
    if (!pab::bin_table(cfg, R0, w))
        return bfail(b, PAB_EINVAL, "pab_batch_admit: invalid bin table");
    int s_idx = -1;
    for (int i = 0; i < b->cfg.max_slots; ++i)
        if (!b->admitted[i]) {
            s_idx = i;
            break;
        }
    if (s_idx < 0)
        return bfail(b, PAB_ENOMEM, "pab_batch_admit: all %d slots are in use", b->cfg.max_slots);
    const long long n = (long long)cfg->n_bins * cfg->n_cells;
    const long long off = arena_take(b, n);
    if (off < 0)
        return bfail(b, PAB_ENOMEM, "pab_batch_admit: %lld bin-states do not fit (%lld of %lld in use)",
                     n, b->used, (long long)b->cfg.capacity_bins);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = wait_last_step(b);  // no step in flight reads the slot tables
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    pab::StepConst &K = b->K_host[s_idx];
    pab::make_const(cfg, R0, w, &K);
    std::vector<double> tab;  // host values of a new gas table, alive until the sync below
    if (e == cudaSuccess && cfg->gas_mode == PAB_GAS_POLYTROPIC) {
        const double a = 3.0 * cfg->gamma;
        unsigned long long key;
        std::memcpy(&key, &a, sizeof(key));
        auto it = b->gas_tabs.find(key);
        if (it == b->gas_tabs.end()) {
            pab_batch_s::GasTab t{nullptr, 0, 0.0};
            pab::gas_table(a, K.gas_dmax_tab, &tab, &t.J, &t.inv_log2q);
            e = cudaMallocAsync((void **)&t.dev, tab.size() * sizeof(double), s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(t.dev, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                it = b->gas_tabs.emplace(key, t).first;
            else if (t.dev)
                cudaFreeAsync(t.dev, s);
        }
        if (e == cudaSuccess) {
            K.gas_tab = it->second.dev;
            K.gas_J = it->second.J;
            K.gas_inv_log2q = (float)it->second.inv_log2q;
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->K_dev + s_idx, &K, sizeof(pab::StepConst), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = pab::launch_init(K, cfg->Rdot0_ref, cfg->R0ref, b->R + off, b->V + off, b->h + off, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->cnt_dev + s_idx, 0, sizeof(pab::SlotCounters), s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        arena_give(b, off, n);
        return bcuda(b, e, "pab_batch_admit");
    }
    pab::SlotDesc &d = b->desc_host[s_idx];
    std::memset(&d, 0, sizeof(d));
    d.K = b->K_dev + s_idx;
    d.R = b->R + off;
    d.V = b->V + off;
    d.h = b->h + off;
    d.C = cfg->n_cells;
    d.B = cfg->n_bins;
    d.n_tiles = (cfg->n_cells + pab::kTile - 1) / pab::kTile;
    d.active = 0;  // until bound
    b->admitted[s_idx] = 1;
    b->offset[s_idx] = off;
    b->size[s_idx] = n;
    *slot = s_idx;
    return PAB_OK;
}

pab_status pab_batch_bind(pab_batch_t *b, int32_t slot, const double *p_inf_dev, const double *nb_dev,
                          double *moments_dev, double dt)
{
    if (!b)
        return PAB_EINVAL;
    if (!valid_slot(b, slot))
        return bfail(b, PAB_EINVAL, "pab_batch_bind: slot %d is not admitted", slot);
    if (!p_inf_dev)
        return bfail(b, PAB_EINVAL, "pab_batch_bind: p_inf_dev is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt))
        return bfail(b, PAB_EINVAL, "pab_batch_bind: dt must be positive and finite");
    const cudaError_t e = wait_last_step(b);
    if (e != cudaSuccess)
        return bcuda(b, e, "pab_batch_bind");
    pab::SlotDesc &d = b->desc_host[slot];
    d.p_inf = p_inf_dev;
    d.nb = nb_dev;
    d.out = moments_dev;
    d.dt = dt;
    d.dt_sub = b->K_host[slot].n_fixed > 0 ? dt / (double)b->K_host[slot].n_fixed : 0.0;
    d.active = 1;
    return PAB_OK;
}

pab_status pab_batch_release(pab_batch_t *b, int32_t slot, void *stream)
{
    if (!b)
        return PAB_EINVAL;
    if (!valid_slot(b, slot))
        return bfail(b, PAB_EINVAL, "pab_batch_release: slot %d is not admitted", slot);
    cudaError_t e = wait_last_step(b);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess)
        return bcuda(b, e, "pab_batch_release");
    std::memset(&b->desc_host[slot], 0, sizeof(pab::SlotDesc));
    arena_give(b, b->offset[slot], b->size[slot]);
    b->admitted[slot] = 0;
    b->size[slot] = 0;
    return PAB_OK;
}

pab_status pab_batch_step(pab_batch_t *b, void *stream)
{
    if (!b)
        return PAB_EINVAL;
    cudaError_t e = enqueue_step(b, (cudaStream_t)stream, resident_ctas(b));
    if (e == cudaSuccess)
        e = mark_step(b, (cudaStream_t)stream);
    return e == cudaSuccess ? PAB_OK : bcuda(b, e, "pab_batch_step");
}

pab_status pab_batch_step_graph(pab_batch_t *b, void *stream)
{
    if (!b)
        return PAB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!b->graph_exec) {
        // capture on the batch's own stream, replay into the caller's
        const int grid = resident_ctas(b);
        cudaStream_t cs = b->capture_stream;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue_step(b, cs, grid);
            e = cudaStreamEndCapture(cs, &b->graph);
            if (e2 != cudaSuccess)
                e = e2;
        }
        if (e == cudaSuccess)
            e = cudaGraphInstantiate(&b->graph_exec, b->graph, 0);
        if (e != cudaSuccess) {
            drop_graph(b);
            cudaGetLastError();
            return bcuda(b, e, "pab_batch_step_graph capture");
        }
    }
    e = cudaGraphLaunch(b->graph_exec, s);
    if (e == cudaSuccess)
        e = mark_step(b, s);
    return e == cudaSuccess ? PAB_OK : bcuda(b, e, "pab_batch_step_graph launch");
}

pab_status pab_batch_status(pab_batch_t *b, int32_t slot, uint32_t *flags, int64_t *n_flagged,
                            int64_t *n_attempts, int64_t *n_fp64, void *stream)
{
    if (!b)
        return PAB_EINVAL;
    if (!valid_slot(b, slot))
        return bfail(b, PAB_EINVAL, "pab_batch_status: slot %d is not admitted", slot);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(b->cnt_host, b->cnt_dev + slot, sizeof(pab::SlotCounters),
                                    cudaMemcpyDeviceToHost, s);
    // reset the read counters, keep the trial history that orders the queue
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->cnt_dev + slot, 0, offsetof(pab::SlotCounters, step_attempts), s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return bcuda(b, e, "pab_batch_status");
    const pab::SlotCounters c = *b->cnt_host;
    if (flags)
        *flags = c.flags_or;
    if (n_flagged)
        *n_flagged = (int64_t)c.n_flagged;
    if (n_attempts)
        *n_attempts = (int64_t)c.n_attempts;
    if (n_fp64)
        *n_fp64 = (int64_t)c.n_fp64;
    if (c.flags_or & PAB_FLAG_NONFINITE)
        return bfail(b, PAB_ENONFINITE, "slot %d: non-finite pressure or state", slot);
    if (c.flags_or & PAB_FLAG_STEP_LIMIT)
        return bfail(b, PAB_ESTEP_LIMIT, "slot %d: max_attempts exhausted", slot);
    return PAB_OK;
}

pab_status pab_batch_get_state(pab_batch_t *b, int32_t slot, double *R_dev, double *Rdot_dev,
                               float *h_dev, void *stream)
{
    if (!b)
        return PAB_EINVAL;
    if (!valid_slot(b, slot))
        return bfail(b, PAB_EINVAL, "pab_batch_get_state: slot %d is not admitted", slot);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)b->size[slot];
    const long long off = b->offset[slot];
    cudaError_t e = cudaSuccess;
    if (R_dev)
        e = cudaMemcpyAsync(R_dev, b->R + off, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && Rdot_dev)
        e = cudaMemcpyAsync(Rdot_dev, b->V + off, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && h_dev)
        e = cudaMemcpyAsync(h_dev, b->h + off, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? PAB_OK : bcuda(b, e, "pab_batch_get_state");
}

pab_status pab_batch_set_state(pab_batch_t *b, int32_t slot, const double *R_dev, const double *Rdot_dev,
                               const float *h_dev, void *stream)
{
    if (!b)
        return PAB_EINVAL;
    if (!valid_slot(b, slot))
        return bfail(b, PAB_EINVAL, "pab_batch_set_state: slot %d is not admitted", slot);
    if (!R_dev || !Rdot_dev)
        return bfail(b, PAB_EINVAL, "pab_batch_set_state: R_dev and Rdot_dev are required");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)b->size[slot];
    const long long off = b->offset[slot];
    cudaError_t e = cudaMemcpyAsync(b->R + off, R_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->V + off, Rdot_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && h_dev)
        e = cudaMemcpyAsync(b->h + off, h_dev, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? PAB_OK : bcuda(b, e, "pab_batch_set_state");
}

pab_status pab_batch_usage(const pab_batch_t *b, int32_t *active_slots, int64_t *bins_used,
                           int64_t *capacity_bins)
{
    if (!b)
        return PAB_EINVAL;
    int n = 0;
    for (int v : b->admitted)
        n += v;
    if (active_slots)
        *active_slots = n;
    if (bins_used)
        *bins_used = b->used;
    if (capacity_bins)
        *capacity_bins = b->cfg.capacity_bins;
    return PAB_OK;
}

pab_status pab_batch_set_launch(pab_batch_t *b, int32_t block_warps, int32_t ctas_per_sm,
                                int32_t bins_per_grab)
{
    if (!b)
        return PAB_EINVAL;
    if (block_warps < 1 || block_warps > 16 || ctas_per_sm < 1 || ctas_per_sm > 32 ||
        bins_per_grab < 1 || bins_per_grab > 8)
        return bfail(b, PAB_EINVAL, "pab_batch_set_launch: out of range");
    b->block_warps = block_warps;
    b->ctas_per_sm = ctas_per_sm;
    b->bins_per_grab = bins_per_grab;
    drop_graph(b);
    return PAB_OK;
}

}  // extern "C"
