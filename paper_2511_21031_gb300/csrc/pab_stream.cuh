// Lane-streamed advance of a tile's (cell, bin) items, and the tile's moments.
//
// A tile is 32 consecutive cells and a range of their bins: (bins x cells)
// items, each one (bin, cell) state to carry over one flow step.  The items
// form a pool in bin-major order (item j: bin j / nc, cell j % nc), so lanes
// that take items together read consecutive cells of one bin.  Every lane
// holds one item at a time and runs one trial of it per loop iteration; a lane
// whose item is finished takes the next item of the pool at the end of the
// iteration instead of waiting for the other lanes' items.  The warp's time is
// then about the tile's trials over 32 rather than the sum over bins of the
// slowest lane's trials, which the stiff bins of a collapse make much larger
// (growth and collapse put very different trial counts on neighbouring cells).
//
// A CTA's warps share one pool (its tiles' items) through a shared counter.
//
// In mixed precision a bin near collapse takes FP64 trials, several times the
// cost of an FP32 trial on GB300's narrow FP64 pipe; a warp in which a few
// lanes take one pays it for all 32.  So while the pool still holds items, a
// lane whose next trial is FP64 parks its item (controller state and all) in
// the CTA's lot in shared memory and takes another; once every warp has
// emptied the pool, the warps resume the parked items of all of them, whose
// FP64 trials then run on fuller warps.  Each item's own sequence of trials is
// the same whatever the schedule, so the state is the same bits in every
// launch shape.
//
// The moments are a separate pass over the tile after every item is done: one
// lane per cell reads its bins' new state back (from L2) and sums the
// quadrature terms in bin order, which no schedule can change.
#pragma once

#include <cuda_runtime.h>

#include "pab_check.cuh"
#include "pab_device.cuh"
#include "pab_internal.h"

namespace pab {

constexpr int kLotPerWarp = 32;  // parked items per warp of the CTA (mixed precision)

// The CTA's lot of parked items in shared memory (Parked entries, pab_internal.h).
__host__ __device__ constexpr size_t lot_bytes(int cap) { return (size_t)cap * sizeof(Parked); }

// The CTA's shared counters: the next pool item, the items parked, the parked items resumed.
// Zero before the first call.
struct PoolCounters {
    int next, lot_n, lot_take;
};

// Where a tile's items live and what they advance over.
struct TileIO {
    const double *p_inf;  // [C]
    double *R, *V;        // [B][C]
    float *h;             // [B][C]
    int32_t *attempts;    // [B][C] or nullptr
    long long C;          // cells (stride between bins)
    long long c0;         // first cell of the CTA's tiles
    int nc;               // cells of the CTA (1..32 x warps)
    int b0, b1;           // bins [b0, b1)
    double dt;            // flow step
    // per cell of the CTA (index c - c0), formed once before the items: B0 = (pv - p_inf)/rho
    // and B0/c (FP64 items), the FP32 image of p0 - p_inf (mixed items)
    const double *cB0 = nullptr, *cB0c = nullptr;
    const float *cA0 = nullptr;
    // [B][C] the gas factor at the stored radii, from the previous flow step's moment pass
    // (FP64 items; nullptr: evaluated afresh)
    const double *G = nullptr;
};

// Status of the items a lane finished.
struct TileCounts {
    uint32_t fl_or = 0, n_flag = 0, n_att = 0, n64 = 0;
};

// The FP32 constants of one bin the FP32 right-hand side reads, held in registers while the
// lane's item is of that bin (accel32, incr32 and gas_dev32 take any type with these fields).
struct Bin32 {
    float R0f, invR0f, pg0f;
};

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Consecutive positions of a shared counter for the lanes in `want`, in lane order (one atomic
// per warp).  The whole warp calls it; returns -1 for the other lanes.  `done` turns true once
// a grab reaches `total`.
__device__ __forceinline__ int grab(unsigned want, int total, int *counter, bool &done)
{
    const int lane = threadIdx.x & 31;
    const int cnt = __popc(want);
    int base = 0;
    if (lane == 0)
        base = atomicAdd(counter, cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base + cnt >= total)
        done = true;
    return ((want >> lane) & 1u) ? base + __popc(want & lanemask_lt()) : -1;
}

// Item j of the tile: its bin and the state index of its cell.
__device__ __forceinline__ void item_of(const TileIO &io, int j, int &b, int &cl, size_t &k)
{
    if ((io.nc & (io.nc - 1)) == 0) {
        const int lg = __ffs(io.nc) - 1;
        b = io.b0 + (j >> lg);
        cl = j & (io.nc - 1);
    } else {
        const int q = j / io.nc;
        b = io.b0 + q;
        cl = j - q * io.nc;
    }
    k = (size_t)b * (size_t)io.C + (size_t)(io.c0 + cl);
}

// ---------------------------------------------------------------------------
// FP64: one lane's item with the controller of advance_adaptive, one trial per
// call.
// ---------------------------------------------------------------------------
struct Item64 {
    int b;
    long long c;
    size_t k;
    BinConst bc;
    double B0, B0c, R, V, h, rem;
    double Gy;  // the gas factor at the current state, when haveG
    bool haveG;
    int n;
    uint32_t fl;
    GasBase g;

    // The start of the flow step from the stored state.  A non-finite input is flagged and
    // counted and left as it is (false: nothing to advance).
    __device__ __forceinline__ bool start(const StepConst &K, const TileIO &io, int b_, long long c_,
                                          TileCounts &tc)
    {
        b = b_;
        c = c_;
        k = (size_t)b * (size_t)io.C + (size_t)c;
        bc = K.bins[b];
        const long long ns = (long long)K.B * io.C;  // state length
        const double p_inf = PAB_LD(io.p_inf, c, io.C);
        R = PAB_LD(io.R, k, ns);
        V = PAB_LD(io.V, k, ns);
        const float hc = PAB_LD(io.h, k, ns);
        g.reset();
        n = 0;
        fl = 0;
        if (!finite64(p_inf) || !finite64(R) || !finite64(V)) {
            if (io.attempts)
                PAB_ST(io.attempts, k, ns, 0);
            tc.fl_or |= PAB_FLAG_NONFINITE;
            tc.n_flag += 1;
            return false;
        }
        B0 = io.cB0[c - io.c0];
        B0c = io.cB0c[c - io.c0];
        haveG = io.G != nullptr;
        Gy = haveG ? PAB_LD(io.G, k, ns) : 0.0;
        h = start_h(hc, io.dt);
        rem = io.dt;
        return true;
    }

    // One trial and the controller; true when the flow step is done.
    __device__ __forceinline__ bool trial(const StepConst &K)
    {
        if (n >= K.max_attempts) {
            fl |= PAB_FLAG_STEP_LIMIT;
            return true;
        }
        bool done = false;
        const bool last = le(rem, h);
        const double ht = last ? rem : h;
        double G0;
        const Trial tr = trial64(K, bc, B0, B0c, R, V, ht, g, haveG, Gy, G0);
        ++n;
        const Decision vd = decide64(K, tr);
        const double fac = f2d_fin(vd.fac);
        // a rejected trial leaves the state, and so its gas factor, as they were
        haveG = !vd.accept;
        Gy = G0;
        if (vd.accept) {
            R = tr.R;
            V = tr.V;
            if (last) {
                const bool clipped = !le(h, rem);
                h = (clipped && vd.fac >= 1.0f) ? h : ht * fac;
                done = true;
            } else {
                rem -= ht;
                h = ht * fac;
            }
        } else {
            h = ht * fac;
        }
        if (!done && n >= K.max_attempts) {
            fl |= PAB_FLAG_STEP_LIMIT;
            done = true;
        }
        return done;
    }

    __device__ __forceinline__ void finish(const StepConst &K, const TileIO &io, TileCounts &tc)
    {
        if (!finite64(R) || !finite64(V))
            fl |= PAB_FLAG_NONFINITE;
        else if (!gt0(R))
            fl |= PAB_FLAG_NONPOS;
        if (abs_ge(V, K.c))
            fl |= PAB_FLAG_SUPERSONIC;
        const long long ns = (long long)K.B * io.C;
        PAB_ST(io.R, k, ns, R);
        PAB_ST(io.V, k, ns, V);
        PAB_ST(io.h, k, ns, d2f(h));
        if (io.attempts)
            PAB_ST(io.attempts, k, ns, n);
        tc.fl_or |= fl;
        tc.n_flag += (fl != 0);
        tc.n_att += n;
    }
};

// The CTA's pool streamed lane by lane.
__device__ __forceinline__ void stream_fp64(const StepConst &K, const TileIO &io, PoolCounters &sh,
                                            TileCounts &tc)
{
    const int total = (io.b1 - io.b0) * io.nc;
    bool exhausted = total <= 0;
    bool have = false;
    Item64 it;
    for (;;) {
        const unsigned want = __ballot_sync(0xffffffffu, !have);
        if (want && !exhausted) {
            const int j = grab(want, total, &sh.next, exhausted);
            if (j >= 0 && j < total) {
                int b, cl;
                size_t k;
                item_of(io, j, b, cl, k);
                have = it.start(K, io, b, io.c0 + cl, tc);
            }
        }
        if (!__any_sync(0xffffffffu, have)) {
            if (exhausted)
                break;
            continue;
        }
        if (have && it.trial(K)) {
            it.finish(K, io, tc);
            have = false;
        }
    }
}

// ---------------------------------------------------------------------------
// Mixed precision: one lane's item with the controller of advance_mixed, one
// trial per call.
// ---------------------------------------------------------------------------
struct ItemMixed {
    int b;
    long long c;
    size_t k;
    Bin32 bf;
    float A;  // p_eq - p_inf of the item's bin and cell
    double xi64, V, h, rem;
    float xi, v;
    int n, n64;
    uint32_t fl;

    // The constants of bin b_ at cell c_; returns the cell's pressure.
    __device__ __forceinline__ double bind(const StepConst &K, const TileIO &io, int b_, long long c_)
    {
        b = b_;
        c = c_;
        k = (size_t)b * (size_t)io.C + (size_t)c;
        const BinConst &bc = K.bins[b];
        bf.R0f = bc.R0f;
        bf.invR0f = bc.invR0f;
        bf.pg0f = bc.pg0f;
        const double p_inf = PAB_LD(io.p_inf, c, io.C);
        A = bc.dpeqf + io.cA0[c - io.c0];
        return p_inf;
    }

    // The start of the flow step from the stored state.  A non-finite input is flagged and
    // counted and left as it is (false: nothing to advance).
    __device__ __forceinline__ bool start(const StepConst &K, const TileIO &io, int b_, long long c_,
                                          TileCounts &tc)
    {
        const double p_inf = bind(K, io, b_, c_);
        const long long ns = (long long)K.B * io.C;
        const double R = PAB_LD(io.R, k, ns);
        V = PAB_LD(io.V, k, ns);
        const float hc = PAB_LD(io.h, k, ns);
        n = 0;
        n64 = 0;
        fl = 0;
        if (!finite64(p_inf) || !finite64(R) || !finite64(V)) {
            if (io.attempts)
                PAB_ST(io.attempts, k, ns, 0);
            tc.fl_or |= PAB_FLAG_NONFINITE;
            tc.n_flag += 1;
            return false;
        }
        h = start_h(hc, io.dt);
        rem = io.dt;
        xi64 = R - K.bins[b].R0;
        xi = d2f(xi64);
        v = d2f(V);
        return true;
    }

    // Near collapse (R/R0 < r_collapse or |Rdot| > v_collapse): the next trial is FP64.
    __device__ __forceinline__ bool near_collapse(const StepConst &K) const
    {
        return xi < (K.r_collapsef - 1.0f) * bf.R0f || fabsf(v) > K.v_collapsef;
    }

    __device__ __forceinline__ void save(Parked &P) const
    {
        P.xi64 = xi64;
        P.V = V;
        P.h = h;
        P.rem = rem;
        P.xi = xi;
        P.v = v;
        P.b = b;
        P.n = n;
        P.n64 = n64;
        P.c = c;
    }

    __device__ __forceinline__ void restore(const StepConst &K, const TileIO &io, const Parked &P)
    {
        bind(K, io, P.b, P.c);
        xi64 = P.xi64;
        V = P.V;
        h = P.h;
        rem = P.rem;
        xi = P.xi;
        v = P.v;
        n = P.n;
        n64 = P.n64;
        fl = 0;
    }

    // One trial (FP64 if use64) and the controller; true when the flow step is done (landed on
    // dt, or the attempt limit reached).
    __device__ __forceinline__ bool trial(const StepConst &K, const TileIO &io, bool use64)
    {
        if (n >= K.max_attempts) {
            fl |= PAB_FLAG_STEP_LIMIT;
            return true;
        }
        bool done = false;
        const bool last = le(rem, h);
        const double ht = last ? rem : h;
        const float htf = d2f(ht);
        double nR = 0.0, nV = 0.0;
        float d3R = 0.0f, d3V = 0.0f, errf;
        bool ok, accept;
        if (use64) {
            const BinConst &bc = K.bins[b];
            const Trial64Out tr = collapse_trial64(K, bc, PAB_LD(io.p_inf, c, io.C), bc.R0 + xi64, V, ht);
            ++n64;
            ok = tr.ok;
            accept = tr.accept;
            errf = tr.errf;
            nR = tr.R - bc.R0;
            nV = tr.V;
        } else {
            const Incr32 in = incr32(K, bf, A, xi, v, htf);
            d3R = in.d3R;
            d3V = in.d3V;
            float dR, dV;
            const float R3f = __fadd_rn(bf.R0f, __fadd_rn(xi, d3R));
            const float aRf = fabsf(R3f);
            const float aVf = fmaxf(fabsf(__fadd_rn(v, d3V)), K.v_floorf);
            ok = in.ok && (R3f > 0.0f);
            // err <= tol as |e_R| <= 3 tol |R3| and |e_Rdot| <= 3 tol max(|Rdot3|, v_floor), the
            // thresholds formed in FP32, the estimate's FP64 sum only where the FP32 bracket does
            // not settle it (embedded_within); the growth factor from the FP32 differences
            const bool wR = embedded_within(in.k1R, in.k2R, in.k3R, __fmul_rn(K.tol3f, aRf), dR);
            const bool wV = embedded_within(in.k1V, in.k2V, in.k3V, __fmul_rn(K.tol3f, aVf), dV);
            accept = ok && wR && wV;
            errf = fmaxf(__fmul_rn(fabsf(dR), rcp32(__fmul_rn(3.0f, aRf))),
                         __fmul_rn(fabsf(dV), rcp32(__fmul_rn(3.0f, aVf))));
        }
        ++n;
        const float fac = growth_factor(K, errf, ok);
        const double hn = f2d_fin(__fmul_rn(htf, fac));  // kept in FP32 between calls anyway
        if (accept) {
            if (use64) {
                xi64 = nR;
                V = nV;
                xi = d2f(xi64);
                v = d2f(V);
            } else {
                // the FP32 images move by the same increments
                xi64 += f2d_fin(d3R);
                V += f2d_fin(d3V);
                xi = __fadd_rn(xi, d3R);
                v = __fadd_rn(v, d3V);
            }
            if (last) {
                const bool clipped = !le(h, rem);
                h = (clipped && fac >= 1.0f) ? h : hn;
                done = true;
            } else {
                rem -= ht;
                h = hn;
            }
        } else {
            h = hn;
        }
        if (!done && n >= K.max_attempts) {
            fl |= PAB_FLAG_STEP_LIMIT;
            done = true;
        }
        return done;
    }

    // Status from the FP32 images, the state stored, the counts added.
    __device__ __forceinline__ void finish(const StepConst &K, const TileIO &io, TileCounts &tc)
    {
        if (!isfinite(xi) || !isfinite(v))
            fl |= PAB_FLAG_NONFINITE;
        else if (!(bf.R0f + xi > 0.0f))
            fl |= PAB_FLAG_NONPOS;
        if (fabsf(v) >= K.cf)
            fl |= PAB_FLAG_SUPERSONIC;
        const long long ns = (long long)K.B * io.C;
        PAB_ST(io.R, k, ns, K.bins[b].R0 + xi64);
        PAB_ST(io.V, k, ns, V);
        PAB_ST(io.h, k, ns, d2f(h));
        if (io.attempts)
            PAB_ST(io.attempts, k, ns, n);
        tc.fl_or |= fl;
        tc.n_flag += (fl != 0);
        tc.n_att += n;
        tc.n64 += n64;
    }
};

// Phase 1 streams the CTA's pool; an item whose next trial is FP64 is parked in the CTA's lot
// in shared memory (while it has room; else it takes the trial where it is).  After a CTA
// barrier, phase 2 streams the lot.  Every warp of the CTA must call it (the barrier).
__device__ __forceinline__ void stream_mixed(const StepConst &K, const TileIO &io, PoolCounters &sh,
                                             Parked *lot, int lot_cap, TileCounts &tc)
{
    const int total = (io.b1 - io.b0) * io.nc;
    bool phase2 = false;
    bool exhausted = total <= 0;  // phase 1: the pool; phase 2: the lot
    int parked = 0;               // phase 2: items in the lot
    bool have = false;
    ItemMixed it;
    for (;;) {
        const unsigned want = __ballot_sync(0xffffffffu, !have);
        if (want && !exhausted) {
            if (!phase2) {
                const int j = grab(want, total, &sh.next, exhausted);
                if (j >= 0 && j < total) {
                    int b, cl;
                    size_t k;
                    item_of(io, j, b, cl, k);
                    have = it.start(K, io, b, io.c0 + cl, tc);
                }
            } else {
                const int s = grab(want, parked, &sh.lot_take, exhausted);
                if (s >= 0 && s < parked) {
                    it.restore(K, io, lot[s]);
                    have = true;
                }
            }
        }
        if (!__any_sync(0xffffffffu, have)) {
            if (!exhausted)
                continue;
            if (phase2)
                break;
            __syncthreads();  // every warp has emptied the pool: the lot is complete
            parked = min(*(volatile int *)&sh.lot_n, lot_cap);
            phase2 = true;
            exhausted = parked == 0;
            continue;
        }
        bool use64 = have && it.near_collapse(K);
        if (!phase2) {
            // park the items whose next trial is FP64 while the pool still holds FP32 work
            const unsigned pm = __ballot_sync(0xffffffffu, use64 && it.n < K.max_attempts);
            if (pm) {
                bool full = false;
                const int s = grab(pm, lot_cap, &sh.lot_n, full);
                if (s >= 0 && s < lot_cap) {
                    it.save(lot[s]);
                    have = false;
                    use64 = false;
                }
            }
        }
        if (have && it.trial(K, io, use64)) {
            it.finish(K, io, tc);
            have = false;
        }
    }
}

// ---------------------------------------------------------------------------
// Moments of one cell from its bins' state, summed in bin order.
// ---------------------------------------------------------------------------
// Running sums of one cell: w R^3 (compensated in MIXED), and the other three
// terms (FP32 sums in MIXED, FP64 otherwise).
struct TermSums {
    double m3 = 0.0, m3c = 0.0, m2v = 0.0, m3p = 0.0, m3v2 = 0.0;
    float m2vf = 0.0f, m3pf = 0.0f, m3v2f = 0.0f;
};
template <bool MIXED>
__device__ __forceinline__ void add_terms(TermSums &S, double x, const float *tf, const double *td)
{
    if (MIXED) {
        neumaier_add(S.m3, S.m3c, x);
        S.m2vf = __fadd_rn(S.m2vf, tf[0]);
        S.m3pf = __fadd_rn(S.m3pf, tf[1]);
        S.m3v2f = __fadd_rn(S.m3v2f, tf[2]);
    } else {
        S.m3 = __dadd_rn(S.m3, x);
        S.m2v = __dadd_rn(S.m2v, td[0]);
        S.m3p = __dadd_rn(S.m3p, td[1]);
        S.m3v2 = __dadd_rn(S.m3v2, td[2]);
    }
}

// The 7 moments of cell c (row stride C) from its sums:
// n_b, alpha = 4/3 pi n_b <R^3>, <R^3>, <R^2 Rdot>, 3 alpha <R^2 Rdot>/<R^3>,
// <R^3 p_bw>/<R^3>, <R^3 Rdot^2>/<R^3>.
template <bool MIXED>
__device__ __forceinline__ void write_moments(const StepConst &K, double nb, long long C, long long c,
                                              const TermSums &S, double *out)
{
    double m3 = S.m3, m2v = S.m2v, m3p = S.m3p, m3v2 = S.m3v2;
    if (MIXED) {
        m3 += S.m3c;
        m2v = f2d(S.m2vf);
        m3p = fma(K.p0, m3, f2d(S.m3pf));  // p0 sum w R^3 + sum w R^3 (p_bw - p0)
        m3v2 = f2d(S.m3v2f);
    }
    const double alpha = (4.0 / 3.0 * 3.14159265358979323846) * nb * m3;
    const double inv_m3 = 1.0 / m3;
    const long long no = 7 * C;
    PAB_ST(out, 0 * C + c, no, nb);
    PAB_ST(out, 1 * C + c, no, alpha);
    PAB_ST(out, 2 * C + c, no, m3);
    PAB_ST(out, 3 * C + c, no, m2v);
    PAB_ST(out, 4 * C + c, no, 3.0 * alpha * m2v * inv_m3);
    PAB_ST(out, 5 * C + c, no, (MIXED ? m3p : K.rho * m3p) * inv_m3);  // FP64 terms are over rho
    PAB_ST(out, 6 * C + c, no, m3v2 * inv_m3);
}

// Sums and moments of cell c over all B bins of the state (R, V), in bin order.  The state
// is read through L2 (__ldcg): the same kernel may have written it from other lanes.
// The loads run AHEAD bins ahead of the arithmetic, so that a lane's dependent sums do not wait
// on one round trip per bin (4 in the step kernel's closing pass, whose reads hit L2 behind other
// CTAs' trials; 8 in the reduce-only kernel, whose reads come from HBM).  The order of the sums
// does not depend on it.
// (Gout, FP64 only: where each bin's gas factor at its radius goes for the next flow step.)
template <bool MIXED, int AHEAD = 4>
__device__ __forceinline__ void cell_moments(const StepConst &K, const double *R, const double *V,
                                             long long C, long long c, double nb, double *out,
                                             double *Gout = nullptr)
{
    constexpr int kMomAhead = AHEAD;
    TermSums S;
    double rb[kMomAhead], vb[kMomAhead];
#pragma unroll
    for (int i = 0; i < kMomAhead; ++i) {
        const size_t k = (size_t)i * (size_t)C + (size_t)c;
        rb[i] = i < K.B ? PAB_LDCG(R, k, (long long)K.B * C) : 0.0;
        vb[i] = i < K.B ? PAB_LDCG(V, k, (long long)K.B * C) : 0.0;
    }
    for (int b0 = 0; b0 < K.B; b0 += kMomAhead) {
#pragma unroll
        for (int i = 0; i < kMomAhead; ++i) {
            const int b = b0 + i;
            if (b >= K.B)
                break;
            const double r = rb[i], v = vb[i];
            const int bn = b + kMomAhead;  // refill this slot with the bin kMomAhead ahead
            if (bn < K.B) {
                const size_t k = (size_t)bn * (size_t)C + (size_t)c;
                rb[i] = PAB_LDCG(R, k, (long long)K.B * C);
                vb[i] = PAB_LDCG(V, k, (long long)K.B * C);
            }
            const BinConst &bc = K.bins[b];
            if (MIXED) {
                float tf[3];
                const double x = quad_terms_mixed(K, bc, r, v, tf);
                add_terms<true>(S, x, tf, nullptr);
            } else {
                double t[4], G;
                GasBase g;
                g.reset();
                quad_terms64(K, bc, r, v, t, g, G);
                add_terms<false>(S, t[0], nullptr, t + 1);
                if (Gout)
                    PAB_ST(Gout, (size_t)b * (size_t)C + (size_t)c, (long long)K.B * C, G);
            }
        }
    }
    write_moments<MIXED>(K, nb, C, c, S, out);
}

// The quadrature terms of bin b at (r, v) added to a cell's sums, with the arithmetic of
// cell_moments.
template <bool MIXED>
__device__ __forceinline__ void add_bin_terms(const StepConst &K, int b, double r, double v, TermSums &S)
{
    const BinConst &bc = K.bins[b];
    if (MIXED) {
        float tf[3];
        const double x = quad_terms_mixed(K, bc, r, v, tf);
        add_terms<true>(S, x, tf, nullptr);
    } else {
        double t[4];
        GasBase g;
        g.reset();
        quad_terms64(K, bc, r, v, t, g);
        add_terms<false>(S, t[0], nullptr, t + 1);
    }
}

// The quadrature terms of the state (R, V) of bin b at state index k into the terms buffer, with
// the arithmetic of the closing moment pass (cell_moments), so that summing them in bin order
// gives its bits.
template <bool MIXED>
__device__ __forceinline__ void store_terms(const StepConst &K, double *terms, int b, size_t k,
                                            double R, double V, double *Gout = nullptr)
{
    const long long ns = (long long)K.B * K.C;
    const BinConst &bc = K.bins[b];
    if (MIXED) {
        float tf[3];
        PAB_ST(terms, k, ns, quad_terms_mixed(K, bc, R, V, tf));
        float *t32 = reinterpret_cast<float *>(terms + ns);
#pragma unroll
        for (int m = 0; m < 3; ++m)
            PAB_ST(t32, (long long)m * ns + (long long)k, 3 * ns, tf[m]);
    } else {
        double t[4], G;
        GasBase g;
        g.reset();
        quad_terms64(K, bc, R, V, t, g, G);
#pragma unroll
        for (int m = 0; m < 4; ++m)
            PAB_ST(terms, (long long)m * ns + (long long)k, 4 * ns, t[m]);
        if (Gout)
            PAB_ST(Gout, k, ns, G);
    }
}


// The moments of cell c from the terms its bins stored (store_terms), summed in bin order as
// cell_moments sums them.  The terms are read through L2: other CTAs of the launch wrote them.
template <bool MIXED>
__device__ __forceinline__ void sum_cell_terms(const StepConst &K, const double *terms, long long c,
                                               double nb, double *out)
{
    const long long ns = (long long)K.B * K.C;
    const float *t32 = reinterpret_cast<const float *>(terms + ns);
    TermSums S;
    constexpr int kAhead = 8;
    for (int b0 = 0; b0 < K.B; b0 += kAhead) {
        double x[kAhead], td[kAhead][3];
        float tf[kAhead][3];
#pragma unroll
        for (int i = 0; i < kAhead; ++i) {
            const long long k = (long long)(b0 + i) * K.C + c;
            if (b0 + i < K.B) {
                x[i] = PAB_LDCG(terms, k, ns);
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    if (MIXED)
                        tf[i][m] = PAB_LDCG(t32, m * ns + k, 3 * ns);
                    else
                        td[i][m] = PAB_LDCG(terms, (m + 1) * ns + k, 4 * ns);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kAhead; ++i) {
            if (b0 + i < K.B)
                add_terms<MIXED>(S, x[i], tf[i], td[i]);
        }
    }
    write_moments<MIXED>(K, nb, K.C, c, S, out);
}

}  // namespace pab
