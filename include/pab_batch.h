/*
 * pab_batch.h - many independent bubble-source instances in one persistent
 * kernel (sm_103a).
 *
 * Each instance is one ensemble of pab.h (its own cells, bins, fluid and
 * forcing) advanced by the same method: Keller-Miksis bins (Sec. 2) with
 * adaptive SSP-RK3(2) sub-steps (Sec. 3) and quadrature moments (Sec. 2.2).
 * Batching is not in the paper; instances are independent, so batching
 * changes no result: an instance's state after a batched step equals the
 * state pab_bubble_step gives it alone (same kernel arithmetic), and its
 * moments agree to the rounding of the sum order.
 *
 * A batch is an arena of `max_slots` slots sharing one device state arena of
 * `capacity_bins` bin-states (20 bytes each: R and Rdot in FP64, h in FP32).
 * pab_batch_admit places an instance in a free slot if its Nb x C bin-states
 * fit the arena (admission by device memory); pab_batch_release frees it.
 * Every pab_batch_step advances all active slots by one flow step with one
 * launch sequence on `stream`:
 *   1. an order kernel sorts the active slots by the trials they needed in
 *      their previous step (stiffest first) and lays out the work queue of
 *      (slot, 32-cell tile) items;
 *   2. a persistent kernel (a fixed grid of CTAs per SM) pulls items from the
 *      queue with an atomic counter; inside an item the CTA's warps pull bins
 *      with a shared-memory counter, so stiff bins and stiff instances are
 *      spread over the idle warps and SMs; per-bin quadrature terms are
 *      reduced in bin order, so the moments do not depend on the schedule.
 * pab_batch_step_graph runs the same sequence as a CUDA graph captured on its
 * first call (the slot table is read by the kernels at run time, so slots may
 * be admitted, bound and released between replays).
 *
 * Conventions are those of pab.h: caller-owned device pointers, stream-ordered
 * calls, status words instead of traps, no exceptions, one batch per thread.
 */
#ifndef PAB_BATCH_H
#define PAB_BATCH_H

#include <stdint.h>

#include "pab.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pab_batch_s pab_batch_t;

typedef struct {
    int32_t max_slots;        /* 1..4096 instances resident at once */
    int32_t precision;        /* PAB_FP64 or PAB_MIXED, for every slot */
    int64_t capacity_bins;    /* arena size in bin-states, at most PAB_MAX_CELLS x PAB_MAX_BINS;
                                 0: 80 % of free device memory / 20 B */
    int32_t block_warps;      /* warps per CTA, 0..16 (0: 8) */
    int32_t ctas_per_sm;      /* persistent CTAs per SM, 0..32 (0: as many as fit, at most 4) */
    int32_t bins_per_grab;    /* bins a warp takes per shared-memory grab, 0..8 (0: 1) */
    int32_t max_bins;         /* largest Nb any slot will use (0: PAB_MAX_BINS); sizes shared memory */
} pab_batch_config;

void pab_batch_config_default(pab_batch_config *cfg);

/* Create an empty batch and allocate its arena on the current device.
 * Errors: PAB_EINVAL, PAB_ENOMEM, PAB_ECUDA. */
pab_status pab_batch_create(const pab_batch_config *cfg, void *stream, pab_batch_t **out);

/* Admit one instance: validate cfg exactly as pab_create does (its
 * precision, record_attempts and block_warps fields are ignored), build its bin
 * table, place its Nb x C state in the arena and initialise it as pab_create
 * does, on `stream`.  *slot receives the slot index.
 * Errors: PAB_EINVAL (bad cfg, Nb above max_bins), PAB_ENOMEM (no free slot or
 * no contiguous arena space: the admission refusal), PAB_ECUDA. */
pab_status pab_batch_admit(pab_batch_t *b, const pab_config *cfg, void *stream, int32_t *slot);

/* Attach the slot's per-step inputs and outputs: p_inf_dev [C] (required),
 * nb_dev [C] or NULL (default n_b), moments_dev [7][C] or NULL, and dt > 0.
 * The pointers are read by every later step until re-bound, so the caller
 * refreshes the pressure in place between steps.  A step reads the slot table
 * when it runs, so bind (like admit and release) first waits, on the host,
 * until the batch's last enqueued step has finished: binding between steps is
 * safe on any stream, and costs that wait.  Steps enqueued into the caller's
 * own stream capture are not waited for.
 * Errors: PAB_EINVAL (slot not admitted, NULL p_inf_dev, dt <= 0 or non-finite),
 * PAB_ECUDA. */
pab_status pab_batch_bind(pab_batch_t *b, int32_t slot, const double *p_inf_dev, const double *nb_dev,
                          double *moments_dev, double dt);

/* Free a slot and its arena space (stream-ordered with later admissions on `stream`). */
pab_status pab_batch_release(pab_batch_t *b, int32_t slot, void *stream);

/* One flow step of every active, bound slot (see above). */
pab_status pab_batch_step(pab_batch_t *b, void *stream);

/* The same step replayed from a CUDA graph captured on the first call (on a
 * stream the batch owns, so any stream, the legacy default one included, may
 * be passed) and launched into `stream`.  pab_batch_set_launch drops the graph. */
pab_status pab_batch_step_graph(pab_batch_t *b, void *stream);

/* Synchronise `stream` and read-and-reset a slot's status, as pab_status_flags. */
pab_status pab_batch_status(pab_batch_t *b, int32_t slot, uint32_t *flags, int64_t *n_flagged,
                            int64_t *n_attempts, int64_t *n_fp64, void *stream);

/* Checkpoint / resume of one slot (device buffers [Nb][C]). */
pab_status pab_batch_get_state(pab_batch_t *b, int32_t slot, double *R_dev, double *Rdot_dev,
                               float *h_dev, void *stream);
pab_status pab_batch_set_state(pab_batch_t *b, int32_t slot, const double *R_dev,
                               const double *Rdot_dev, const float *h_dev, void *stream);

/* Occupancy: active slots, bin-states in use and arena capacity. */
pab_status pab_batch_usage(const pab_batch_t *b, int32_t *active_slots, int64_t *bins_used,
                           int64_t *capacity_bins);

/* Launch shape used by later steps (the autotuner's knobs); invalidates the
 * captured graph.  block_warps 1..16, ctas_per_sm 1..32, bins_per_grab 1..8; a CTA of
 * one warp sums its tile's moment terms itself (no shared per-bin terms, so more
 * CTAs fit on an SM), with the same results as the wider shapes. */
pab_status pab_batch_set_launch(pab_batch_t *b, int32_t block_warps, int32_t ctas_per_sm,
                                int32_t bins_per_grab);

/* Free everything (synchronises the creation stream).  NULL-safe. */
void pab_batch_destroy(pab_batch_t *b);

const char *pab_batch_last_error(const pab_batch_t *b);

#ifdef __cplusplus
}
#endif

#endif /* PAB_BATCH_H */
