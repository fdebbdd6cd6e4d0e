/* hspeak.h -- integer issue-rate microbenchmarks (libhspeak.so).
 *
 * Measurement helper for the database scan's roofline, not part of the
 * search library's ABI and with no counterpart in the paper: the scan is
 * bound by integer instruction issue (one packed add scores 4 virtual-score
 * cells), so its fraction of peak needs the GPU's measured integer rate.
 */
#ifndef HSPEAK_H
#define HSPEAK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The measured operation. */
#define HSP_IADD 0          /* 32-bit integer add */
#define HSP_DPX_MAX3 1      /* DPX three-way signed maximum (__vimax3_s32) */
#define HSP_DPX_ADDMAX 2    /* DPX add-then-maximum, max(a + b, c) (__viaddmax_s32) */

/* Operations one thread performs per loop trip (ops per launch =
 * blocks * 1024 threads * iters * this). */
int hsp_ops_per_thread_trip(void);

/* Runs the microbenchmark for `op` on the current device: one untimed
 * launch, then `reps` launches of `iters` loop trips each, timed by CUDA
 * events on `stream` (NULL: the default stream); the grid fills every SM
 * with as many 1024-thread blocks as fit.  Outputs: the best launch's rate
 * (operations per second over the whole GPU), its time in ms, and the
 * operations of one launch.  Allocates and frees a small sink buffer.
 * Returns 0, or 1 for a bad argument, 2 for a CUDA error, 3 when the sink
 * cannot be allocated. */
int hsp_measure(int op, int iters, int reps, void *stream, double *ops_per_s, double *best_ms,
                int64_t *ops_per_launch);

#ifdef __cplusplus
}
#endif

#endif
