/*
 * fbp_fixed.h -- a run of a static-strategy graph that allocates nothing.
 *
 * The paper has no counterpart of this entry point: it is a library-level
 * variant of fbp_run (include/fbp.h) with the same arithmetic and results.
 *
 * Why it exists.  fbp_run may allocate device memory inside the call: the
 * per-iteration residual words of a run are sized by max_iters and grown on
 * demand through the graph's allocator.  Some callers must not allocate once
 * they are running: a serving loop that has handed all of its device memory
 * to resident graphs up front and must not fail on an allocation halfway
 * through a request, or a latency-bound caller for whom an allocation (and
 * the device synchronisation a cudaMalloc may imply) is not acceptable on the
 * hot path.  fbp_run_fixed_scratch takes its per-run scratch from one
 * fixed-size array in the library's static device memory instead.
 */
#ifndef FBP_FIXED_H
#define FBP_FIXED_H

#include "fbp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest max_iters fbp_run_fixed_scratch accepts, and the size in bytes of
 * the library's static device scratch array (a 256-byte header holding the
 * grid-barrier words, the run's result words and the guard counter, then one
 * 4-byte residual word per iteration). */
#define FBP_FIXED_SCRATCH_MAX_ITERS 16384
#define FBP_FIXED_SCRATCH_BYTES (256 + 4 * FBP_FIXED_SCRATCH_MAX_ITERS)

/* Run graph g from its current messages as fbp_run does for a static
 * strategy (SEQFIX, TOPO, TOPO_FB, CUSTOM_RANK), stopping at the first
 * iteration whose residual is below tol or after max_iters iterations.  The
 * paper has no counterpart of this call.  Same return values, outputs and
 * message state as fbp_run on the same graph, bit for bit, and the same
 * fbp_get_stats figures except kernel_launches: this call always runs the
 * persistent level engine in one launch (kernel_launches = 1), also when
 * FBP_OPT_ENGINE = 0 asks fbp_run for one launch per level, which computes
 * the same messages.  FBP_OPT_ENGINE = 3 (the belief-form sequential engine,
 * which rounds differently) is not honoured here: the comparison holds
 * against fbp_run with FBP_OPT_ENGINE 0, 1 or 2.
 *
 * Memory: allocates no device memory (no cudaMalloc, no call of the graph's
 * allocator, no library routine that allocates).  The per-run scratch -- the
 * barrier counter and generation, the result words, the guard counter and
 * the per-iteration residual words -- lives in one file-scope static device
 * array of FBP_FIXED_SCRATCH_BYTES.  All of these words must be zero when the
 * kernel starts; the call clears the header and the first max_iters residual
 * words on the graph's stream before its launch, so nothing has to be zero
 * beforehand.  The graph's own buffers it uses (messages, levels, the event
 * pair that times the run) were all made by fbp_graph_create and
 * fbp_schedule_set.
 *
 * First call on a device: the library looks up the array's device address
 * with cudaGetSymbolAddress once per device, with that device current, and
 * keeps it; that lookup (and the first launch of the engine kernel, as for
 * fbp_run) may load the library's device code on that device.  Make the
 * first call on each device before any stream capture is begun on it.  Call
 * with the graph's device current, as for every entry point.
 *
 * Concurrency: there is ONE scratch array per device per process.  Calls
 * that overlap in time on the same device -- from two host threads, or on two
 * graphs at once -- share it and race (corrupted barrier counts, results and
 * residuals).  The call itself is synchronous (it returns after the run), so
 * calls from a single host thread never overlap.
 *
 * Errors: FBP_ERR_INVALID_ARG for g == NULL, max_iters < 0, max_iters >
 * FBP_FIXED_SCRATCH_MAX_ITERS (the message names the limit), tol < 0 or NaN,
 * a graph whose strategy is PARALL or RESIDUAL (both need per-run buffers
 * this entry point does not have), or generic factors without their terms; FBP_ERR_CUDA when the symbol
 * lookup or a launch fails; FBP_ERR_TIMEOUT as fbp_run.  Nothing runs and
 * the graph is unchanged when an argument is rejected. */
int fbp_run_fixed_scratch(fbp_graph *g, int32_t max_iters, double tol, int32_t *iters_out,
                          double *residual_out);

#ifdef __cplusplus
}
#endif
#endif /* FBP_FIXED_H */
