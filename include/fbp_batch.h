/*
 * fbp_batch.h -- batched and served forms of the belief-propagation library
 * (extensions of include/fbp.h; the paper has no counterpart of either: they
 * run many independent FastLBP problems, each with its own update strategy and
 * stopping rule, without changing the arithmetic of any of them).
 *
 * Batched form.  Hundreds of independent graphs of uneven sizes run
 * together: graphs with a static strategy (SEQFIX, TOPO, TOPO_FB, CUSTOM_RANK)
 * share one persistent level-engine launch (each graph keeps its own
 * Algorithm 2 levels; level k of every graph runs in step k), flooding
 * (PARALL) graphs share one flooding loop, and the two parts run concurrently.
 * Every graph stops at its own first iteration with residual < its tol (or
 * at its own max_iters), exactly as a single-graph fbp_run would, so results
 * equal the per-graph runs.
 *
 * Served form: include/fbp_serve.h.
 */
#ifndef FBP_BATCH_H
#define FBP_BATCH_H

#include "fbp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One graph of a batch (arrays as in fbp_graph_create; borrowed for the
 * duration of fbp_batch_create).  schedule.strategy may be any static
 * strategy or PARALL (RESIDUAL is rejected); generic (FBP_TERMS) factors are
 * rejected (they need fbp_set_factor_terms on a single graph). */
typedef struct {
    int32_t n_vars, n_factors;
    const int64_t *factor_ptr;
    const int32_t *factor_vars;
    const uint8_t *factor_type;
    const float *factor_param;
    const float *prior_p1;       /* may be NULL */
    const int8_t *evidence;      /* may be NULL */
    fbp_schedule_spec schedule;
    int32_t max_iters;
    double tol;
} fbp_graph_desc;

typedef struct fbp_batch fbp_batch;

/* Launch shapes (the autotuner's knobs): blocks of the level engine (0 =
 * automatic), whether it runs as one thread-block cluster (0 automatic, 1
 * never, 8 or 16 = cluster size; for the member queue, 16 = 16-block
 * clusters, anything else 8), the flooding split of long variable rows over
 * blocks (FBP_OPT_FLOOD_HUB_MIN / FBP_OPT_FLOOD_CHUNK; 0 = default), the
 * engine's level-fusion and one-block thresholds (FBP_OPT_ENGINE_FUSE_LANES,
 * FBP_OPT_ENGINE_SOLO_LANES; -1 = default), and the clusters the member queue
 * launches (0 = automatic: half of those that can be resident when flooding
 * members run beside the queue, so that their kernels find free SMs, else
 * all; larger values are clamped to what can be resident).  No knob changes
 * a result. */
typedef struct {
    int32_t engine_grid;
    int32_t engine_cluster;
    int32_t flood_hub_min;
    int32_t flood_chunk;
    int32_t engine_fuse_lanes;
    int32_t engine_solo_lanes;
    int32_t queue_clusters;
} fbp_batch_tuning;

/* Build every graph on the device (copies all arrays; Algorithm 2 per graph
 * on the host).  Returns FBP_ERR_INVALID_ARG for a bad graph (the message
 * names it), FBP_ERR_SCHEDULE for TOPO on a cyclic graph. */
int fbp_batch_create(int32_t n_graphs, const fbp_graph_desc *graphs, const fbp_allocator *alloc,
                     void *cuda_stream, fbp_batch **out);

/* How a batch runs.  Every form computes every member's messages exactly as
 * a single-graph run of it does.
 *  - The member queue: one persistent kernel launch (a CUDA graph captured
 *    once) of thread-block clusters (8 blocks, or 16: fbp_batch_tuning's
 *    engine_cluster) that take whole members from a queue, largest first,
 *    and run each to its own stopping rule with barriers among the blocks of
 *    a cluster only.
 *  - Flooding side by side: the flooding members together as one union graph
 *    run by the whole-GPU flooding kernels (captured iterations), on a second
 *    stream.
 * one_launch = 1: every member in the member queue (one launch in all).
 * one_launch = 0, static_queue = 1 (the default): static members in the
 *   member queue, flooding members side by side; two launches that run
 *   concurrently (the queue is not a cooperative launch).
 * one_launch = 0, static_queue = 0: static members in one cooperative level
 *   engine launch over the union of their levels merged by index, flooding
 *   members side by side. */
typedef struct {
    int32_t one_launch;
    int32_t static_queue;
} fbp_batch_config;

/* fbp_batch_create with a configuration (NULL = defaults).  Returns
 * FBP_ERR_INVALID_ARG for a bad configuration, FBP_ERR_CUDA when one launch
 * is asked for on a device that cannot launch the queue kernel. */
int fbp_batch_create_ex(int32_t n_graphs, const fbp_graph_desc *graphs, const fbp_allocator *alloc,
                        void *cuda_stream, const fbp_batch_config *config, fbp_batch **out);

/* 1 if the batch runs in one launch, 0 if on two streams, -1 for NULL. */
int fbp_batch_one_launch(const fbp_batch *b);

/* Run every graph from its current messages to its own stopping rule.
 * iters_out / residual_out / status_out: [n_graphs] host arrays or NULL;
 * status FBP_OK (converged) or FBP_NOT_CONVERGED.  Returns FBP_OK when all
 * graphs converged, FBP_NOT_CONVERGED otherwise. */
int fbp_batch_run(fbp_batch *b, int32_t *iters_out, double *residual_out, int32_t *status_out);

/* Marginals of one graph of the batch ([n_vars of that graph]). */
int fbp_batch_marginals(const fbp_batch *b, int32_t graph, float *out_p1, int out_is_device);

/* a->v messages of one graph as (m0, m1) pairs, [2 * n_edges of that graph]. */
int fbp_batch_messages_export(const fbp_batch *b, int32_t graph, float *a2v);

/* All messages back to uniform (a cold start for the next run). */
int fbp_batch_reset(fbp_batch *b);

/* Launch shapes; NULL or zero fields = automatic.  For the member queue,
 * engine_cluster is its cluster size (16: 16 blocks; otherwise 8) and
 * engine_grid caps its clusters (0: as many as can be resident; a cap leaves
 * room for the flooding kernels that run beside it). */
int fbp_batch_set_tuning(fbp_batch *b, const fbp_batch_tuning *t);

/* Totals of the last run: updates, guards, run_ms (device time of the whole
 * batch), kernel_launches; iters = the largest per-graph iteration count. */
int fbp_batch_get_stats(const fbp_batch *b, fbp_stats *out);

void fbp_batch_destroy(fbp_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* FBP_BATCH_H */
