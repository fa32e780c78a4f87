/*
 * fbp.h -- C ABI of the GB300 belief-propagation library (FastLBP's method,
 * arXiv 2509.22337, re-designed for sm_103a).
 *
 * Scope: sum-product belief propagation on factor graphs over binary
 * variables whose factors carry logical local structure (Sec. 2.2, Sec. 3.3):
 * AND, OR, NOT, EQ, NOISY_IMPLY(p), NOISY_AND(p) and unary PRIOR(p).  Each
 * factor-to-variable message is evaluated in O(fan-in) from the factor's type
 * code (never from a dense table).  Messages are updated under an update
 * strategy (Table 1 and Definition 2), turned into ordered levels of mutually
 * independent updates by the dependency analysis of Algorithm 2.
 *
 * Conventions used by every entry point
 *   - V variables, A factors, E edges.  An edge is a (factor, variable) pair;
 *     its id is its position in the factor-major CSR given to
 *     fbp_graph_create (the "edge id" of Sec. 4.3.3).
 *   - Each factor row lists its variables premises first and the output
 *     (conclusion) variable last; a variable appears at most once per row.
 *     NOT has exactly [x, y]; PRIOR exactly [y]; EQ is symmetric.
 *   - Messages are normalised pairs (m0, m1), m0 + m1 = 1, FP32.
 *   - A message whose unnormalised entries sum to zero (contradictory hard
 *     evidence through deterministic factors) becomes the uniform message (the
 *     zero-mass guard); the same guard applies to marginals.
 *   - All host pointers are borrowed for the duration of the call only; the
 *     library copies what it keeps.  Device memory is owned by the library
 *     (allocated through the caller's allocator, if one is given) and freed by
 *     the matching destroy call.
 *   - Work is ordered on the CUDA stream given at creation.  A handle must not
 *     be used by two threads at once.
 *   - Every int-returning entry point returns FBP_OK (0) on success, a
 *     positive status, or a negative error code; on error the thread-local
 *     message of fbp_last_error() says what was wrong and the handle is left
 *     as it was before the call unless stated otherwise.
 */
#ifndef FBP_H
#define FBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FBP_OK               0
#define FBP_NOT_CONVERGED    1   /* a status: max_iters reached above tol  */
#define FBP_ERR_INVALID_ARG (-1) /* bad pointer, size, CSR, type, arity, p */
#define FBP_ERR_OOM         (-2) /* device allocation failed               */
#define FBP_ERR_CUDA        (-3) /* a CUDA runtime call failed             */
#define FBP_ERR_SCHEDULE    (-4) /* TOPO on a cyclic graph; bad rank array */
#define FBP_ERR_TIMEOUT     (-5) /* a bounded device wait expired          */

/* ---- factor type codes (Sec. 2.2 and Sec. 3.3), with these semantics:
 *      NOISY_AND(p): all premises true -> y=1 w.p. p,
 *      any false premise forces y=0; NOISY_IMPLY(p): all premises true ->
 *      y=1 w.p. p, a false premise leaves y free; PRIOR(p): P(y=1) = p) ---- */
enum {
    FBP_AND = 0, FBP_OR = 1, FBP_NOT = 2, FBP_EQ = 3,
    FBP_NOISY_IMPLY = 4, FBP_NOISY_AND = 5, FBP_PRIOR = 6,
    FBP_TERMS = 7  /* generic: local structure from fbp_set_factor_terms */
};

/* ---- update strategies (Table 1; Definition 2) -------------------------
 * PARALL      every edge in one class: synchronous (flooding) BP.
 * SEQFIX      a total order: edge_rank if given, else edge-id order.
 * TOPO        rank = depth of the factor's output variable (or factor_rank).
 * TOPO_FB     one iteration = the TOPO order, then the reversed TOPO order.
 * RESIDUAL    dynamic: iteration 1 is PARALL; afterwards factors are ranked
 *             by the largest message change at their variables in the
 *             previous iteration (>= 1e-2, >= 1e-4, >= tol) and factors
 *             below tol are skipped; levels are rebuilt every iteration.
 * CUSTOM_RANK any weak order given as an integer rank per edge.            */
enum {
    FBP_PARALL = 0, FBP_SEQFIX = 1, FBP_TOPO = 2, FBP_TOPO_FB = 3,
    FBP_RESIDUAL = 4, FBP_CUSTOM_RANK = 5
};

typedef struct fbp_graph fbp_graph;

/* Device allocator: alloc(bytes, ctx) returns device memory or NULL;
 * free(ptr, ctx) releases it.  Pass NULL to use cudaMalloc/cudaFree. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
} fbp_allocator;

/* Strategy specification (Sec. 4.2.1: a strategy name or a custom preorder).
 * edge_rank:   [E] int64; required for CUSTOM_RANK, optional for SEQFIX.
 * factor_rank: [A] int32; optional for TOPO/TOPO_FB (replaces the depth).
 * residual_buckets: reserved, must be 0 or 3.                              */
typedef struct {
    int32_t strategy;
    const int64_t *edge_rank;
    const int32_t *factor_rank;
    int32_t residual_buckets;
} fbp_schedule_spec;

/* Counters of the last fbp_run on a handle. */
typedef struct {
    int64_t updates;        /* factor-to-variable messages written        */
    int64_t guards;         /* zero-mass guards in a->v messages           */
    int32_t iters;          /* iterations executed                         */
    int32_t levels;         /* levels per iteration (static strategies)    */
    double  residual;       /* residual of the last iteration              */
    double  run_ms;         /* device time of the run (CUDA events)        */
    int64_t kernel_launches;/* kernels launched by the run                 */
} fbp_stats;

/* Build a graph on the device (Sec. 4.1 "Initialization": the CSR layouts
 * of Sec. 4.3.2).
 *   factor_ptr  [n_factors+1] int64, non-decreasing, factor_ptr[0] = 0,
 *               E = factor_ptr[n_factors] < 2^31.
 *   factor_vars [E] int32 in [0, n_vars), distinct within a row.
 *   factor_type [n_factors] uint8 type code; factor_param [n_factors] float,
 *               p in [0,1] for NOISY_IMPLY, NOISY_AND, PRIOR (ignored else).
 *   prior_p1    [n_vars] float prior P(x=1) in [0,1], NaN = none; may be NULL.
 *   evidence    [n_vars] int8: -1 none, 0 or 1 clamps; may be NULL.
 *   alloc       device allocator or NULL.  cuda_stream: cudaStream_t or NULL.
 * Evidence overrides a prior.  The schedule starts as PARALL.  All messages
 * start uniform.  On success *out owns its device memory. */
int fbp_graph_create(int32_t n_vars, int32_t n_factors, const int64_t *factor_ptr,
                     const int32_t *factor_vars, const uint8_t *factor_type,
                     const float *factor_param, const float *prior_p1,
                     const int8_t *evidence, const fbp_allocator *alloc,
                     void *cuda_stream, fbp_graph **out);

/* Set the update strategy: build the per-edge ranks, run Algorithm 2
 * (Sec. 4.2.3) on the host and upload the level lists.  Returns
 * FBP_ERR_SCHEDULE for TOPO/TOPO_FB on a cyclic graph, FBP_ERR_INVALID_ARG
 * for a missing rank array.  Messages are not reset. */
int fbp_schedule_set(fbp_graph *g, const fbp_schedule_spec *spec);

/* Run BP (Sec. 4.1 "Message Passing"): iterate until the residual of an
 * iteration (largest |new m1 - old m1| over its a->v writes) is below tol,
 * or for max_iters iterations.  Continues from the current messages (warm
 * start).  iters_out / residual_out may be NULL.  Returns FBP_OK when
 * converged, FBP_NOT_CONVERGED otherwise. */
int fbp_run(fbp_graph *g, int32_t max_iters, double tol, int32_t *iters_out,
            double *residual_out);

/* Marginals P(x_v = 1) of Eq. (3) into out_p1[n_vars]; out_is_device = 1 if
 * out_p1 is device memory (written on the graph's stream, not synchronised),
 * 0 for host memory (the call synchronises). */
int fbp_marginals(const fbp_graph *g, float *out_p1, int out_is_device);

/* The current schedule's levels (the sequence S of Algorithm 2).  With NULL
 * buffers only *n_levels (and the total edge count through level_ptr == NULL)
 * is reported.  level_ptr [n_levels+1] int64, level_edges [level_ptr[n]]
 * int32 in canonical (rank, edge id) order.  TOPO_FB reports the forward
 * levels followed by the backward levels (2E entries).  RESIDUAL reports
 * the levels of its most recent iteration. */
int fbp_schedule_levels(const fbp_graph *g, int32_t *n_levels, int64_t *level_ptr,
                        int32_t *level_edges);

/* Host-only dependency analysis, for checking Algorithm 2 without a device:
 * the same ranks and levels fbp_schedule_set would build for this CSR.
 * backward = 1 gives the backward half of TOPO_FB.  NULL level buffers =
 * size query (*n_levels set, and *n_edges_out if non-NULL). */
int fbp_schedule_build_host(int32_t n_vars, int32_t n_factors, const int64_t *factor_ptr,
                            const int32_t *factor_vars, const fbp_schedule_spec *spec,
                            int32_t backward, int32_t *n_levels, int64_t *level_ptr,
                            int32_t *level_edges);

/* Clamp variable var to value (0/1), or release it (-1: back to its prior).
 * Used by the serving loop; takes effect at the next fbp_run. */
int fbp_set_evidence(fbp_graph *g, int32_t var, int8_t value);

/* Local structure of the generic (FBP_TERMS) factors, given explicitly as
 * the indicator array of Sec. 4.3.2 with a weight per term (Eq. 4): the
 * factor is the sum of its terms, term t being w_t on the assignments that
 * agree with its fixed variables and 0 elsewhere; its messages are computed
 * by Algorithm 1.
 *   term_ptr [n_factors+1] int64, term_ptr[0] = 0: factor a's terms are
 *            term_ptr[a] .. term_ptr[a+1]-1 (none for typed factors;
 *            at most 256 per factor).
 *   term_ind int8: factor a's indicators are a block of
 *            (terms of a) x (variables of a) values, term after term, each
 *            variable in the factor's row order: 0 or 1 (the term fixes the
 *            variable) or -1 (free); blocks in factor order.
 *   term_w   [term_ptr[n_factors]] float, finite and >= 0.
 * Arrays are copied.  A graph with FBP_TERMS factors (at most 32 variables
 * each) must receive their terms before its first fbp_run, which otherwise
 * returns FBP_ERR_INVALID_ARG; calling it again replaces them.  Returns
 * FBP_ERR_INVALID_ARG for a malformed list (the message names the factor). */
int fbp_set_factor_terms(fbp_graph *g, const int64_t *term_ptr, const int8_t *term_ind,
                         const float *term_w);

/* Copy the a->v messages out as normalised (m0, m1) pairs, a2v[2E] host, or
 * in (checkpoint / resume; warm start). */
int fbp_messages_export(const fbp_graph *g, float *a2v);
int fbp_messages_import(fbp_graph *g, const float *a2v);

/* Reset every a->v message to the uniform message (a cold start). */
int fbp_messages_reset(fbp_graph *g);

/* Counters of the last run. */
int fbp_get_stats(const fbp_graph *g, fbp_stats *out);

/* Tuning and failure-detection options of a graph handle.
 * FBP_OPT_SPIN_LIMIT   cycles a device-side barrier may wait before the run
 *                      fails with FBP_ERR_TIMEOUT (default 4e9, about 2 s);
 *                      0 makes every wait expire at once (used to test the
 *                      timeout path).
 * FBP_OPT_ENGINE_GRID  blocks of the persistent level engine in grid mode
 *                      (0 = automatic choice of mode and size).
 * FBP_OPT_ENGINE       1 (default): static strategies run in the persistent
 *                      engine with a grid barrier between levels; 2: the
 *                      persistent engine in dataflow form (a lane waits only
 *                      for the messages it reads from earlier levels; same
 *                      results); 0: one launch per level (reference path);
 *                      3: the belief-form sequential engine for graphs with
 *                      high-degree variables (each variable's belief is kept
 *                      current level by level and v->a = belief / own
 *                      message, so a message costs its factor's size instead
 *                      of its variables' degrees; the same schedule and
 *                      iteration count, FP32 products grouped as in the
 *                      flooding kernels, so results differ from 0-2 by
 *                      rounding).  Batches always use the level engine.
 * FBP_OPT_ENGINE_CLUSTER 0 (default): automatic; 1: never run the engine as
 *                      one thread-block cluster; 8 or 16: always, with that
 *                      cluster size.
 * FBP_OPT_FLOOD_HUB_MIN  flooding: variables with more incident factors than
 *                      this (8..256, default 256) are split over blocks.
 * FBP_OPT_FLOOD_CHUNK  flooding: entries of such a variable per block
 *                      (a multiple of 256 in 256..65536, default 1024).
 *                      Neither split option changes a result: a long row's
 *                      product is grouped one fixed way (32-entry sub-chunks
 *                      dealt to 256 slots, then a butterfly) whichever kernel
 *                      carries it, so messages are bit-identical.
 * FBP_OPT_ENGINE_FUSE_LANES  level fusion of the grid engine (0..256,
 *                      default 0 = off): a level of at most this many lanes
 *                      (one lane per variable of each factor it touches) and
 *                      no factor wider than a warp runs in one block, and
 *                      consecutive such levels of an iteration are separated
 *                      by block barriers instead of grid barriers.  Levels
 *                      are never merged: results are unchanged.
 * FBP_OPT_ENGINE_SOLO_LANES  the whole run goes to one block when the
 *                      schedule's levels average at most this many lanes
 *                      (default 128; 0 = never).  Results are unchanged.
 * FBP_OPT_RESIDUAL_DEVICE 1 (default): RESIDUAL builds each iteration's
 *                      classes and Algorithm 2 levels on the device and runs
 *                      the levels with the flooding kernels; 0: classes and
 *                      levels on the host, levels run by the level engine. */
enum {
    FBP_OPT_SPIN_LIMIT = 1, FBP_OPT_ENGINE_GRID = 2, FBP_OPT_ENGINE = 3, FBP_OPT_ENGINE_CLUSTER = 4,
    FBP_OPT_FLOOD_HUB_MIN = 5, FBP_OPT_FLOOD_CHUNK = 6, FBP_OPT_RESIDUAL_DEVICE = 7,
    FBP_OPT_ENGINE_FUSE_LANES = 8, FBP_OPT_ENGINE_SOLO_LANES = 9
};
int fbp_set_option(fbp_graph *g, int32_t option, int64_t value);

/* Free the graph's device memory (after the stream's pending work). */
void fbp_graph_destroy(fbp_graph *g);

/* Thread-local description of the last error ("" if none). */
const char *fbp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FBP_H */
