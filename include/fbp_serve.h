/*
 * fbp_serve.h -- served form of the belief-propagation library (an extension
 * of include/fbp.h; the paper has no counterpart).
 *
 * A server keeps interactive-analysis sessions resident on the device: each
 * session is one factor graph with its messages and evidence.  A request
 * clamps one variable of one session to a value (the user feedback of
 * BINGO-style alarm inspection, Sec. 5.2.2) and re-runs belief propagation
 * from the session's stored messages (a warm start) under the session's
 * strategy until the residual is below tol or max_iters iterations have run,
 * exactly as fbp_set_evidence followed by fbp_run on the same graph would:
 * the arithmetic is the plain path's, so a result does not depend on which
 * other requests ran at the same time.
 *
 * Scheduling (continuous batching).  A worker thread owned by the server
 * admits work at every tick: a session is loaded onto the device when its
 * memory fits the HBM budget (otherwise it waits until closed sessions free
 * memory); a request starts when its session has no request running (requests
 * to one session run one at a time in submission order) and fewer than
 * max_inflight requests are running.  Every running request advances by
 * iters_per_tick iterations per tick on its session's own stream, so the
 * kernels of all running requests overlap on the device, and a request that
 * arrives while others run joins at the next tick.  Static strategies run
 * their persistent level engine (one launch per request); those launches are
 * serialised among themselves (one grid-wide engine at a time) but overlap
 * with flooding sessions.
 *
 * Threading: every entry point may be called from any host thread.  The
 * server's device is the device current when fbp_server_create is called.
 * Device memory of sessions comes from cudaMalloc and is counted against the
 * budget byte for byte.
 */
#ifndef FBP_SERVE_H
#define FBP_SERVE_H

#include "fbp.h"
#include "fbp_batch.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fbp_server fbp_server;

typedef struct {
    int64_t hbm_budget_bytes;  /* device bytes resident sessions may hold; 0 = no limit */
    int32_t max_inflight;      /* requests running at once; 0 = 64 */
    int32_t iters_per_tick;    /* flooding iterations queued per session per tick; 0 = 16 */
} fbp_server_config;

/* Request states. */
enum { FBP_REQ_QUEUED = 0, FBP_REQ_RUNNING = 1, FBP_REQ_DONE = 2, FBP_REQ_FAILED = 3 };

typedef struct {
    int32_t state;        /* FBP_REQ_* */
    int32_t status;       /* DONE: FBP_OK (converged) or FBP_NOT_CONVERGED; FAILED: the error code */
    int32_t iters;        /* iterations the re-run took */
    int32_t session;
    double residual;      /* residual of the last iteration */
    double queue_ms;      /* submission -> start (host clock) */
    double latency_ms;    /* submission -> result available (host clock) */
    double device_ms;     /* device time from the clamp to the last kernel of the run (CUDA events) */
} fbp_request_info;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t ticks;             /* worker ticks that launched work */
    int64_t kernel_launches;
    int64_t resident_bytes;    /* device bytes held by loaded sessions now */
    int64_t peak_resident_bytes;
    int32_t sessions_resident, sessions_waiting;
    int32_t sessions_warming;  /* resident sessions whose load-time run has not finished */
    int32_t peak_inflight;     /* most requests running in one tick */
} fbp_server_stats;

/* Create a server (and its worker thread) on the current device.
 * FBP_ERR_INVALID_ARG for negative fields; FBP_ERR_CUDA if the device cannot
 * be queried. */
int fbp_server_create(const fbp_server_config *cfg, fbp_server **out);

/* Open a session: the graph's arrays are copied (borrowed for the call only;
 * layout as fbp_graph_create).  graph->schedule.strategy is PARALL or a static
 * strategy (RESIDUAL is rejected); graph->max_iters and graph->tol apply to
 * every request of the session.  The session is loaded (device arrays,
 * schedule, then one run from uniform messages to its stopping rule -- the
 * state requests warm-start from) as soon as its memory fits the budget;
 * requests submitted before that wait.  FBP_ERR_INVALID_ARG for a bad graph,
 * or one whose estimated size exceeds the whole budget; FBP_ERR_SCHEDULE for
 * TOPO on a cyclic graph. */
int fbp_server_session_open(fbp_server *s, const fbp_graph_desc *graph, int32_t *session_out);

/* Close a session once its queued and running requests have finished; its
 * device memory is freed and counted off the budget.  Blocks until then. */
int fbp_server_session_close(fbp_server *s, int32_t session);

/* Submit a request: clamp variable var of the session to value (0 or 1; -1
 * removes the clamp) and re-run.  result_p1 (may be NULL): [n_vars of the
 * session] buffer, host (result_is_device = 0) or device memory, that
 * receives the marginals P(x=1) after the re-run (Eq. 3); it must stay valid
 * until the request is done.  *ticket_out identifies the request.
 * FBP_ERR_INVALID_ARG for an unknown or closing session, var out of range or
 * a bad value. */
int fbp_server_submit(fbp_server *s, int32_t session, int32_t var, int8_t value, float *result_p1,
                      int result_is_device, int64_t *ticket_out);

/* Current state of a request (does not block). */
int fbp_server_poll(fbp_server *s, int64_t ticket, fbp_request_info *info);

/* Block until the request is done or failed, then as fbp_server_poll. */
int fbp_server_wait(fbp_server *s, int64_t ticket, fbp_request_info *info);

/* Block until every submitted request is done or failed. */
int fbp_server_drain(fbp_server *s);

int fbp_server_get_stats(fbp_server *s, fbp_server_stats *out);

/* Finish running requests, fail queued ones, free everything. */
void fbp_server_destroy(fbp_server *s);

#ifdef __cplusplus
}
#endif
#endif /* FBP_SERVE_H */
