// Flooding (PARALL) plan shared by the host driver and the flooding kernels.
#pragma once

#include "fbp_internal.h"

namespace fbp {

// Product of binary messages: each entry as mantissa * 2^exponent, with exact
// zeros counted instead of multiplied in.
struct XP {
    float m0, m1;
    int e0, e1;
    int z0, z1;
};

constexpr int kFloodSmallMax = 8;      // rows up to this degree: one thread each
constexpr int kFloodMediumMax = 256;   // rows up to this degree: one warp each
constexpr int kFloodHubChunk = 1024;   // longer rows: chunks of this many entries (one block)
constexpr int kFloodSub = 256;         // the grouping unit of a long row's product (= kFloodMediumMax)
static_assert(kFloodSub == kFloodMediumMax, "a warp-per-row row is exactly one sub-chunk");
static_assert(kFloodHubChunk % kFloodSub == 0, "chunks hold whole sub-chunks");
constexpr int kFloodChunk = 8;         // iterations per captured CUDA graph

struct FloodPlanDev {
    int32_t nb_small = 0;              // blocks of the one-thread-per-row role (degree 3..8)
    int32_t n_small = 0;
    const int32_t *small = nullptr;    // [n_small] variables of degree 3..8
    int32_t nb_medium = 0;             // blocks of the warp-per-row role
    int32_t n_medium = 0;
    const int32_t *medium = nullptr;   // [n_medium] variables of medium degree
    int32_t n_hub = 0;                 // hub chunks
    const int4 *hub = nullptr;         // [n_hub] {variable, chunk begin, chunk end, first sub-chunk of the chunk}
    const int2 *hub_row = nullptr;     // [n_hub] {first sub-chunk of the chunk's row, sub-chunks of the row}
    XP *agg = nullptr;                 // [sub-chunks of all hub rows] partial product of each sub-chunk
    // phase 2: warps of whole consecutive factors; factors wider than a warp
    // edge by edge
    int32_t n_warps = 0;
    const int4 *warps = nullptr;       // [n_warps] {first edge, end edge, first factor, end factor}
    int32_t n_wide = 0;
    const int32_t *wide = nullptr;     // [n_wide] edges of factors wider than a warp
    const int *done = nullptr;         // set once the run has converged
    // one level of the device-scheduled RESIDUAL strategy: phase 2 writes only
    // the edges with elevel[e] == level, and records each written edge's
    // |dP(x=1)| in dres (unused when elevel is null)
    const int8_t *elevel = nullptr;
    int32_t level = 0;
    float *dres = nullptr;
    // batched graphs: graph of each variable and factor; per-graph state
    const int32_t *vgraph = nullptr;
    const int32_t *fgraph = nullptr;
    BatchCtl batch;
};

// One flooding iteration: phase 1 over every variable row, phase 2 over
// every factor (in place on a2v), then the convergence check.  done[4] is the
// run's control block on the device: [0] 0 while running, 1 once converged
// (or, for a batch, once no graph runs), 2 at the iteration limit; [1] the
// last iteration executed (the device counts iterations itself, so queued or
// captured iterations need no argument); [3] the iteration limit.
// hist[it-1] receives iteration it's residual bits.  Every kernel returns at
// once when done[0] is set, so iterations can be queued in batches, or
// replayed from a captured graph, without a host synchronisation per
// iteration.
void flood_iteration(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *v2a, IterCtl ctl, float tol,
                     unsigned *hist, int *done, cudaStream_t s);
// The two phases of one level of a device-scheduled RESIDUAL iteration
// (F.elevel, F.level, F.dres set): every v->a message from the level-start
// state, then the level's a->v messages.  No convergence check.
void flood_level(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *v2a, IterCtl ctl, int *done,
                 cudaStream_t s);
// End of a device-scheduled RESIDUAL iteration: the check of flood_iteration.
void flood_check(IterCtl ctl, float tol, unsigned *hist, int *done, cudaStream_t s);
// A CUDA graph of `iters` consecutive flood_iterations (captured on a private
// stream; launch it on any stream).
cudaError_t flood_capture(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *v2a, IterCtl ctl, float tol,
                          unsigned *hist, int *done, int iters, cudaGraphExec_t *exec);
// Kernel launches of one flood_iteration.
int flood_launches(const DevGraph &g, const FloodPlanDev &F);

}  // namespace fbp
