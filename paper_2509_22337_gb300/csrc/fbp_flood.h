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
static_assert(sizeof(XP) == 24 && alignof(XP) == 4, "XP: three 8-byte pairs");

constexpr int kFloodSmallMax = 8;      // rows up to this degree: one thread each, in row order
constexpr int kFloodSub = 32;          // the grouping unit of a longer row's product
constexpr int kFloodMediumMax = 256;   // rows up to this degree may combine in one thread
static_assert(kFloodMediumMax <= 8 * kFloodSub, "a medium row has at most 8 sub-chunks");
constexpr int kFloodSlots = 256;       // slots of a longer row's product (one block's threads)
static_assert(kFloodSlots >= 64 && (kFloodSlots & (kFloodSlots - 1)) == 0, "a power of two above a warp");
constexpr int kFloodChunkUnit = 256;   // FBP_OPT_FLOOD_CHUNK is a multiple of this many entries
constexpr int kFloodHubChunk = 8192;   // entries per block of the sub-chunk pass (default)
static_assert(kFloodHubChunk % kFloodChunkUnit == 0 && kFloodChunkUnit % kFloodSub == 0, "whole sub-chunks");
constexpr int kFloodChunk = 8;         // iterations per captured CUDA graph

struct FloodPlanDev {
    // phase 1 (beliefs, variable-major): every variable of degree <= 8 one
    // thread (nb_vars blocks stepping through the variables); every longer row in 32-entry
    // sub-chunks, one thread each (a row of one sub-chunk writes its belief
    // there); then one thread per medium row (2..8 sub-chunks) or one block per
    // hub row combines the sub-chunk products
    int32_t nb_vars = 0;
    int32_t n_subs = 0;
    const int4 *subs = nullptr;        // [n_subs] {variable, begin, end, agg slot or -1: the row's only one}
    int32_t sub_threads = 0;           // threads per block of the sub-chunk pass
    int32_t nb_medium = 0;             // blocks of the thread-per-medium-row role
    int32_t n_medium = 0;
    const int4 *medium = nullptr;      // [n_medium] {variable, first agg slot, sub-chunks, 0}, by sub-chunk count
    int32_t n_hub_rows = 0;
    const int4 *hub_row = nullptr;     // [n_hub_rows] {variable, first agg slot, sub-chunks, 0}
    XP *agg = nullptr;                 // product of each sub-chunk of a row of several
    uint2 *belief = nullptr;           // [nv] belief record of each variable (see fbp_flood.cu)
    // phase 2 (factor-major): runs of consecutive typed factors of at most
    // 32 variables in warps of whole factors (twarps); runs of consecutive
    // generic factors likewise (warps); factors wider than a warp edge by edge
    int32_t n_twarps = 0;
    const int4 *twarps = nullptr;      // [n_twarps] {first edge, end edge, first factor, end factor}
    int32_t n_warps = 0;
    const int4 *warps = nullptr;       // [n_warps] {first edge, end edge, first factor, end factor}
    int32_t n_wide = 0;
    const int32_t *wide = nullptr;     // [n_wide] edges of factors wider than a warp, factor by factor
    float *wide_v2a = nullptr;         // [n_wide] their v->a messages, formed before phase 2
    const int32_t *vpos = nullptr;     // [ne] slot of each edge in the variable-major message copy
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

// The batch-queue kernel's arguments.  Each thread-block cluster takes the
// next member from the queue (order[queue++]) and runs it to completion;
// clusters never wait on one another.
struct QueueArgs {
    DevGraph g;                        // the union graph of every member
    const int4 *erow = nullptr;        // [ne] engine row records (static members)
    float *a2v = nullptr;              // messages in and out (factor-major)
    float *a2v_alt = nullptr;          // the static members' second buffer
    float *a2v_vm = nullptr;           // flooding members' variable-major copy
    FloodPlanDev F;                    // the union's flooding plan (flooding members' ranges)
    const MemberDev *members = nullptr;
    const int32_t *order = nullptr;    // members by descending work
    int32_t n_members = 0;
    int32_t *queue = nullptr;          // [1] next position in order (zeroed per run)
    unsigned *cbar = nullptr;          // [clusters] barrier counter of each cluster (zeroed per run)
    unsigned *cres = nullptr;          // [clusters] residual word of each cluster's current iteration
    int32_t *cword = nullptr;          // [clusters * 4] words one block publishes to its cluster
    int32_t *out_iters = nullptr;      // [n_members]
    int32_t *out_status = nullptr;     // [n_members] 0 converged, 1 stopped at max_iters
    unsigned *out_res = nullptr;       // [n_members] residual bits of the last iteration
    unsigned long long *guards = nullptr;
    int32_t *err = nullptr;            // [1] set when a barrier wait expired
    long long spin_limit = 0;
};
// Clusters of `cluster` (8 or 16) blocks of the batch-queue kernel that can be
// resident at once (0 if the device cannot launch it).
int batch_queue_clusters(int cluster);
cudaError_t launch_batch_queue(const QueueArgs &q, int cluster, int clusters, cudaStream_t s);

// The flooding kernels keep two copies of the a->v messages: a2v in the
// factor-major (edge id) order every other part of the library uses, and
// a2v_vm in variable-major order (slot k of variable v's row holds the
// message of edge vedge[k]), which phase 1 reads contiguously.  Phase 2
// writes both.  flood_sync makes a2v_vm a copy of a2v; call it before the
// first flooding iteration whenever a2v was written by anything else
// (reset, import, the level engine).
void flood_sync(const DevGraph &g, const float *a2v, float *a2v_vm, cudaStream_t s);
// One flooding iteration: phase 1 over every variable row, phase 2 over
// every factor (in place on a2v, mirrored into a2v_vm), then the convergence
// check.  done[4] is the run's control block on the device: [0] 0 while
// running, 1 once converged (or, for a batch, once no graph runs), 2 at the
// iteration limit; [1] the last iteration executed (the device counts
// iterations itself, so queued or captured iterations need no argument); [3]
// the iteration limit.  hist[it-1] receives iteration it's residual bits.
// Every kernel returns at once when done[0] is set, so iterations can be
// queued in batches, or replayed from a captured graph, without a host
// synchronisation per iteration.
void flood_iteration(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *a2v_vm, IterCtl ctl, float tol,
                     unsigned *hist, int *done, cudaStream_t s);
// The two phases of one level of a device-scheduled RESIDUAL iteration
// (F.elevel, F.level, F.dres set): every belief from the level-start state,
// then the level's a->v messages.  No convergence check.
void flood_level(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *a2v_vm, IterCtl ctl, int *done,
                 cudaStream_t s);
// Phase 1 alone: every variable's belief record from a2v_vm (F.done must
// point to a word that reads 0).
void flood_beliefs(const DevGraph &g, const FloodPlanDev &F, const float *a2v_vm, cudaStream_t s);
// End of a device-scheduled RESIDUAL iteration: the check of flood_iteration.
void flood_check(IterCtl ctl, float tol, unsigned *hist, int *done, cudaStream_t s);
// A CUDA graph of `iters` consecutive flood_iterations (captured on a private
// stream; launch it on any stream).
cudaError_t flood_capture(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *a2v_vm, IterCtl ctl, float tol,
                          unsigned *hist, int *done, int iters, cudaGraphExec_t *exec);
// Kernel launches of one flood_iteration.
int flood_launches(const DevGraph &g, const FloodPlanDev &F);

}  // namespace fbp
