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

struct FloodPlanDev {
    int32_t nb_small = 0;              // blocks of the one-thread-per-row role (degree 3..8)
    int32_t n_small = 0;
    const int32_t *small = nullptr;    // [n_small] variables of degree 3..8
    int32_t nb_medium = 0;             // blocks of the warp-per-row role
    int32_t n_medium = 0;
    const int32_t *medium = nullptr;   // [n_medium] variables of medium degree
    int32_t n_hub = 0;                 // hub chunks
    const int4 *hub = nullptr;         // [n_hub] {variable, row begin, row end, first chunk of the row}
    const int32_t *hub_nchunks = nullptr;  // [n_hub] chunks of the chunk's row
    XP *agg = nullptr;                 // [n_hub] partial product of each chunk
    const int *done = nullptr;         // set once the run has converged
    // batched graphs: graph of each variable and factor; per-graph state
    const int32_t *vgraph = nullptr;
    const int32_t *fgraph = nullptr;
    BatchCtl batch;
};

// One flooding iteration (number `it`): phase 1 over every variable row,
// phase 2 over every factor (in place on a2v), then the convergence check:
// hist[it-1] receives the residual bits; done[0] is set at the first
// iteration below tol and done[1] holds the last iteration executed.  Every
// kernel returns at once when done[0] is set, so iterations can be queued in
// batches without a host synchronisation per iteration.  `staged` = factor
// row entries staged in shared memory per block (flood_smem_bytes of it).
void flood_iteration(const DevGraph &g, const FloodPlanDev &F, float *a2v, float *v2a, IterCtl ctl,
                     int staged, int it, float tol, unsigned *hist, int *done, cudaStream_t s);
size_t flood_smem_bytes(int staged);
void flood_prepare(size_t smem_bytes);

}  // namespace fbp
