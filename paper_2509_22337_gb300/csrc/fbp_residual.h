// Device-side schedule of the RESIDUAL strategy (fbp_residual.cu).
#pragma once

#include "fbp_internal.h"

namespace fbp {

// Slots of the schedule's control words.
constexpr int kRsActive = 0;  // active edges this iteration
constexpr int kRsCut1 = 1;    // first edge of the level that class 1 opens (INT_MAX: none)
constexpr int kRsCut2 = 2;    // same for class 2

struct ResidualWork {
    unsigned *vres = nullptr; // [nv] largest change into each variable (float bits)
    int *cnt = nullptr;       // [nv] 1 if a NextSet edge enters the variable
    int8_t *fcls = nullptr;   // [na] class of each factor (-1: skipped)
    int8_t *elev = nullptr;   // [ne] level of each edge this iteration (-1: skipped)
    int *ctl = nullptr;       // [4] control words (kRs*)
};

// Classes of the factors from the previous iteration's per-edge changes
// (dres), then Algorithm 2's levels over the active edges, all on the device:
// w.elev and w.ctl hold the result (read ctl after the stream reaches it).
void residual_schedule(const DevGraph &g, const float *dres, double tol, ResidualWork &w, cudaStream_t s);

}  // namespace fbp
