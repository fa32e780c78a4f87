// Internal interface between the host side (fbp_host.cpp) and the CUDA
// kernels (fbp_kernels.cu) of the belief-propagation library.
//
// Message encoding.  A binary message (m0, m1) is stored as one float rho:
//   rho >= +0  means (m0, m1) proportional to (rho, 1)   [m1 is the larger]
//   rho <= -0  means (m0, m1) proportional to (1, -rho)  [m0 is the larger]
// so |rho| in [0, 1] is the smaller entry over the larger one and the sign bit
// says which entry is the larger.  +0 is the hard message (0, 1), -0 the hard
// message (1, 0), +-1 the uniform message.  This keeps the full FP32 relative
// precision of both normalised entries in 4 bytes instead of 8, and decoding
// is a select, not a transcendental.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fbp {

constexpr int kTypeAND = 0, kTypeOR = 1, kTypeNOT = 2, kTypeEQ = 3, kTypeNOISY_IMPLY = 4,
              kTypeNOISY_AND = 5, kTypePRIOR = 6, kTypeTERMS = 7;
constexpr int kTermsMaxVars = 32;    // a generic factor fits one warp
constexpr int kTermsMaxTerms = 256;

// Number of residual slots one iteration spreads its atomics over.
constexpr int kResSlots = 64;

struct DevGraph {
    int32_t nv = 0, na = 0, ne = 0;
    const int32_t *fptr = nullptr;    // [na+1] factor-major row offsets
    const uint8_t *ftype = nullptr;   // [na]
    const float *fparam = nullptr;    // [na]
    const int32_t *fvars = nullptr;   // [ne] variable of each edge
    const int32_t *efac = nullptr;    // [ne] factor of each edge
    const int32_t *vptr = nullptr;    // [nv+1] variable-major row offsets
    const int32_t *vedge = nullptr;   // [ne] edge ids of each variable, ascending
    const float *phi = nullptr;       // [nv] unary potential, rho-encoded
    // generic (TERMS) factors: term lists (other factors have none)
    const int32_t *tptr = nullptr;    // [na+1] first term of each factor
    const int32_t *tioff = nullptr;   // [na] offset of each factor's indicator block
    const int8_t *tind = nullptr;     // indicators, (terms x variables) per factor, -1 = free
    const float *tw = nullptr;        // [terms] weights
};

// Per-graph convergence state of a batch of independent graphs run together.
struct BatchCtl {
    int32_t n_graphs = 0;              // 0: a single graph (the batch fields are unused)
    int32_t *done = nullptr;           // [n_graphs] 0 running, 1 converged, 2 stopped at its max_iters
    int32_t *iters = nullptr;          // [n_graphs] iterations run
    unsigned *res = nullptr;           // [n_graphs] residual bits of the current iteration
    unsigned *last_res = nullptr;      // [n_graphs] residual bits of the graph's last iteration
    const float *tol = nullptr;        // [n_graphs]
    const int32_t *max_iters = nullptr;// [n_graphs]
    int32_t *active = nullptr;         // [1] graphs still running
};

// One half-iteration's levels, as the persistent engine reads them.
struct LevelPlanDev {
    const int4 *lanes = nullptr;       // warp-packed lane records, level after level
    const int2 *lrow = nullptr;        // per lane: {row begin, row end} of the lane's variable
    const int32_t *lane_ptr = nullptr; // [n_levels+1] (multiples of 32)
    const int32_t *big = nullptr;      // edges of factors wider than a warp
    const int32_t *big_ptr = nullptr;  // [n_levels+1]
    const int2 *vel = nullptr;         // [ne] var-major (edge id, level of the edge)
    int32_t n_levels = 0;
    int32_t level_base = 0;            // index of lane_ptr[0]'s level (per-level launches)
};

struct EngineArgs {
    DevGraph g;
    const int4 *erow = nullptr;        // [ne] {row begin, row end, variable, 0} of each edge's variable
    LevelPlanDev half[2];
    int32_t n_halves = 1;
    float *buf[2] = {nullptr, nullptr};// buf[0]: messages at launch; buf[1]: the other buffer
    unsigned *res = nullptr;           // [max_iters] residual bits per iteration (zeroed)
    unsigned long long *guards = nullptr;
    float *dres = nullptr;             // optional [ne] |dP| of each written edge
    unsigned *bar = nullptr;           // [2] barrier counter and generation (zeroed)
    int32_t *out = nullptr;            // [4] iterations, status, error word, spare (zeroed)
    int32_t max_iters = 0;
    float tol = 0.f;
    long long spin_limit = 0;          // clock64 cycles one barrier may wait
    int32_t max_lanes = 0;             // widest level of the plans, in lanes (launch shape)
    int32_t dataflow = 0;              // grid mode: per-message waits instead of a barrier per level
    int32_t fuse_lanes = 0;            // grid mode: levels of at most this many lanes run in block 0 (0: off)
    // batched graphs (n_graphs > 0): every lane record carries its graph in
    // bits 15.. of its packed word; each graph stops on its own residual.
    BatchCtl batch;
};

int engine_block();
int engine_max_fan();
int engine_max_grid();
int engine_cluster_size();
// cluster > 0: the grid is one cluster of that many blocks (hardware
// barrier); otherwise a cooperative grid of `grid` blocks.
cudaError_t launch_engine(const EngineArgs &a, int grid, int cluster, cudaStream_t s);

// One member of a batch run by the batch-queue kernel: a thread-block cluster
// takes it whole and runs it to its own stopping iteration.
struct MemberDev {
    int32_t kind = 0;                  // 0: flooding (PARALL); 1 or 2: level lists per iteration
    int32_t v0 = 0, v1 = 0;            // variables [v0, v1) of the union graph
    int32_t e0 = 0, e1 = 0;            // edges [e0, e1)
    int32_t sub0 = 0, sub1 = 0;        // flooding plan ranges: sub-chunks, medium rows,
    int32_t med0 = 0, med1 = 0;        //   hub rows, typed-factor warps, wide-list entries
    int32_t hub0 = 0, hub1 = 0;
    int32_t tw0 = 0, tw1 = 0;
    int32_t wide0 = 0, wide1 = 0;
    int32_t max_iters = 0;
    float tol = 0.f;
    LevelPlanDev half[2];              // static members: their own level lists
};

struct IterCtl {
    unsigned *res = nullptr;           // [kResSlots] residual bits of this iteration
    unsigned long long *guards = nullptr;
};

int num_sms();



// Eq. (3).
void launch_marginals(const DevGraph &g, const float *a2v, float *p1, cudaStream_t s);
// rho <-> normalised (m0, m1) pairs.
void launch_decode_pairs(const float *rho, float *pairs, int32_t n, cudaStream_t s);
void launch_encode_pairs(const float *pairs, float *rho, int32_t n, cudaStream_t s);
void launch_fill(float *x, float v, int32_t n, cudaStream_t s);

}  // namespace fbp
