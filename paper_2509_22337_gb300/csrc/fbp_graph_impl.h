// Internal state of a graph handle and the host helpers shared by the
// single-graph C ABI (fbp_host.cpp) and the batched form (fbp_batch.cpp).
#pragma once

#include <cstdint>
#include <vector>

#include "fbp.h"
#include "fbp_flood.h"
#include "fbp_internal.h"
#include "fbp_sched.h"
#include "fbp_residual.h"

using fbp::DevGraph;
using fbp::FloodPlanDev;
using fbp::HostCSR;
using fbp::LevelPlanDev;

struct LevelSet {                    // one level list (one half of TOPO_FB)
    std::vector<int64_t> lp;         // level_ptr (Algorithm 2's S)
    std::vector<int32_t> le;         // level_edges (canonical order)
    // engine plan (device)
    int4 *d_lanes = nullptr;
    int2 *d_lrow = nullptr;
    int32_t *d_lane_ptr = nullptr, *d_big = nullptr, *d_big_ptr = nullptr;
    int2 *d_vel = nullptr;
    int32_t max_lanes = 0;           // widest level, in lanes
    int64_t n_lanes = 0;
};

// One level list of the belief-form sequential engine (FBP_OPT_ENGINE = 3):
// per level, its edges and the work that keeps the beliefs current after
// the level's writes.
struct SeqHalf {
    int32_t n_levels = 0;
    int32_t max_level = 0;           // edges of the widest level
    int32_t *lp = nullptr;           // [n_levels + 1] level starts in le
    int32_t *le = nullptr;           // level edges
    int4 *dp = nullptr;              // [n_levels + 1] starts of {short items, sub-chunk items, whole medium rows, whole hub rows}
    int4 *ds = nullptr;              // short rows to recompute {variable, patch begin, patch end, 0}
    int4 *dk = nullptr;              // sub-chunks to recompute {sub-chunk, patch begin, patch end, finish}
    int32_t *dm = nullptr;           // medium rows with several touched sub-chunks
    int32_t *dh = nullptr;           // hub rows with several touched sub-chunks
    int2 *pt = nullptr;              // patches {position in the row or sub-chunk, index in the level}
};

struct fbp_graph {
    HostCSR h;                        // host CSR + transpose (also used by scheduling)
    std::vector<float> prior;
    std::vector<int8_t> evidence;
    std::vector<float> phi;           // rho-encoded unary potentials
    DevGraph d;
    cudaStream_t stream = nullptr;
    fbp_allocator alloc{};
    bool has_alloc = false;
    std::vector<void *> owned;
    // messages
    float *a2v[2] = {nullptr, nullptr};
    int cur = 0;
    float *a2v_vm = nullptr;          // flooding: variable-major copy of the a->v messages [E]
    float *pairs = nullptr;           // export/import staging [2E]
    float *p1 = nullptr;              // marginals [V]
    int32_t *marg_rows = nullptr;     // variables whose rows exceed marginals_row_max() (built at first use)
    int32_t n_marg_rows = -1;         // -1: not built yet
    // schedule
    int strategy = FBP_PARALL;
    std::vector<LevelSet> halves;     // 1 (static) or 2 (TOPO_FB)
    // residual strategy working state
    float *dres = nullptr;            // [E] |delta m1| of the last write
    int32_t *d_act = nullptr;         // [E] active edges (residual)
    // persistent engine
    int4 *erow = nullptr;             // [E] row record of each edge's variable
    unsigned *d_res_it = nullptr;     // [res_cap] residual bits per iteration
    int32_t res_cap = 0;
    unsigned *d_bar = nullptr;        // [2] barrier words
    int32_t *d_out = nullptr;         // [4] engine outputs
    int32_t *h_out = nullptr;         // pinned copy
    long long spin_limit = 4000000000LL;
    int engine_grid = 0;              // 0 = automatic
    int engine_cluster = 0;           // 0 = automatic, 1 = never, 8 or 16 = cluster size
    int engine_fuse = 0;              // level fusion: narrow levels (<= this many lanes) in one block (0: off)
    int engine_solo = 128;            // whole run in one block when levels average <= this many lanes
    int use_engine = 1;
    // flooding plan, with host copies of its row lists (the sequential
    // engine's plan indexes them)
    FloodPlanDev flood;
    bool flood_ready = false;
    std::vector<int4> flood_subs_h, flood_medium_h, flood_hub_h;
    // belief-form sequential engine: plan (built for the current flooding
    // plan and schedule; empty when stale) and the staging of wide levels
    std::vector<SeqHalf> seq;
    float *seq_tmp = nullptr;
    int64_t seq_tmp_cap = 0;
    fbp::XP *seq_tree = nullptr;      // butterfly nodes of every hub row
    // captured chunk of flooding iterations and what it was captured for
    cudaGraphExec_t flood_exec = nullptr;
    int flood_exec_iters = 0;
    float flood_exec_tol = 0.f;
    const void *flood_exec_key[3] = {nullptr, nullptr, nullptr};  // messages, residual words, plan
    // per-iteration control
    unsigned *d_res = nullptr;
    unsigned long long *d_guards = nullptr;
    unsigned *h_res = nullptr;        // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    fbp_stats stats{};
    // flooding split: rows longer than flood_hub_min run in chunks of
    // flood_chunk entries (tunable; see FBP_OPT_FLOOD_*)
    int flood_hub_min = fbp::kFloodMediumMax;
    int flood_chunk = fbp::kFloodHubChunk;
    // RESIDUAL: schedule built on the device (default) or on the host
    bool residual_device = true;
    fbp::ResidualWork rs;
    bool rs_levels_pending = false;   // the last device iteration's levels are not on the host yet
    // generic factors: present in the graph, and their term lists uploaded
    bool terms_needed = false;
    bool terms_set = false;
    // batched union graphs: the batch member of every factor (empty for a
    // single graph); lane records carry it in bits 15.. of their packed word
    std::vector<int32_t> fac_graph;
};


namespace fbp {

int dalloc(fbp_graph *g, void **p, size_t bytes);
void dfree(fbp_graph *g, void *p);
template <class T>
int dalloc_n(fbp_graph *g, T **p, size_t n)
{
    return dalloc(g, (void **)p, n * sizeof(T));
}
template <class T>
int upload(fbp_graph *g, T **p, const T *src, size_t n)
{
    int rc = dalloc_n(g, p, n);
    if (rc) return rc;
    if (n) {
        cudaError_t e = cudaMemcpyAsync(*p, src, n * sizeof(T), cudaMemcpyHostToDevice, g->stream);
        if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(e));
    }
    return FBP_OK;
}
void free_levels_one(fbp_graph *g, LevelSet &ls);
void free_levels(fbp_graph *g);
// The belief-form sequential engine (csrc/fbp_seq.cu): drop its plan (after
// the schedule or the flooding plan changed), and run a static schedule.
void free_seq(fbp_graph *g);
int run_seq(fbp_graph *g, int32_t max_iters, double tol, int32_t *iters_out, double *residual_out);
// Upload a level list's engine plan: `packed` when given (pack_levels of the
// same list), else packed here.
int upload_levels(fbp_graph *g, LevelSet &ls, const fbp::LevelPack *packed = nullptr);
int build_flood_plan(fbp_graph *g, const std::vector<int4> *ranges = nullptr,
                     std::vector<fbp::MemberDev> *slices = nullptr);
int ensure_res_cap(fbp_graph *g, int32_t n);
LevelPlanDev plan_of(const LevelSet &ls);
void engine_shape(const fbp_graph *g, int *grid, int *cluster);
EngineArgs engine_args(fbp_graph *g);
int engine_check(fbp_graph *g);
int check_graph_args(int32_t nv, int32_t na, const int64_t *fptr, const int32_t *fvars, const uint8_t *ftype,
                     const float *fparam, const float *prior, const int8_t *evidence);
int finish_run(fbp_graph *g, int32_t it, double res, int status, int32_t *iters_out, double *residual_out);
double residual_at(fbp_graph *g, int32_t it);
// Marginals of every variable of g's current messages into device buffer
// dst on stream s: rows of at most marginals_row_max() entries one thread
// each, longer rows one block each (csrc/fbp_kernels.cu).
int marginals_launch(fbp_graph *g, float *dst, cudaStream_t s);
int marginals_row_max();
void launch_marginals_long(const DevGraph &g, const float *a2v, float *p1, const int32_t *rows, int32_t n,
                           cudaStream_t s);
// The graph's captured chunk of `iters` flooding iterations under plan F and
// tolerance tol (captured again when any of them, the message buffer or the
// residual words changed).
int flood_exec_for(fbp_graph *g, const FloodPlanDev &F, float tol, int iters, cudaGraphExec_t *out);
int fetch_residual_levels(fbp_graph *g);
void flood_exec_drop(fbp_graph *g);

}  // namespace fbp
