// Host-side graph layout and scheduling: the factor-major CSR and its
// variable-major transpose (Sec. 4.3.2), update strategy -> integer ranks
// (Table 1, Definition 2), and the dependency analysis of Algorithm 2.
#pragma once

#include <algorithm>
#include <cstdint>
#include <thread>
#include <vector>
#include <vector_types.h>

#include "fbp.h"

namespace fbp {

// Host threads for one parallel host pass (the two halves of TOPO_FB run
// their schedule builds side by side, each with this many).
inline int host_threads()
{
    static const int t = [] {
        const unsigned hw = std::thread::hardware_concurrency();
        return (int)std::max(1u, std::min(hw / 2, 8u));
    }();
    return t;
}

// Host threads for a pass that runs alone (graph creation, the flooding
// plan): every hardware thread, at most 32.
inline int host_threads_all()
{
    static const int t = [] { return (int)std::max(1u, std::min(std::thread::hardware_concurrency(), 32u)); }();
    return t;
}

// body(begin, end) over [0, n) in up to `threads` contiguous parts, the first
// on the calling thread.  Bodies must not throw (they only write into
// preallocated arrays).
template <class Body>
inline void parallel_for(int64_t n, int threads, int64_t min_part, const Body &body)
{
    const int64_t parts = std::min<int64_t>(threads, std::max<int64_t>(1, n / std::max<int64_t>(min_part, 1)));
    if (parts <= 1) {
        body((int64_t)0, n);
        return;
    }
    const int64_t step = (n + parts - 1) / parts;
    std::vector<std::thread> pool;
    pool.reserve(parts - 1);
    for (int64_t k = 1; k < parts; ++k) {
        const int64_t b = k * step, e = std::min(n, b + step);
        if (b >= e) break;
        try {
            pool.emplace_back([&body, b, e] { body(b, e); });
        } catch (...) {  // no thread to be had: run the part here
            body(b, e);
        }
    }
    body((int64_t)0, std::min(n, step));
    for (auto &t : pool) t.join();
}

struct HostCSR {
    int32_t nv = 0, na = 0, ne = 0;
    std::vector<int64_t> fptr;    // [na+1]
    std::vector<int32_t> fvars;   // [ne]
    std::vector<uint8_t> ftype;   // [na]
    std::vector<float> fparam;    // [na]
    std::vector<int32_t> efac;    // [ne] factor of each edge
    std::vector<int32_t> vptr;    // [nv+1]
    std::vector<int32_t> vedge;   // [ne] edges of each variable, ascending id
};

// Sets the thread-local error message; returns code.
int fail(int code, const char *fmt, ...);
// Clear the thread's last error message (entry points call it first).
void clear_error();

void build_host_csr(int32_t nv, int32_t na, const int64_t *fptr, const int32_t *fvars,
                    const uint8_t *ftype, const float *fparam, HostCSR &h);

// Per-edge rank of a static strategy (PARALL, SEQFIX, TOPO, TOPO_FB, CUSTOM_RANK);
// half = 1 selects the backward half of TOPO_FB.
int build_ranks(const HostCSR &h, const fbp_schedule_spec &spec, int half, std::vector<int64_t> &rank);
// TOPO_FB's backward half from the forward ranks: max(0, ranks) - rank.
void backward_ranks(const std::vector<int64_t> &fwd, std::vector<int64_t> &bwd);

// Algorithm 2 over `edges` (all edges when NULL): canonical (rank, edge id)
// order, greedy cuts.  lp = level_ptr, le = level_edges.
void dependency_levels(const HostCSR &h, const int64_t *rank, const int32_t *edges, int64_t n,
                       std::vector<int64_t> &lp, std::vector<int32_t> &le);

// The persistent engine's plan of one level list (host copy): whole factors
// packed into warps, one lane record per edge {edge, packed word, p bits,
// variable} and the lane's row bounds; factors wider than max_fan go to the
// `big` list; vel pairs every variable-major edge with its level.
struct LevelPack {
    std::vector<int4> lanes;
    std::vector<int2> lrow;
    std::vector<int32_t> lane_ptr, big, big_ptr;
    std::vector<int2> vel;
    int32_t max_lanes = 0;
};
// fac_graph: batch member of every factor (empty for a single graph).
void pack_levels(const HostCSR &h, const std::vector<int32_t> &fac_graph, const std::vector<int64_t> &lp,
                 const std::vector<int32_t> &le, int max_fan, LevelPack &out);

// The residual strategy's classes for the next iteration from the previous
// iteration's per-edge |delta m1|; fills rank for every edge and the active
// edge list; returns the number of active edges.
int64_t residual_classes(const HostCSR &h, const float *dres, double tol, int64_t *rank,
                         std::vector<int32_t> &act);

}  // namespace fbp

struct fbp_graph;
int fbp_run_residual_device(fbp_graph *g, int32_t max_iters, double tol, int32_t *iters_out,
                            double *residual_out);
int fbp_run_residual(fbp_graph *g, int32_t max_iters, double tol, int32_t *iters_out,
                     double *residual_out);
