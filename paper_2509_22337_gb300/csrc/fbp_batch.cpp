// Batched form (include/fbp_batch.h): many independent graphs in one run.
//
// The graphs are split by the shape of their iteration: flooding (PARALL)
// graphs form one union graph run by the flooding kernels; graphs with a
// static strategy form one union graph per number of level lists per
// iteration (one for SEQFIX/TOPO/CUSTOM_RANK, two for TOPO_FB), run by one
// persistent level-engine launch.  Each member keeps the levels of its own
// Algorithm 2 (a union-wide Algorithm 2 would cut levels where another graph
// needs a cut, which changes a member's semantics); level k of every member
// is merged into level k of the union.  Members carry their own tolerance and
// iteration limit; the device marks each one done at its own stopping
// iteration and freezes its messages, so every member ends exactly where a
// single-graph run of it ends.  The parts run concurrently on separate streams.
#include "fbp_batch.h"
#include "fbp_graph_impl.h"

#include <algorithm>
#include <thread>
#include <atomic>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

using namespace fbp;

namespace {

enum { kFlood = 0, kStatic1 = 1, kStatic2 = 2, kQueue = 3, kParts = 4 };

struct Part {
    fbp_graph *g = nullptr;
    std::vector<int32_t> members;          // batch indices
    std::vector<int32_t> var_off, fac_off, edge_off;
    int32_t max_iters = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // device per-member state
    int32_t *done = nullptr, *iters = nullptr, *active = nullptr;
    unsigned *res = nullptr, *last_res = nullptr;
    float *tol = nullptr;
    int32_t *maxit = nullptr;
    int32_t *vgraph = nullptr, *fgraph = nullptr;
    // the one-launch part (every member): member records and queue state
    std::vector<MemberDev> mem;        // host copy of the member records
    MemberDev *d_members = nullptr;
    int32_t *d_order = nullptr;
    int32_t *d_qwords = nullptr;       // [2 + 4 * clusters]: queue position, error word, per-cluster words
    unsigned *d_cbar = nullptr;        // [2 * clusters]: barrier counters, residual words
    int32_t *d_out = nullptr;          // [3 * members]: iterations, status, residual bits
    int cluster = 8;                   // blocks per cluster (8 or 16)
    int clusters = 0;                  // clusters launched (resident at once)
    int cap8 = 0;                      // clusters the queue words are sized for (the 8-block count)
    bool has_flood = false;
    cudaGraphExec_t exec = nullptr;    // the captured run
    BatchCtl ctl() const
    {
        BatchCtl c;
        c.n_graphs = (int32_t)members.size();
        c.done = done;
        c.iters = iters;
        c.res = res;
        c.last_res = last_res;
        c.tol = tol;
        c.max_iters = maxit;
        c.active = active;
        return c;
    }
};

int kind_of(int strategy)
{
    if (strategy == FBP_PARALL) return kFlood;
    if (strategy == FBP_TOPO_FB) return kStatic2;
    return kStatic1;
}

}  // namespace

struct fbp_batch {
    int32_t n = 0;
    std::vector<int32_t> part_of, slot_of;  // per batch graph: part and member index
    std::vector<int32_t> nv, ne;
    Part parts[kParts];
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evp[kParts] = {nullptr, nullptr, nullptr, nullptr};
    bool one_launch = false;
    fbp_batch_tuning tuning{0, 0, 0, 0, -1, -1, 0};
    fbp_stats stats{};
    float *scratch = nullptr;  // [largest union] marginals / pairs staging
    size_t scratch_n = 0;
};

namespace {

// One union graph of the part's members: their arrays side by side (variable,
// factor and edge ids offset per member), fac_graph / var_graph the member of
// every factor / variable.
int build_union(Part &P, const fbp_graph_desc *graphs, const fbp_allocator *alloc, std::vector<int32_t> &var_graph)
{
    // every member's offsets first, then each member copied into place (the
    // members on every host thread)
    const size_t m = P.members.size();
    int32_t nv = 0, na = 0;
    int64_t ne = 0;
    for (size_t k = 0; k < m; ++k) {
        const fbp_graph_desc &d = graphs[P.members[k]];
        P.var_off.push_back(nv);
        P.fac_off.push_back(na);
        P.edge_off.push_back((int32_t)ne);
        nv += d.n_vars;
        na += d.n_factors;
        ne += d.factor_ptr[d.n_factors];
        P.max_iters = std::max(P.max_iters, d.max_iters);
    }
    if (ne >= (int64_t)1 << 31) return fail(FBP_ERR_INVALID_ARG, "batch part too large (%lld edges)", (long long)ne);
    std::vector<int64_t> fptr((size_t)na + 1, 0);
    std::vector<int32_t> fvars((size_t)ne), fac_graph((size_t)na);
    std::vector<uint8_t> ftype((size_t)na);
    std::vector<float> fparam((size_t)na), prior((size_t)nv);
    std::vector<int8_t> ev((size_t)nv);
    var_graph.resize((size_t)nv);
    std::atomic<size_t> next{0};
    auto work = [&] {
        for (size_t k; (k = next.fetch_add(1)) < m;) {
            const fbp_graph_desc &d = graphs[P.members[k]];
            const int32_t v0 = P.var_off[k], a0 = P.fac_off[k];
            const int64_t e0 = P.edge_off[k];
            for (int32_t a = 0; a < d.n_factors; ++a) {
                for (int64_t e = d.factor_ptr[a]; e < d.factor_ptr[a + 1]; ++e) fvars[e0 + e] = d.factor_vars[e] + v0;
                fptr[a0 + a + 1] = e0 + d.factor_ptr[a + 1];
                ftype[a0 + a] = d.factor_type[a];
                fparam[a0 + a] = d.factor_param[a];
                fac_graph[a0 + a] = (int32_t)k;
            }
            for (int32_t v = 0; v < d.n_vars; ++v) {
                prior[v0 + v] = d.prior_p1 ? d.prior_p1[v] : std::numeric_limits<float>::quiet_NaN();
                ev[v0 + v] = d.evidence ? d.evidence[v] : (int8_t)-1;
                var_graph[v0 + v] = (int32_t)k;
            }
        }
    };
    const int threads = std::max(1, std::min<int>(host_threads_all(), (int)m));
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) {
        try {
            pool.emplace_back(work);
        } catch (...) {  // no thread to be had: the others take its members
            break;
        }
    }
    work();
    for (auto &th : pool) th.join();

    int rc = fbp_graph_create(nv, na, fptr.data(), fvars.data(), ftype.data(), fparam.data(), prior.data(),
                              ev.data(), alloc, P.stream, &P.g);
    if (rc) return rc;
    P.g->fac_graph = std::move(fac_graph);
    return FBP_OK;
}

// Every static member's own Algorithm 2 level lists (one per half), built on
// every host thread, members taken in turn (their sizes differ); the
// callers concatenate them in member order, so the result is the one a
// member-by-member loop builds.  rc and msg hold a member's failure.
struct MemberLevels {
    std::vector<int64_t> lp[2];
    std::vector<int32_t> le[2];
    int rc = FBP_OK;
    std::string msg;
};

void member_levels(const fbp_graph_desc *graphs, const std::vector<int32_t> &members, const std::vector<int> &halves,
                   std::vector<MemberLevels> &out)
{
    const int32_t m = (int32_t)members.size();
    out.assign(m, MemberLevels{});
    std::atomic<int32_t> next{0};
    auto work = [&] {
        for (int32_t k; (k = next.fetch_add(1)) < m;) {
            if (halves[k] == 0) continue;
            const fbp_graph_desc &d = graphs[members[k]];
            HostCSR h;
            build_host_csr(d.n_vars, d.n_factors, d.factor_ptr, d.factor_vars, d.factor_type, d.factor_param, h);
            for (int hf = 0; hf < halves[k]; ++hf) {
                std::vector<int64_t> rank;
                const int rc = build_ranks(h, d.schedule, hf, rank);
                if (rc) {
                    out[k].rc = rc;
                    out[k].msg = fbp_last_error();  // this thread's message
                    break;
                }
                dependency_levels(h, rank.data(), nullptr, h.ne, out[k].lp[hf], out[k].le[hf]);
            }
        }
    };
    const int threads = std::max(1, std::min<int>(host_threads_all(), m));
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) {
        try {
            pool.emplace_back(work);
        } catch (...) {  // no thread to be had: the others take its members
            break;
        }
    }
    work();
    for (auto &th : pool) th.join();
}

int build_part(fbp_batch *b, int kind, const fbp_graph_desc *graphs, const fbp_allocator *alloc)
{
    Part &P = b->parts[kind];
    if (P.members.empty()) return FBP_OK;
    std::vector<int32_t> var_graph;
    int rc = build_union(P, graphs, alloc, var_graph);
    if (rc) return rc;
    fbp_graph *g = P.g;
    const std::vector<int32_t> &fac_graph = g->fac_graph;
    const int32_t m = (int32_t)P.members.size();
    // per-member state
    std::vector<float> tol(m);
    std::vector<int32_t> maxit(m);
    for (int32_t k = 0; k < m; ++k) {
        tol[k] = (float)graphs[P.members[k]].tol;
        maxit[k] = graphs[P.members[k]].max_iters;
    }
    if ((rc = dalloc_n(g, &P.done, m)) || (rc = dalloc_n(g, &P.iters, m)) || (rc = dalloc_n(g, &P.active, 1)) ||
        (rc = dalloc_n(g, &P.res, m)) || (rc = dalloc_n(g, &P.last_res, m)) ||
        (rc = upload(g, &P.tol, tol.data(), tol.size())) || (rc = upload(g, &P.maxit, maxit.data(), maxit.size())))
        return rc;
    if (kind == kFlood) {
        g->strategy = FBP_PARALL;
        if ((rc = upload(g, &P.vgraph, var_graph.data(), var_graph.size())) ||
            (rc = upload(g, &P.fgraph, fac_graph.data(), fac_graph.size())) || (rc = build_flood_plan(g)))
            return rc;
        if (!g->a2v_vm && (rc = dalloc_n(g, &g->a2v_vm, (size_t)g->h.ne))) return rc;
        return FBP_OK;
    }
    // static parts: each member's own levels, merged by level index
    const int halves = kind == kStatic2 ? 2 : 1;
    std::vector<MemberLevels> ml;
    member_levels(graphs, P.members, std::vector<int>(m, halves), ml);
    for (int32_t k = 0; k < m; ++k)
        if (ml[k].rc) return fail(ml[k].rc, "batch graph %d: %s", P.members[k], ml[k].msg.c_str());
    std::vector<LevelSet> merged(halves);
    for (int hf = 0; hf < halves; ++hf) {
        size_t nl = 0;
        for (int32_t k = 0; k < m; ++k) nl = std::max(nl, ml[k].lp[hf].size() - 1);
        LevelSet &ls = merged[hf];
        ls.lp.assign(1, 0);
        for (size_t L = 0; L < nl; ++L) {
            for (int32_t k = 0; k < m; ++k) {
                const std::vector<int64_t> &lpk = ml[k].lp[hf];
                if (L + 1 >= lpk.size()) continue;
                for (int64_t i = lpk[L]; i < lpk[L + 1]; ++i) ls.le.push_back(ml[k].le[hf][i] + P.edge_off[k]);
            }
            ls.lp.push_back((int64_t)ls.le.size());
        }
    }
    free_levels(g);
    g->halves = std::move(merged);
    g->strategy = kind == kStatic2 ? FBP_TOPO_FB : FBP_TOPO;
    for (auto &ls : g->halves)
        if ((rc = upload_levels(g, ls))) return rc;
    if (!g->a2v[1] && (rc = dalloc_n(g, &g->a2v[1], (size_t)g->h.ne))) return rc;
    return FBP_OK;
}

// The one-launch part: every member in one union graph.  Flooding members
// get their own ranges of a flooding plan built member by member; static
// members' own Algorithm 2 level lists are concatenated per half (forward
// lists of every static member, backward lists of the TOPO_FB members) and
// packed once, and each member's plan is its range of levels (the packed
// (edge, level) pairs stay valid: every edge is in exactly one member's
// levels).  Members are queued largest first.
int build_queue_part(fbp_batch *b, const fbp_graph_desc *graphs, const fbp_allocator *alloc)
{
    Part &P = b->parts[kQueue];
    if (P.members.empty()) return FBP_OK;
    std::vector<int32_t> var_graph;
    int rc = build_union(P, graphs, alloc, var_graph);
    if (rc) return rc;
    fbp_graph *g = P.g;
    const int32_t m = (int32_t)P.members.size();
    P.mem.assign(m, MemberDev{});
    std::vector<int4> ranges;
    std::vector<int32_t> flood_members;
    for (int32_t k = 0; k < m; ++k) {
        const fbp_graph_desc &d = graphs[P.members[k]];
        MemberDev &M = P.mem[k];
        const int kind = kind_of(d.schedule.strategy);
        M.kind = kind == kFlood ? 0 : kind == kStatic2 ? 2 : 1;
        M.v0 = P.var_off[k];
        M.v1 = M.v0 + d.n_vars;
        M.e0 = P.edge_off[k];
        M.e1 = M.e0 + (int32_t)d.factor_ptr[d.n_factors];
        M.max_iters = d.max_iters;
        M.tol = (float)d.tol;
        if (M.kind == 0) {
            ranges.push_back(make_int4(M.v0, M.v1, P.fac_off[k], P.fac_off[k] + d.n_factors));
            flood_members.push_back(k);
        }
    }
    if (!ranges.empty()) {
        std::vector<MemberDev> sl;
        if ((rc = build_flood_plan(g, &ranges, &sl))) return rc;
        for (size_t r = 0; r < ranges.size(); ++r) {
            MemberDev &M = P.mem[flood_members[r]];
            M.sub0 = sl[r].sub0, M.sub1 = sl[r].sub1, M.med0 = sl[r].med0, M.med1 = sl[r].med1;
            M.hub0 = sl[r].hub0, M.hub1 = sl[r].hub1, M.tw0 = sl[r].tw0, M.tw1 = sl[r].tw1;
            M.wide0 = sl[r].wide0, M.wide1 = sl[r].wide1;
        }
        if (!g->a2v_vm && (rc = dalloc_n(g, &g->a2v_vm, (size_t)std::max(g->h.ne, 1)))) return rc;
        P.has_flood = true;
    }
    // static members: their own level lists, concatenated per half
    std::vector<int64_t> lp[2] = {std::vector<int64_t>(1, 0), std::vector<int64_t>(1, 0)};
    std::vector<int32_t> le[2];
    std::vector<int32_t> base[2] = {std::vector<int32_t>(m, 0), std::vector<int32_t>(m, 0)};
    std::vector<int32_t> count[2] = {std::vector<int32_t>(m, 0), std::vector<int32_t>(m, 0)};
    bool any_static = false;
    std::vector<int> kinds(m);
    for (int32_t k = 0; k < m; ++k) kinds[k] = P.mem[k].kind;
    std::vector<MemberLevels> ml;
    member_levels(graphs, P.members, kinds, ml);
    for (int32_t k = 0; k < m; ++k) {
        if (P.mem[k].kind == 0) continue;
        any_static = true;
        if (ml[k].rc) return fail(ml[k].rc, "batch graph %d: %s", P.members[k], ml[k].msg.c_str());
        for (int hf = 0; hf < P.mem[k].kind; ++hf) {
            const std::vector<int64_t> &lpk = ml[k].lp[hf];
            const std::vector<int32_t> &lek = ml[k].le[hf];
            base[hf][k] = (int32_t)lp[hf].size() - 1;
            count[hf][k] = (int32_t)lpk.size() - 1;
            for (size_t L = 0; L + 1 < lpk.size(); ++L) {
                for (int64_t i = lpk[L]; i < lpk[L + 1]; ++i) le[hf].push_back(lek[i] + P.edge_off[k]);
                lp[hf].push_back((int64_t)le[hf].size());
            }
        }
    }
    if (any_static) {
        free_levels(g);
        g->halves.clear();
        const int nh = lp[1].size() > 1 ? 2 : 1;
        for (int hf = 0; hf < nh; ++hf) {
            LevelSet ls;
            ls.lp = std::move(lp[hf]);
            ls.le = std::move(le[hf]);
            g->halves.push_back(std::move(ls));
        }
        for (auto &ls : g->halves)
            if ((rc = upload_levels(g, ls))) return rc;
        if (!g->a2v[1] && (rc = dalloc_n(g, &g->a2v[1], (size_t)std::max(g->h.ne, 1)))) return rc;
        for (int32_t k = 0; k < m; ++k) {
            MemberDev &M = P.mem[k];
            for (int hf = 0; hf < M.kind; ++hf) {
                LevelPlanDev pl = plan_of(g->halves[hf]);
                pl.lane_ptr += base[hf][k];
                pl.big_ptr += base[hf][k];
                pl.n_levels = count[hf][k];
                pl.level_base = base[hf][k];
                M.half[hf] = pl;
            }
        }
    }
    // largest work first: edges x iterations, static lanes weighted above flooding edges
    std::vector<int32_t> order(m);
    std::vector<double> work(m);
    for (int32_t k = 0; k < m; ++k) {
        const MemberDev &M = P.mem[k];
        work[k] = (double)(M.e1 - M.e0) * std::max(M.max_iters, 1) * (M.kind == 0 ? 1.0 : 3.0 * M.kind);
        order[k] = k;
    }
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) { return work[a] > work[c]; });
    P.cap8 = std::max(batch_queue_clusters(8), batch_queue_clusters(16));
    P.cluster = 8;
    P.clusters = batch_queue_clusters(P.cluster);
    if (P.clusters < 1) return fail(FBP_ERR_CUDA, "the batch-queue kernel cannot be launched on this device");
    if ((rc = upload(g, &P.d_members, P.mem.data(), P.mem.size())) || (rc = upload(g, &P.d_order, order.data(), order.size())) ||
        (rc = dalloc_n(g, &P.d_qwords, (size_t)(2 + 4 * P.cap8))) ||
        (rc = dalloc_n(g, &P.d_cbar, (size_t)(2 * P.cap8))) || (rc = dalloc_n(g, &P.d_out, (size_t)(3 * m))))
        return rc;
    return FBP_OK;
}

// Enqueue one whole run of the one-launch part: clear the queue and cluster
// words and the guard counter, refresh the flooding members' variable-major
// copy, launch the queue kernel.  Captured once as a CUDA graph, replayed.
int queue_enqueue(fbp_batch *b, Part &P, cudaStream_t s)
{
    fbp_graph *g = P.g;
    cudaError_t e = cudaMemsetAsync(P.d_qwords, 0, sizeof(int32_t) * (2 + 4 * P.cap8), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.d_cbar, 0, sizeof(unsigned) * 2 * P.cap8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_guards, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "batch queue: %s", cudaGetErrorString(e));
    if (P.has_flood) flood_sync(g->d, g->a2v[g->cur], g->a2v_vm, s);
    QueueArgs Q;
    Q.g = g->d;
    Q.erow = g->erow;
    Q.a2v = g->a2v[g->cur];
    Q.a2v_alt = g->a2v[g->cur ^ 1];
    Q.a2v_vm = g->a2v_vm;
    Q.F = g->flood;
    Q.members = P.d_members;
    Q.order = P.d_order;
    Q.n_members = (int32_t)P.members.size();
    Q.queue = P.d_qwords;
    Q.err = P.d_qwords + 1;
    Q.cword = P.d_qwords + 2;
    Q.cbar = P.d_cbar;
    Q.cres = P.d_cbar + P.cap8;
    Q.out_iters = P.d_out;
    Q.out_status = P.d_out + P.members.size();
    Q.out_res = reinterpret_cast<unsigned *>(P.d_out + 2 * P.members.size());
    Q.guards = g->d_guards;
    Q.spin_limit = g->spin_limit;
    e = launch_batch_queue(Q, P.cluster, P.clusters, s);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "batch queue launch: %s", cudaGetErrorString(e));
    return FBP_OK;
}

int run_queue(fbp_batch *b, Part &P)
{
    fbp_graph *g = P.g;
    if (!P.exec) {
        cudaStream_t cap = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "batch queue: %s", cudaGetErrorString(e));
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        int rc = e == cudaSuccess ? queue_enqueue(b, P, cap) : FBP_ERR_CUDA;
        const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess && rc == FBP_OK) e = cudaGraphInstantiate(&P.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (rc) return rc;
        if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "batch queue capture: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaGraphLaunch(P.exec, g->stream);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "batch queue: %s", cudaGetErrorString(e));
    b->stats.kernel_launches += 1 + (P.has_flood ? 1 : 0);
    return FBP_OK;
}

int collect_queue(fbp_batch *b, Part &P, int32_t *iters_out, double *residual_out, int32_t *status_out, int *all_ok)
{
    const size_t m = P.members.size();
    std::vector<int32_t> out(3 * m);
    int32_t err = 0;
    fbp_graph *g = P.g;
    unsigned long long guards = 0;
    cudaError_t e = cudaMemcpyAsync(out.data(), P.d_out, sizeof(int32_t) * 3 * m, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, P.d_qwords + 1, sizeof err, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&guards, g->d_guards, sizeof guards, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "batch collect: %s", cudaGetErrorString(e));
    if (err) return fail(FBP_ERR_TIMEOUT, "a device-side barrier wait of the batch queue expired");
    b->stats.guards += (int64_t)guards;
    for (size_t k = 0; k < m; ++k) {
        const int32_t i = P.members[k];
        const int32_t it = out[k];
        float r;
        std::memcpy(&r, &out[2 * m + k], sizeof r);
        const int st = out[m + k] == 0 ? FBP_OK : FBP_NOT_CONVERGED;
        if (st != FBP_OK) *all_ok = 0;
        if (iters_out) iters_out[i] = it;
        if (residual_out) residual_out[i] = (double)r;
        if (status_out) status_out[i] = st;
        const MemberDev &M = P.mem[k];
        b->stats.updates += (int64_t)it * (M.e1 - M.e0) * (M.kind == 0 ? 1 : M.kind);
        b->stats.iters = std::max(b->stats.iters, it);
    }
    return FBP_OK;
}

int part_reset_state(Part &P)
{
    fbp_graph *g = P.g;
    const size_t m = P.members.size();
    cudaStream_t s = g->stream;
    cudaError_t e = cudaMemsetAsync(P.done, 0, sizeof(int32_t) * m, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.iters, 0, sizeof(int32_t) * m, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.res, 0, sizeof(unsigned) * m, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.last_res, 0, sizeof(unsigned) * m, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.active, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_guards, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_out, 0, sizeof(int32_t) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_bar, 0, sizeof(unsigned) * 2, s);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "batch reset: %s", cudaGetErrorString(e));
    return FBP_OK;
}

// Enqueue the static part's run (one persistent launch); checked later.
int launch_static(fbp_batch *b, Part &P)
{
    fbp_graph *g = P.g;
    int rc = ensure_res_cap(g, std::max(P.max_iters, 1));
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(g->d_res_it, 0, sizeof(unsigned) * std::max(P.max_iters, 1), g->stream);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "%s", cudaGetErrorString(e));
    if ((rc = part_reset_state(P))) return rc;
    EngineArgs A = engine_args(g);
    A.res = g->d_res_it;
    A.max_iters = P.max_iters;
    A.tol = 0.f;
    A.batch = P.ctl();
    if (P.max_iters <= 0) return FBP_OK;
    g->engine_grid = b->tuning.engine_grid;
    g->engine_cluster = b->tuning.engine_cluster;
    int grid = 1, cluster = 0;
    engine_shape(g, &grid, &cluster);
    e = launch_engine(A, grid, cluster, g->stream);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "engine launch: %s", cudaGetErrorString(e));
    b->stats.kernel_launches += 1;
    return FBP_OK;
}

// The flooding part: iterations queued in growing batches on its stream.
int run_flood(fbp_batch *b, Part &P)
{
    fbp_graph *g = P.g;
    int rc = part_reset_state(P);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(g->d_res, 0, sizeof(unsigned) * kResSlots, g->stream);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "%s", cudaGetErrorString(e));
    rc = ensure_res_cap(g, std::max(P.max_iters, 1));
    if (rc) return rc;
    FloodPlanDev F = g->flood;
    F.vgraph = P.vgraph;
    F.fgraph = P.fgraph;
    F.batch = P.ctl();
    // captured chunks of iterations, replayed in growing batches; the device
    // counts iterations and stops each member at its own rule
    if (P.max_iters == 0) return FBP_OK;
    cudaGraphExec_t exec = nullptr;
    if ((rc = flood_exec_for(g, F, 0.f, kFloodChunk, &exec))) return rc;
    flood_sync(g->d, g->a2v[g->cur], g->a2v_vm, g->stream);  // after the reset of part_reset_state
    b->stats.kernel_launches += g->h.ne > 0;
    g->h_out[0] = g->h_out[1] = g->h_out[2] = 0;
    g->h_out[3] = P.max_iters;
    e = cudaMemcpyAsync(g->d_out, g->h_out, sizeof(int32_t) * 4, cudaMemcpyHostToDevice, g->stream);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "flood batch: %s", cudaGetErrorString(e));
    const int per_iter = flood_launches(g->d, F);
    int32_t queued = 0, reps = 1;
    while (queued < P.max_iters) {
        for (int32_t r = 0; r < reps && queued < P.max_iters; ++r) {
            e = cudaGraphLaunch(exec, g->stream);
            if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "flood batch: %s", cudaGetErrorString(e));
            queued += kFloodChunk;
            b->stats.kernel_launches += (int64_t)kFloodChunk * per_iter;
        }
        e = cudaMemcpyAsync(g->h_out, g->d_out, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "flood batch: %s", cudaGetErrorString(e));
        if (g->h_out[0] != 0) break;
        reps = std::min(reps * 2, 8);
    }
    return FBP_OK;
}

int collect(fbp_batch *b, Part &P, int32_t *iters_out, double *residual_out, int32_t *status_out, int *all_ok)
{
    const size_t m = P.members.size();
    std::vector<int32_t> done(m), iters(m);
    std::vector<unsigned> res(m);
    fbp_graph *g = P.g;
    cudaError_t e = cudaMemcpyAsync(done.data(), P.done, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(iters.data(), P.iters, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(res.data(), P.last_res, sizeof(unsigned) * m, cudaMemcpyDeviceToHost, g->stream);
    unsigned long long guards = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&guards, g->d_guards, sizeof guards, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "batch collect: %s", cudaGetErrorString(e));
    b->stats.guards += (int64_t)guards;
    const int halves = std::max<int>(1, (int)g->halves.size());
    for (size_t k = 0; k < m; ++k) {
        const int32_t i = P.members[k];
        float r;
        std::memcpy(&r, &res[k], sizeof r);
        const int st = done[k] == 1 ? FBP_OK : FBP_NOT_CONVERGED;
        if (st != FBP_OK) *all_ok = 0;
        if (iters_out) iters_out[i] = iters[k];
        if (residual_out) residual_out[i] = (double)r;
        if (status_out) status_out[i] = st;
        const int64_t e_k = (k + 1 < m ? P.edge_off[k + 1] : g->h.ne) - P.edge_off[k];
        b->stats.updates += (int64_t)iters[k] * e_k * (g->strategy == FBP_PARALL ? 1 : halves);
        b->stats.iters = std::max(b->stats.iters, iters[k]);
    }
    return FBP_OK;
}

// The member queue's launch shape: cluster size (16 on request, else 8) and
// clusters (requested, clamped to what can be resident; 0 = half of that
// when flooding members run beside the queue on the whole GPU, else all).
void queue_shape(fbp_batch *b, int cluster, int clusters)
{
    Part &Qp = b->parts[kQueue];
    if (!Qp.g) return;
    const int want = cluster == 16 ? 16 : 8;
    const int cl = batch_queue_clusters(want) > 0 ? want : 8;
    const int fit = batch_queue_clusters(cl);
    const bool beside = b->parts[kFlood].g != nullptr;
    const int n = clusters > 0 ? std::min(clusters, fit) : beside ? std::max(1, (fit + 1) / 2) : fit;
    if (cl != Qp.cluster || n != Qp.clusters) {
        Qp.cluster = cl;
        Qp.clusters = n;
        if (Qp.exec) cudaGraphExecDestroy(Qp.exec);
        Qp.exec = nullptr;
    }
}

}  // namespace

extern "C" int fbp_batch_create(int32_t n_graphs, const fbp_graph_desc *graphs, const fbp_allocator *alloc,
                                void *cuda_stream, fbp_batch **out)
{
    return fbp_batch_create_ex(n_graphs, graphs, alloc, cuda_stream, nullptr, out);
}

extern "C" int fbp_batch_create_ex(int32_t n_graphs, const fbp_graph_desc *graphs, const fbp_allocator *alloc,
                                   void *cuda_stream, const fbp_batch_config *config, fbp_batch **out)
{
    if (!out || n_graphs < 0 || (n_graphs > 0 && !graphs)) return fail(FBP_ERR_INVALID_ARG, "bad argument");
    *out = nullptr;
    for (int32_t i = 0; i < n_graphs; ++i) {
        const fbp_graph_desc &d = graphs[i];
        int rc = check_graph_args(d.n_vars, d.n_factors, d.factor_ptr, d.factor_vars, d.factor_type, d.factor_param,
                                  d.prior_p1, d.evidence);
        if (rc) {
            std::string msg = std::string("batch graph ") + std::to_string(i) + ": " + fbp_last_error();
            return fail(rc, "%s", msg.c_str());
        }
        if (d.schedule.strategy == FBP_RESIDUAL || d.schedule.strategy < 0 || d.schedule.strategy > FBP_CUSTOM_RANK)
            return fail(FBP_ERR_INVALID_ARG, "batch graph %d: strategy %d not supported in a batch", i,
                        d.schedule.strategy);
        if (d.max_iters < 0 || !(d.tol >= 0.0)) return fail(FBP_ERR_INVALID_ARG, "batch graph %d: bad max_iters/tol", i);
        for (int32_t a = 0; a < d.n_factors; ++a)
            if (d.factor_type[a] == FBP_TERMS)
                return fail(FBP_ERR_INVALID_ARG, "batch graph %d: generic (FBP_TERMS) factors are for single graphs", i);
    }
    if (config && ((config->one_launch != 0 && config->one_launch != 1) ||
                   (config->static_queue != 0 && config->static_queue != 1)))
        return fail(FBP_ERR_INVALID_ARG, "one_launch and static_queue must be 0 or 1");
    fbp_batch *b = new fbp_batch();
    b->n = n_graphs;
    b->stream = (cudaStream_t)cuda_stream;
    const bool can_queue = batch_queue_clusters(8) > 0;
    b->one_launch = config ? config->one_launch == 1 : false;
    const bool static_queue = !b->one_launch && (config ? config->static_queue == 1 : can_queue);
    b->part_of.resize(n_graphs);
    b->slot_of.resize(n_graphs);
    for (int32_t i = 0; i < n_graphs; ++i) {
        const int kind = kind_of(graphs[i].schedule.strategy);
        const int k = b->one_launch ? kQueue : (static_queue && kind != kFlood) ? kQueue : kind;
        b->part_of[i] = k;
        b->slot_of[i] = (int32_t)b->parts[k].members.size();
        b->parts[k].members.push_back(i);
        b->nv.push_back(graphs[i].n_vars);
        b->ne.push_back((int32_t)graphs[i].factor_ptr[graphs[i].n_factors]);
    }
    int rc = FBP_OK;
    bool first = true;
    for (int k = 0; k < kParts && !rc; ++k) {
        Part &P = b->parts[k];
        if (P.members.empty()) continue;
        if (first) {
            P.stream = b->stream;
            first = false;
        } else {
            cudaError_t e = cudaStreamCreateWithFlags(&P.stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) rc = fail(FBP_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
            P.own_stream = true;
        }
        if (!rc) rc = k == kQueue ? build_queue_part(b, graphs, alloc) : build_part(b, k, graphs, alloc);
    }
    cudaError_t e = cudaSuccess;
    if (!rc) queue_shape(b, 0, 0);
    if (!rc) e = cudaEventCreate(&b->ev0);
    if (!rc && e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    for (int k = 0; k < kParts && !rc && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&b->evp[k], cudaEventDisableTiming);
    if (!rc && e != cudaSuccess) rc = fail(FBP_ERR_CUDA, "events: %s", cudaGetErrorString(e));
    if (!rc) {
        size_t mx = 1;
        for (auto &P : b->parts)
            if (P.g) mx = std::max(mx, (size_t)std::max<int64_t>(P.g->h.nv, 2 * (int64_t)P.g->h.ne));
        e = cudaMalloc(&b->scratch, mx * sizeof(float));
        if (e != cudaSuccess) rc = fail(FBP_ERR_OOM, "batch scratch: %s", cudaGetErrorString(e));
        b->scratch_n = mx;
    }
    if (rc) {
        std::string keep = fbp_last_error();
        fbp_batch_destroy(b);
        return fail(rc, "%s", keep.c_str());
    }
    *out = b;
    return FBP_OK;
}

extern "C" int fbp_batch_run(fbp_batch *b, int32_t *iters_out, double *residual_out, int32_t *status_out)
{
    if (!b) return fail(FBP_ERR_INVALID_ARG, "NULL batch");
    b->stats = fbp_stats{};
    cudaError_t e = cudaEventRecord(b->ev0, b->stream);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "%s", cudaGetErrorString(e));
    // side streams start after ev0
    for (auto &P : b->parts)
        if (P.g && P.stream != b->stream) cudaStreamWaitEvent(P.stream, b->ev0, 0);
    int rc = FBP_OK;
    if (b->parts[kQueue].g) rc = run_queue(b, b->parts[kQueue]);
    for (int k : {kStatic1, kStatic2})
        if (b->parts[k].g && !rc) rc = launch_static(b, b->parts[k]);
    if (!rc && b->parts[kFlood].g) rc = run_flood(b, b->parts[kFlood]);
    if (rc) return rc;
    for (int k : {kStatic1, kStatic2}) {
        Part &P = b->parts[k];
        if (!P.g || P.max_iters <= 0) continue;
        rc = engine_check(P.g);
        if (rc) return rc;
        const int32_t it = P.g->h_out[0];
        P.g->cur ^= (it * (int)P.g->halves.size()) & 1;
    }
    for (int k = 0; k < kParts; ++k) {
        Part &P = b->parts[k];
        if (P.g && P.stream != b->stream) {
            cudaEventRecord(b->evp[k], P.stream);
            cudaStreamWaitEvent(b->stream, b->evp[k], 0);
        }
    }
    e = cudaEventRecord(b->ev1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b->ev1);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "%s", cudaGetErrorString(e));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->ev0, b->ev1);
    b->stats.run_ms = ms;
    int all_ok = 1;
    for (int k = 0; k < kParts; ++k) {
        Part &P = b->parts[k];
        if (!P.g) continue;
        rc = k == kQueue ? collect_queue(b, P, iters_out, residual_out, status_out, &all_ok)
                         : collect(b, P, iters_out, residual_out, status_out, &all_ok);
        if (rc) return rc;
    }
    return all_ok ? FBP_OK : FBP_NOT_CONVERGED;
}

extern "C" int fbp_batch_marginals(const fbp_batch *b, int32_t graph, float *out_p1, int out_is_device)
{
    if (!b || graph < 0 || graph >= b->n) return fail(FBP_ERR_INVALID_ARG, "bad graph index");
    const Part &P = b->parts[b->part_of[graph]];
    const int32_t k = b->slot_of[graph];
    if (b->nv[graph] == 0) return FBP_OK;
    if (!out_p1) return fail(FBP_ERR_INVALID_ARG, "NULL output");
    int rc = fbp_marginals(P.g, b->scratch, 1);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(out_p1, b->scratch + P.var_off[k], sizeof(float) * b->nv[graph],
                                    out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, P.g->stream);
    if (e == cudaSuccess && !out_is_device) e = cudaStreamSynchronize(P.g->stream);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "%s", cudaGetErrorString(e));
    return FBP_OK;
}

extern "C" int fbp_batch_messages_export(const fbp_batch *b, int32_t graph, float *a2v)
{
    if (!b || graph < 0 || graph >= b->n) return fail(FBP_ERR_INVALID_ARG, "bad graph index");
    const Part &P = b->parts[b->part_of[graph]];
    const int32_t k = b->slot_of[graph];
    if (b->ne[graph] == 0) return FBP_OK;
    if (!a2v) return fail(FBP_ERR_INVALID_ARG, "NULL output");
    fbp_graph *g = P.g;
    launch_decode_pairs(g->a2v[g->cur] + P.edge_off[k], b->scratch, b->ne[graph], g->stream);
    cudaError_t e = cudaMemcpyAsync(a2v, b->scratch, sizeof(float) * 2 * b->ne[graph], cudaMemcpyDeviceToHost,
                                    g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return fail(FBP_ERR_CUDA, "%s", cudaGetErrorString(e));
    return FBP_OK;
}

extern "C" int fbp_batch_reset(fbp_batch *b)
{
    if (!b) return fail(FBP_ERR_INVALID_ARG, "NULL batch");
    for (auto &P : b->parts) {
        if (!P.g) continue;
        int rc = fbp_messages_reset(P.g);
        if (rc) return rc;
    }
    return FBP_OK;
}

extern "C" int fbp_batch_set_tuning(fbp_batch *b, const fbp_batch_tuning *t)
{
    if (!b) return fail(FBP_ERR_INVALID_ARG, "NULL batch");
    const fbp_batch_tuning v = t ? *t : fbp_batch_tuning{0, 0, 0, 0, -1, -1, 0};
    if (v.engine_grid < 0 || v.queue_clusters < 0 ||
        (v.engine_cluster != 0 && v.engine_cluster != 1 && v.engine_cluster != 8 && v.engine_cluster != 16))
        return fail(FBP_ERR_INVALID_ARG, "bad tuning");
    b->tuning = v;
    queue_shape(b, v.engine_cluster, v.queue_clusters);
    if (b->one_launch) return FBP_OK;
    for (int k : {kStatic1, kStatic2}) {
        Part &S = b->parts[k];
        if (!S.g) continue;
        int rc = fbp_set_option(S.g, FBP_OPT_ENGINE_FUSE_LANES, v.engine_fuse_lanes >= 0 ? v.engine_fuse_lanes : 0);
        if (!rc) rc = fbp_set_option(S.g, FBP_OPT_ENGINE_SOLO_LANES, v.engine_solo_lanes >= 0 ? v.engine_solo_lanes : 128);
        if (rc) return rc;
    }
    Part &F = b->parts[kFlood];
    if (F.g) {
        int rc = fbp_set_option(F.g, FBP_OPT_FLOOD_HUB_MIN, v.flood_hub_min ? v.flood_hub_min : kFloodMediumMax);
        if (!rc) rc = fbp_set_option(F.g, FBP_OPT_FLOOD_CHUNK, v.flood_chunk ? v.flood_chunk : kFloodHubChunk);
        if (rc) return rc;
        if (!F.g->flood_ready && (rc = build_flood_plan(F.g))) return rc;
    }
    b->tuning = v;
    return FBP_OK;
}

extern "C" int fbp_batch_one_launch(const fbp_batch *b) { return b ? (b->one_launch ? 1 : 0) : -1; }

extern "C" int fbp_batch_get_stats(const fbp_batch *b, fbp_stats *out)
{
    if (!b || !out) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    *out = b->stats;
    return FBP_OK;
}

extern "C" void fbp_batch_destroy(fbp_batch *b)
{
    if (!b) return;
    for (auto &P : b->parts) {
        if (P.exec) cudaGraphExecDestroy(P.exec);
        if (P.g) fbp_graph_destroy(P.g);
        if (P.own_stream && P.stream) cudaStreamDestroy(P.stream);
    }
    if (b->scratch) cudaFree(b->scratch);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    for (auto &ev : b->evp)
        if (ev) cudaEventDestroy(ev);
    delete b;
}
