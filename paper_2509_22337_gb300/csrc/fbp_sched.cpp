// Graph layout and dependency analysis on the host.
#include "fbp_sched.h"

#include <algorithm>
#include <cstring>
#include <limits>
#include <numeric>

namespace fbp {

void build_host_csr(int32_t nv, int32_t na, const int64_t *fptr, const int32_t *fvars,
                    const uint8_t *ftype, const float *fparam, HostCSR &h)
{
    h.nv = nv;
    h.na = na;
    h.ne = (int32_t)fptr[na];
    h.fptr.assign(fptr, fptr + na + 1);
    h.fvars.assign(fvars, fvars + h.ne);
    h.ftype.assign(ftype, ftype + na);
    h.fparam.assign(fparam, fparam + na);
    h.efac.resize(h.ne);
    h.vptr.assign((size_t)nv + 1, 0);
    for (int32_t a = 0; a < na; ++a)
        for (int64_t e = fptr[a]; e < fptr[a + 1]; ++e) {
            h.efac[e] = a;
            h.vptr[fvars[e] + 1]++;
        }
    for (int32_t v = 0; v < nv; ++v) h.vptr[v + 1] += h.vptr[v];
    h.vedge.resize(h.ne);
    std::vector<int32_t> fill(h.vptr.begin(), h.vptr.end() - 1);
    for (int32_t e = 0; e < h.ne; ++e) h.vedge[fill[fvars[e]]++] = e;  // ascending edge id per row
}

// TOPO: depth of every variable over the "premise -> output" relation of the
// factors (a variable without a defining factor has depth 0; a factor with no
// premises defines depth 0).  Returns false on a cycle.
static bool variable_depths(const HostCSR &h, std::vector<int64_t> &depth)
{
    std::vector<int32_t> pending(h.nv, 0);     // premises of defining factors still unresolved
    std::vector<int32_t> uptr(h.nv + 1, 0);     // factors in which a variable is a premise
    for (int32_t a = 0; a < h.na; ++a) {
        const int64_t lo = h.fptr[a], hi = h.fptr[a + 1];
        if (hi <= lo) continue;
        pending[h.fvars[hi - 1]] += (int32_t)(hi - 1 - lo);
        for (int64_t e = lo; e < hi - 1; ++e) uptr[h.fvars[e] + 1]++;
    }
    for (int32_t v = 0; v < h.nv; ++v) uptr[v + 1] += uptr[v];
    std::vector<int32_t> uses(uptr[h.nv]);
    std::vector<int32_t> pos(uptr.begin(), uptr.end() - 1);
    for (int32_t a = 0; a < h.na; ++a)
        for (int64_t e = h.fptr[a]; e + 1 < h.fptr[a + 1]; ++e) uses[pos[h.fvars[e]]++] = a;
    depth.assign(h.nv, 0);
    std::vector<int32_t> ready;
    ready.reserve(h.nv);
    for (int32_t v = 0; v < h.nv; ++v)
        if (pending[v] == 0) ready.push_back(v);
    for (size_t r = 0; r < ready.size(); ++r) {
        const int32_t u = ready[r];
        for (int32_t k = uptr[u]; k < uptr[u + 1]; ++k) {
            const int32_t a = uses[k];
            const int32_t y = h.fvars[h.fptr[a + 1] - 1];
            depth[y] = std::max(depth[y], depth[u] + 1);
            if (--pending[y] == 0) ready.push_back(y);
        }
    }
    return (int32_t)ready.size() == h.nv;
}

void backward_ranks(const std::vector<int64_t> &fwd, std::vector<int64_t> &bwd)
{
    int64_t mx = 0;
    for (int64_t r : fwd) mx = std::max(mx, r);
    bwd.resize(fwd.size());
    for (size_t e = 0; e < fwd.size(); ++e) bwd[e] = mx - fwd[e];
}

int build_ranks(const HostCSR &h, const fbp_schedule_spec &spec, int half, std::vector<int64_t> &rank)
{
    rank.assign(h.ne, 0);
    switch (spec.strategy) {
    case FBP_PARALL:
        return FBP_OK;
    case FBP_SEQFIX:
        for (int32_t e = 0; e < h.ne; ++e) rank[e] = spec.edge_rank ? spec.edge_rank[e] : e;
        return FBP_OK;
    case FBP_CUSTOM_RANK:
        if (!spec.edge_rank) return fail(FBP_ERR_INVALID_ARG, "CUSTOM_RANK needs edge_rank");
        for (int32_t e = 0; e < h.ne; ++e) rank[e] = spec.edge_rank[e];
        return FBP_OK;
    case FBP_TOPO:
    case FBP_TOPO_FB: {
        if (spec.factor_rank) {
            for (int32_t e = 0; e < h.ne; ++e) rank[e] = spec.factor_rank[h.efac[e]];
        } else {
            std::vector<int64_t> depth;
            if (!variable_depths(h, depth))
                return fail(FBP_ERR_SCHEDULE, "TOPO: the premise->output relation has a cycle");
            for (int32_t a = 0; a < h.na; ++a) {
                const int64_t lo = h.fptr[a], hi = h.fptr[a + 1];
                for (int64_t e = lo; e < hi; ++e) rank[e] = depth[h.fvars[hi - 1]];
            }
        }
        if (half == 1) {
            std::vector<int64_t> fwd = std::move(rank);
            backward_ranks(fwd, rank);
        }
        return FBP_OK;
    }
    default:
        return fail(FBP_ERR_INVALID_ARG, "unknown strategy %d", spec.strategy);
    }
}

// Canonical order (Definition 2): edges by (rank, edge id).  `edges` (NULL =
// all edges) lists edge ids in ascending order.  Ranks spanning a range no
// wider than a few times the edge count (every strategy's but a sparse
// custom one) are placed by a stable counting sort, which keeps the ascending
// id order inside each rank; others by a comparison sort of (rank, id) pairs.
static void canonical_order(const int64_t *rank, const int32_t *edges, int64_t n, std::vector<int32_t> &le)
{
    le.resize(n);
    if (n == 0) return;
    auto id = [edges](int64_t i) { return edges ? edges[i] : (int32_t)i; };
    int64_t lo = rank[id(0)], hi = lo;
    for (int64_t i = 1; i < n; ++i) {
        const int64_t r = rank[id(i)];
        lo = std::min(lo, r);
        hi = std::max(hi, r);
    }
    const uint64_t span = (uint64_t)hi - (uint64_t)lo;  // exact for hi >= lo
    if (span <= (uint64_t)(4 * n + 1024)) {
        std::vector<int64_t> start(span + 2, 0);
        for (int64_t i = 0; i < n; ++i) ++start[(uint64_t)rank[id(i)] - (uint64_t)lo + 1];
        for (uint64_t k = 1; k < span + 2; ++k) start[k] += start[k - 1];
        for (int64_t i = 0; i < n; ++i) {
            const int32_t e = id(i);
            le[start[(uint64_t)rank[e] - (uint64_t)lo]++] = e;
        }
        return;
    }
    struct Key {
        int64_t r;
        int32_t e;
    };
    std::vector<Key> keys(n);
    for (int64_t i = 0; i < n; ++i) keys[i] = Key{rank[id(i)], id(i)};
    std::sort(keys.begin(), keys.end(), [](const Key &x, const Key &y) { return x.r != y.r ? x.r < y.r : x.e < y.e; });
    for (int64_t i = 0; i < n; ++i) le[i] = keys[i].e;
}

// Algorithm 2 with per-variable counters instead of the scan over NextSet.
// The cut test for e_i = (a, v) asks whether NextSet holds an edge
// (a*, v*) with v* in N(a) \ v, a* != a and rank < rank(e_i) (Definition 1).
// NextSet only holds edges of rank <= rank(e_i) (canonical order), so per
// variable v* it suffices to know how many NextSet edges end at v* in total
// and how many of those belong to the current class; the one edge (a, v*) of
// factor a itself is discounted.  Counters are reset lazily by stamps (the
// level index, and a class id that also changes at every cut).  With a single
// class nothing can cut, and the edges form one level.
void dependency_levels(const HostCSR &h, const int64_t *rank, const int32_t *edges, int64_t n,
                       std::vector<int64_t> &lp, std::vector<int32_t> &le)
{
    canonical_order(rank, edges, n, le);
    lp.assign(1, 0);
    if (n == 0) return;
    if (rank[le[0]] == rank[le[n - 1]]) {
        lp.push_back(n);
        return;
    }
    struct VarCount {           // one cache line holds a variable's counters
        int64_t st_all = -1;    // level of cnt_all
        int64_t st_cls = -1;    // class of cnt_cls
        int32_t cnt_all = 0;    // NextSet edges into the variable
        int32_t cnt_cls = 0;    // ... of the current class
    };
    std::vector<VarCount> vc(h.nv);
    std::vector<int32_t> elev(h.ne, -1);
    int64_t level = 0, cls = 0;
    int64_t cls_rank = rank[le[0]];
    for (int64_t i = 0; i < n; ++i) {
        const int32_t e = le[i];
        const int64_t r = rank[e];
        if (r != cls_rank) {
            cls_rank = r;
            ++cls;
        }
        const int32_t a = h.efac[e], v = h.fvars[e];
        bool cut = false;
        for (int64_t q = h.fptr[a]; q < h.fptr[a + 1] && !cut; ++q) {
            const int32_t vs = h.fvars[q];
            if (vs == v) continue;
            const VarCount &c = vc[vs];
            int64_t earlier = (c.st_all == level ? c.cnt_all : 0) - (c.st_cls == cls ? c.cnt_cls : 0);
            if (elev[q] == level && rank[q] < r) --earlier;
            cut = earlier > 0;
        }
        if (cut) {
            lp.push_back(i);
            ++level;
            ++cls;
        }
        elev[e] = (int32_t)level;
        VarCount &c = vc[v];
        if (c.st_all != level) { c.st_all = level; c.cnt_all = 0; }
        ++c.cnt_all;
        if (c.st_cls != cls) { c.st_cls = cls; c.cnt_cls = 0; }
        ++c.cnt_cls;
    }
    lp.push_back(n);
}

static inline int4 i4(int32_t x, int32_t y, int32_t z, int32_t w)
{
    int4 r;
    r.x = x; r.y = y; r.z = z; r.w = w;
    return r;
}

static inline int2 i2(int32_t x, int32_t y)
{
    int2 r;
    r.x = x; r.y = y;
    return r;
}

void pack_levels(const HostCSR &h, const std::vector<int32_t> &fac_graph, const std::vector<int64_t> &lp,
                 const std::vector<int32_t> &le, int max_fan, LevelPack &P)
{
    const int32_t nl = (int32_t)lp.size() - 1;
    P = LevelPack{};
    P.lane_ptr.assign(1, 0);
    P.big_ptr.assign(1, 0);
    P.lanes.reserve((size_t)h.ne + (size_t)h.ne / 4 + 32 * (size_t)std::max(nl, 0));
    P.lrow.reserve(P.lanes.capacity());
    std::vector<int32_t> elev(h.ne, std::numeric_limits<int32_t>::max());
    std::vector<int32_t> stamp(h.na, -1);
    std::vector<uint32_t> fmask(h.na, 0);
    std::vector<int32_t> order;
    auto pad = [&P] {
        while (P.lanes.size() % 32) {
            P.lanes.push_back(i4(-1, 0, 0, 0));
            P.lrow.push_back(i2(0, 0));
        }
    };
    for (int32_t L = 0; L < nl; ++L) {
        order.clear();
        for (int64_t i = lp[L]; i < lp[L + 1]; ++i) {
            const int32_t e = le.empty() ? (int32_t)i : le[i];
            elev[e] = L;
            const int32_t a = h.efac[e];
            const int32_t lo = (int32_t)h.fptr[a], n = (int32_t)(h.fptr[a + 1] - h.fptr[a]);
            if (n > max_fan) {
                P.big.push_back(e);
                continue;
            }
            if (stamp[a] != L) {
                stamp[a] = L;
                fmask[a] = 0;
                order.push_back(a);
            }
            fmask[a] |= 1u << (e - lo);
        }
        const size_t base = P.lanes.size();
        int used = 32;  // lanes used in the current warp
        for (int32_t a : order) {
            const int32_t lo = (int32_t)h.fptr[a], n = (int32_t)(h.fptr[a + 1] - h.fptr[a]);
            if (used + n > 32) {
                pad();
                used = 0;
            }
            int32_t pb;
            std::memcpy(&pb, &h.fparam[a], sizeof pb);
            const int32_t member = fac_graph.empty() ? 0 : fac_graph[a];
            const int32_t common = (n << 5) | ((int32_t)h.ftype[a] << 11) | (member << 15);
            for (int32_t j = 0; j < n; ++j) {
                const int32_t pk = used | common | ((int32_t)((fmask[a] >> j) & 1u) << 14);
                const int32_t v = h.fvars[lo + j];
                P.lanes.push_back(i4(lo + j, pk, pb, v));
                P.lrow.push_back(i2(h.vptr[v], h.vptr[v + 1]));
            }
            used += n;
        }
        pad();
        P.max_lanes = std::max(P.max_lanes, (int32_t)(P.lanes.size() - base));
        P.lane_ptr.push_back((int32_t)P.lanes.size());
        P.big_ptr.push_back((int32_t)P.big.size());
    }
    P.vel.resize(h.ne);
    for (int32_t k = 0; k < h.ne; ++k) P.vel[k] = i2(h.vedge[k], elev[h.vedge[k]]);
}

int64_t residual_classes(const HostCSR &h, const float *dres, double tol, int64_t *rank,
                         std::vector<int32_t> &act)
{
    std::vector<float> vres(h.nv, 0.f);
    for (int32_t e = 0; e < h.ne; ++e) {
        const int32_t v = h.fvars[e];
        vres[v] = std::max(vres[v], dres[e]);
    }
    act.clear();
    for (int32_t a = 0; a < h.na; ++a) {
        float rho = 0.f;
        for (int64_t q = h.fptr[a]; q < h.fptr[a + 1]; ++q) rho = std::max(rho, vres[h.fvars[q]]);
        const double r = rho;
        const int64_t c = r >= 1e-2 ? 0 : r >= 1e-4 ? 1 : r >= tol ? 2 : -1;
        for (int64_t q = h.fptr[a]; q < h.fptr[a + 1]; ++q) {
            rank[q] = c;
            if (c >= 0) act.push_back((int32_t)q);
        }
    }
    return (int64_t)act.size();
}

}  // namespace fbp
