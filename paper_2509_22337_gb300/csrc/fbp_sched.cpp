// Graph layout and dependency analysis on the host.
#include "fbp_sched.h"

#include <algorithm>
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
            int64_t mx = 0;
            for (int64_t r : rank) mx = std::max(mx, r);
            for (int64_t &r : rank) r = mx - r;
        }
        return FBP_OK;
    }
    default:
        return fail(FBP_ERR_INVALID_ARG, "unknown strategy %d", spec.strategy);
    }
}

// Algorithm 2 with per-variable counters instead of the scan over NextSet.
// The cut test for e_i = (a, v) asks whether NextSet holds an edge
// (a*, v*) with v* in N(a) \ v, a* != a and rank < rank(e_i) (Definition 1).
// NextSet only holds edges of rank <= rank(e_i) (canonical order), so per
// variable v* it suffices to know how many NextSet edges end at v* in total
// and how many of those belong to the current class; the one edge (a, v*) of
// factor a itself is discounted.  Counters are reset lazily by stamps (the
// level index, and a class id that also changes at every cut).
void dependency_levels(const HostCSR &h, const int64_t *rank, const int32_t *edges, int64_t n,
                       std::vector<int64_t> &lp, std::vector<int32_t> &le)
{
    le.resize(n);
    if (edges) std::copy(edges, edges + n, le.begin());
    else std::iota(le.begin(), le.end(), 0);
    std::sort(le.begin(), le.end(), [rank](int32_t x, int32_t y) {
        return rank[x] != rank[y] ? rank[x] < rank[y] : x < y;
    });
    lp.assign(1, 0);
    if (n == 0) return;
    std::vector<int32_t> cnt_all(h.nv, 0), cnt_cls(h.nv, 0);
    std::vector<int64_t> st_all(h.nv, -1), st_cls(h.nv, -1);
    std::vector<int64_t> elev(h.ne, -1);
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
            int64_t earlier = (st_all[vs] == level ? cnt_all[vs] : 0) - (st_cls[vs] == cls ? cnt_cls[vs] : 0);
            if (elev[q] == level && rank[q] < r) --earlier;
            cut = earlier > 0;
        }
        if (cut) {
            lp.push_back(i);
            ++level;
            ++cls;
        }
        elev[e] = level;
        if (st_all[v] != level) { st_all[v] = level; cnt_all[v] = 0; }
        ++cnt_all[v];
        if (st_cls[v] != cls) { st_cls[v] = cls; cnt_cls[v] = 0; }
        ++cnt_cls[v];
    }
    lp.push_back(n);
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
