// Host side of the belief-propagation library: the C ABI of include/fbp.h,
// graph ingest and layout (Sec. 4.1 "Initialization", Sec. 4.3.2), update
// strategy -> ranks (Table 1, Definition 2), the dependency analysis of
// Algorithm 2 (Sec. 4.2.3) and the iteration driver (Sec. 4.1 "Kernel
// Launch" / "Message Passing").
#include "fbp.h"
#include "fbp_internal.h"
#include "fbp_flood.h"
#include "fbp_sched.h"
#include "fbp_graph_impl.h"

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

using namespace fbp;

namespace {
thread_local std::string t_err;
}  // namespace

void fbp::clear_error() { t_err.clear(); }

int fbp::fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

namespace {

#define CUDA_TRY(call)                                                                       \
    do {                                                                                     \
        cudaError_t _e = (call);                                                             \
        if (_e != cudaSuccess)                                                               \
            return fail(FBP_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(_e));       \
    } while (0)

// rho encoding of a normalised pair computed in double, rounded once.
float enc_host(double m0, double m1)
{
    if (!(m0 + m1 > 0.0)) return 1.0f;
    if (m1 >= m0) return (float)(m0 / m1);
    float r = (float)(m1 / m0);
    return -r;  // -0.0f for the hard message (1, 0)
}

float phi_of(float prior, int8_t ev)
{
    if (ev == 0) return -0.0f;
    if (ev == 1) return 0.0f;
    if (!std::isnan(prior)) return enc_host(1.0 - (double)prior, (double)prior);
    return 1.0f;
}

}  // namespace

// ---------------------------------------------------------------------------
// graph handle
// ---------------------------------------------------------------------------
namespace fbp {

int dalloc(fbp_graph *g, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    if (g->has_alloc) {
        *p = g->alloc.alloc(bytes, g->alloc.ctx);
        if (!*p) return fail(FBP_ERR_OOM, "allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return fail(FBP_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    g->owned.push_back(*p);
    return FBP_OK;
}

void dfree(fbp_graph *g, void *p)
{
    if (!p) return;
    auto it = std::find(g->owned.begin(), g->owned.end(), p);
    if (it != g->owned.end()) g->owned.erase(it);
    if (g->has_alloc) g->alloc.free(p, g->alloc.ctx);
    else cudaFree(p);
}

void free_levels_one(fbp_graph *g, LevelSet &ls)
{
    dfree(g, ls.d_lanes);
    dfree(g, ls.d_lrow);
    ls.d_lrow = nullptr;
    dfree(g, ls.d_lane_ptr);
    dfree(g, ls.d_big);
    dfree(g, ls.d_big_ptr);
    dfree(g, ls.d_vel);
    ls.d_lanes = nullptr;
    ls.d_lane_ptr = ls.d_big = ls.d_big_ptr = nullptr;
    ls.d_vel = nullptr;
}

void free_levels(fbp_graph *g)
{
    for (auto &ls : g->halves) free_levels_one(g, ls);
    g->halves.clear();
    free_seq(g);  // built from these level lists
}

// Engine plan of one level list.  Per level, the factors the level touches
// (in order of first appearance) are packed into warps of 32 lanes, one lane
// per variable of the factor and every factor inside a single warp; each lane
// record is {edge, first lane of its factor | n << 5 | type << 11 | in-level
// bit << 14, p bits, variable}, with the variable's row range beside it in
// lrow; idle lanes have edge -1.  Factors wider than a warp
// go to a per-edge list.  vel[k] pairs the k-th var-major edge with its level
// (INT_MAX if the edge is in no level: inactive under the residual strategy).
int upload_erow(fbp_graph *g);

int upload_levels(fbp_graph *g, LevelSet &ls, const LevelPack *packed)
{
    // the engine's per-edge row records, built with the first level plan (a
    // graph that only floods never needs them)
    if (!g->erow && g->h.ne > 0) {
        int rc = upload_erow(g);
        if (rc) return rc;
    }
    LevelPack local;
    if (!packed) {
        pack_levels(g->h, g->fac_graph, ls.lp, ls.le, engine_max_fan(), local);
        packed = &local;
    }
    const LevelPack &P = *packed;
    free_levels_one(g, ls);
    int rc = upload(g, &ls.d_lanes, P.lanes.data(), P.lanes.size());
    if (!rc) rc = upload(g, &ls.d_lrow, P.lrow.data(), P.lrow.size());
    if (!rc) rc = upload(g, &ls.d_lane_ptr, P.lane_ptr.data(), P.lane_ptr.size());
    if (!rc) rc = upload(g, &ls.d_big, P.big.data(), P.big.size());
    if (!rc) rc = upload(g, &ls.d_big_ptr, P.big_ptr.data(), P.big_ptr.size());
    if (!rc) rc = upload(g, &ls.d_vel, P.vel.data(), P.vel.size());
    ls.max_lanes = P.max_lanes;
    ls.n_lanes = (int64_t)P.lanes.size();
    return rc;
}

// Row record of each edge's variable: {vptr[v], vptr[v+1], v, 0}.
int upload_erow(fbp_graph *g)
{
    const HostCSR &h = g->h;
    std::vector<int4> er(h.ne);
    parallel_for(h.ne, host_threads(), 1 << 16, [&](int64_t b, int64_t e) {
        for (int64_t q = b; q < e; ++q) {
            const int32_t v = h.fvars[q];
            er[q] = make_int4(h.vptr[v], h.vptr[v + 1], v, 0);
        }
    });
    return upload(g, &g->erow, er.data(), er.size());
}

// Flooding plan: variables by degree class (every row of degree <= 8 one
// thread, longer rows in sub-chunks combined by one thread or one warp), the
// slot of every edge in the variable-major message copy, and phase 2's warps
// of whole factors.  With `ranges` (a batch run in one launch), lists are
// built only over the given {first variable, end variable, first factor, end
// factor} ranges, range after range, and each range's slices of the lists are
// returned in `slices` (one MemberDev per range, flooding fields filled);
// warps never cross a range boundary.
int build_flood_plan(fbp_graph *g, const std::vector<int4> *ranges, std::vector<MemberDev> *slices)
{
    const HostCSR &h = g->h;
    flood_exec_drop(g);
    free_seq(g);  // indexes this plan's lists
    if (g->flood_ready) {  // a rebuild after retuning
        dfree(g, (void *)g->flood.subs);
        dfree(g, (void *)g->flood.medium);
        dfree(g, (void *)g->flood.hub_row);
        dfree(g, (void *)g->flood.agg);
        dfree(g, (void *)g->flood.belief);
        dfree(g, (void *)g->flood.warps);
        dfree(g, (void *)g->flood.twarps);
        dfree(g, (void *)g->flood.wide);
        dfree(g, (void *)g->flood.wide_v2a);
        dfree(g, (void *)g->flood.vpos);
        g->flood = FloodPlanDev{};
        g->flood_ready = false;
    }
    FloodPlanDev F;
    std::vector<int4> subs, medium, hub_row;
    std::vector<int4> twarps, warps;
    std::vector<int32_t> wide;
    int32_t n_agg = 0;  // sub-chunk products of rows of several sub-chunks
    std::vector<int4> whole;
    if (!ranges) whole.push_back(make_int4(0, h.nv, 0, h.na));
    const std::vector<int4> &R = ranges ? *ranges : whole;
    if (slices) slices->assign(R.size(), MemberDev{});
    for (size_t r = 0; r < R.size(); ++r) {
        const int4 rg = R[r];
        const size_t sub0 = subs.size(), med0 = medium.size(), hub0 = hub_row.size();
        for (int32_t v = rg.x; v < rg.y; ++v) {
            const int32_t lo = h.vptr[v], hi = h.vptr[v + 1], d = hi - lo;
            if (d <= kFloodSmallMax) continue;  // the one-thread rows
            const int32_t ns = (d + kFloodSub - 1) / kFloodSub;
            for (int32_t c = 0; c < ns; ++c)
                subs.push_back(
                    make_int4(v, lo + c * kFloodSub, std::min(hi, lo + (c + 1) * kFloodSub), ns == 1 ? -1 : n_agg + c));
            if (ns == 1) continue;
            (d <= g->flood_hub_min ? medium : hub_row).push_back(make_int4(v, n_agg, ns, 0));
            n_agg += ns;
        }
        // rows of one sub-chunk count side by side: the combines of a warp then
        // run the same branches (each row is independent: same results)
        std::stable_sort(medium.begin() + med0, medium.end(), [](const int4 &a, const int4 &b) { return a.z < b.z; });
        // phase 2: runs of consecutive typed factors of at most 32 variables
        // are packed whole into warps of at most 32 edges (twarps), runs of
        // consecutive generic factors likewise (warps); a factor wider than a
        // warp goes edge by edge to the wide list
        const size_t tw0 = twarps.size(), wide0 = wide.size();
        int32_t t0 = rg.z, w0 = rg.z;  // open typed / generic warp: first factor
        auto close_t = [&](int32_t a1) {
            if (a1 > t0) twarps.push_back(make_int4((int)h.fptr[t0], (int)h.fptr[a1], t0, a1));
            t0 = a1;
        };
        auto close_w = [&](int32_t a1) {
            if (a1 > w0) warps.push_back(make_int4((int)h.fptr[w0], (int)h.fptr[a1], w0, a1));
            w0 = a1;
        };
        for (int32_t a = rg.z; a < rg.w; ++a) {
            const int64_t n = h.fptr[a + 1] - h.fptr[a];
            if (n > 32) {
                close_t(a);
                close_w(a);
                for (int64_t e = h.fptr[a]; e < h.fptr[a + 1]; ++e) wide.push_back((int32_t)e);
                t0 = w0 = a + 1;
                continue;
            }
            if (h.ftype[a] == FBP_TERMS) {
                close_t(a);
                if (h.fptr[a + 1] - h.fptr[w0] > 32) close_w(a);
                t0 = a + 1;
            } else {
                close_w(a);
                if (h.fptr[a + 1] - h.fptr[t0] > 32) close_t(a);
                w0 = a + 1;
            }
        }
        close_t(rg.w);
        close_w(rg.w);
        if (slices) {
            MemberDev &M = (*slices)[r];
            M.v0 = rg.x;
            M.v1 = rg.y;
            M.sub0 = (int32_t)sub0;
            M.sub1 = (int32_t)subs.size();
            M.med0 = (int32_t)med0;
            M.med1 = (int32_t)medium.size();
            M.hub0 = (int32_t)hub0;
            M.hub1 = (int32_t)hub_row.size();
            M.tw0 = (int32_t)tw0;
            M.tw1 = (int32_t)twarps.size();
            M.wide0 = (int32_t)wide0;
            M.wide1 = (int32_t)wide.size();
        }
    }
    // slot of each edge in the variable-major copy: the inverse of vedge
    std::vector<int32_t> vpos(h.ne);
    parallel_for(h.ne, host_threads_all(), 1 << 16, [&](int64_t b, int64_t e) {
        for (int64_t k = b; k < e; ++k) vpos[h.vedge[k]] = (int32_t)k;
    });
    // the short rows' blocks: one resident grid (8 blocks of 256 per SM)
    // whose threads step through the variables
    F.nb_vars = (int32_t)std::min<int64_t>((h.nv + 255) / 256, 8 * (int64_t)num_sms());
    F.n_subs = (int32_t)subs.size();
    F.sub_threads = std::max(32, std::min(256, g->flood_chunk / kFloodSub));
    F.n_medium = (int32_t)medium.size();
    F.nb_medium = (F.n_medium + kFloodSlots - 1) / kFloodSlots;
    F.n_hub_rows = (int32_t)hub_row.size();
    int32_t *d_vpos = nullptr;
    int4 *d_subs = nullptr, *d_medium = nullptr, *d_hub_row = nullptr;
    XP *d_agg = nullptr;
    uint2 *d_belief = nullptr;
    int rc = upload(g, &d_subs, subs.data(), subs.size());
    if (!rc) rc = upload(g, &d_medium, medium.data(), medium.size());
    if (!rc) rc = upload(g, &d_hub_row, hub_row.data(), hub_row.size());
    if (!rc) rc = dalloc_n(g, &d_agg, std::max<size_t>(n_agg, 1));
    if (!rc) rc = dalloc_n(g, &d_belief, std::max<size_t>(h.nv, 1));
    if (!rc) rc = upload(g, &d_vpos, vpos.data(), vpos.size());
    if (rc) return rc;
    F.subs = d_subs;
    F.medium = d_medium;
    F.hub_row = d_hub_row;
    F.agg = d_agg;
    F.belief = d_belief;
    F.vpos = d_vpos;
    int4 *d_warps = nullptr, *d_twarps = nullptr;
    int32_t *d_wide = nullptr;
    float *d_wide_v2a = nullptr;
    if ((rc = upload(g, &d_twarps, twarps.data(), twarps.size())) ||
        (rc = upload(g, &d_warps, warps.data(), warps.size())) || (rc = upload(g, &d_wide, wide.data(), wide.size())) ||
        (rc = dalloc_n(g, &d_wide_v2a, std::max<size_t>(wide.size(), 1))))
        return rc;
    F.n_twarps = (int32_t)twarps.size();
    F.twarps = d_twarps;
    F.n_warps = (int32_t)warps.size();
    F.warps = d_warps;
    F.n_wide = (int32_t)wide.size();
    F.wide = d_wide;
    F.wide_v2a = d_wide_v2a;
    g->flood = F;
    g->flood_subs_h = std::move(subs);
    g->flood_medium_h = std::move(medium);
    g->flood_hub_h = std::move(hub_row);
    g->flood_ready = true;
    return FBP_OK;
}

// One factor's row and type: variables in range and distinct, arity valid for
// the type, parameter in [0, 1] where the type has one.  With report set, the
// first problem in row order becomes the thread's error message.
static int check_factor(int32_t nv, const int64_t *fptr, const int32_t *fvars, const uint8_t *ftype,
                        const float *fparam, int32_t a, bool report)
{
    const int64_t lo = fptr[a], n = fptr[a + 1] - lo;
    for (int64_t e = lo; e < lo + n; ++e) {
        const int32_t v = fvars[e];
        if (v < 0 || v >= nv)
            return report ? fail(FBP_ERR_INVALID_ARG, "factor %d: variable %d out of range", a, v) : FBP_ERR_INVALID_ARG;
        if (n <= 64)
            for (int64_t q = lo; q < e; ++q)
                if (fvars[q] == v)
                    return report ? fail(FBP_ERR_INVALID_ARG, "factor %d lists variable %d twice", a, v)
                                  : FBP_ERR_INVALID_ARG;
    }
    if (n > 64) {  // a wide factor: sort a copy; report the first repeat in row order
        try {  // (this may run on a worker thread: nothing may escape it)
            std::vector<int32_t> tmp(fvars + lo, fvars + lo + n);
            std::sort(tmp.begin(), tmp.end());
            if (std::adjacent_find(tmp.begin(), tmp.end()) != tmp.end()) {
                if (!report) return FBP_ERR_INVALID_ARG;
                std::vector<int32_t> seen;
                for (int64_t e = lo; e < lo + n; ++e) {
                    const auto it = std::lower_bound(seen.begin(), seen.end(), fvars[e]);
                    if (it != seen.end() && *it == fvars[e])
                        return fail(FBP_ERR_INVALID_ARG, "factor %d lists variable %d twice", a, fvars[e]);
                    seen.insert(it, fvars[e]);
                }
            }
        } catch (const std::bad_alloc &) {
            return report ? fail(FBP_ERR_OOM, "host memory exhausted checking factor %d", a) : FBP_ERR_OOM;
        }
    }
    const int t = ftype[a];
    const float p = fparam[a];
    bool ok;
    switch (t) {
    case FBP_AND: case FBP_OR: case FBP_NOISY_IMPLY: case FBP_NOISY_AND: ok = n >= 2; break;
    case FBP_NOT: ok = n == 2; break;
    case FBP_EQ: ok = n >= 1; break;
    case FBP_PRIOR: ok = n == 1; break;
    case FBP_TERMS: ok = n >= 1 && n <= kTermsMaxVars; break;
    default: return report ? fail(FBP_ERR_INVALID_ARG, "factor %d: unknown type %d", a, t) : FBP_ERR_INVALID_ARG;
    }
    if (!ok)
        return report ? fail(FBP_ERR_INVALID_ARG, "factor %d: arity %lld invalid for type %d", a, (long long)n, t)
                      : FBP_ERR_INVALID_ARG;
    if ((t == FBP_NOISY_IMPLY || t == FBP_NOISY_AND || t == FBP_PRIOR) && !(p >= 0.f && p <= 1.f))
        return report ? fail(FBP_ERR_INVALID_ARG, "factor %d: parameter outside [0,1]", a) : FBP_ERR_INVALID_ARG;
    return FBP_OK;
}

int check_graph_args(int32_t nv, int32_t na, const int64_t *fptr, const int32_t *fvars,
                     const uint8_t *ftype, const float *fparam, const float *prior,
                     const int8_t *evidence)
{
    if (nv < 0 || na < 0) return fail(FBP_ERR_INVALID_ARG, "negative size");
    if (!fptr) return fail(FBP_ERR_INVALID_ARG, "factor_ptr is NULL");
    if (fptr[0] != 0) return fail(FBP_ERR_INVALID_ARG, "factor_ptr[0] != 0");
    for (int32_t a = 0; a < na; ++a)
        if (fptr[a + 1] < fptr[a]) return fail(FBP_ERR_INVALID_ARG, "factor_ptr decreases at %d", a);
    const int64_t E = fptr[na];
    if (E >= (int64_t)1 << 31) return fail(FBP_ERR_INVALID_ARG, "too many edges (%lld)", (long long)E);
    if (E > 0 && !fvars) return fail(FBP_ERR_INVALID_ARG, "factor_vars is NULL");
    if (na > 0 && (!ftype || !fparam)) return fail(FBP_ERR_INVALID_ARG, "factor_type/param NULL");
    // the factors in parallel; the lowest-numbered bad factor is reported
    std::atomic<int32_t> first_bad{std::numeric_limits<int32_t>::max()};
    parallel_for(na, host_threads_all(), 1 << 15, [&](int64_t b, int64_t e) {
        for (int64_t a = b; a < e && a < first_bad.load(std::memory_order_relaxed); ++a)
            if (check_factor(nv, fptr, fvars, ftype, fparam, (int32_t)a, false)) {
                int32_t cur = first_bad.load(std::memory_order_relaxed);
                while ((int32_t)a < cur && !first_bad.compare_exchange_weak(cur, (int32_t)a)) {
                }
                break;
            }
    });
    if (first_bad.load() != std::numeric_limits<int32_t>::max())
        return check_factor(nv, fptr, fvars, ftype, fparam, first_bad.load(), true);
    if (prior)
        for (int32_t v = 0; v < nv; ++v)
            if (!std::isnan(prior[v]) && !(prior[v] >= 0.f && prior[v] <= 1.f))
                return fail(FBP_ERR_INVALID_ARG, "prior of variable %d outside [0,1]", v);
    if (evidence)
        for (int32_t v = 0; v < nv; ++v)
            if (evidence[v] < -1 || evidence[v] > 1)
                return fail(FBP_ERR_INVALID_ARG, "evidence of variable %d not in {-1,0,1}", v);
    return FBP_OK;
}

}  // namespace fbp

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" const char *fbp_last_error(void) { return t_err.c_str(); }

extern "C" void fbp_graph_destroy(fbp_graph *g)
{
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    else cudaDeviceSynchronize();
    flood_exec_drop(g);
    std::vector<void *> all = g->owned;
    for (void *p : all) dfree(g, p);
    if (g->h_res) cudaFreeHost(g->h_res);
    if (g->h_out) cudaFreeHost(g->h_out);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    delete g;
}

extern "C" int fbp_graph_create(int32_t n_vars, int32_t n_factors, const int64_t *factor_ptr,
                                const int32_t *factor_vars, const uint8_t *factor_type,
                                const float *factor_param, const float *prior_p1,
                                const int8_t *evidence, const fbp_allocator *alloc,
                                void *cuda_stream, fbp_graph **out)
{
    t_err.clear();
    if (!out) return fail(FBP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_graph_args(n_vars, n_factors, factor_ptr, factor_vars, factor_type, factor_param,
                              prior_p1, evidence);
    if (rc) return rc;
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(FBP_ERR_INVALID_ARG, "allocator incomplete");

    fbp_graph *g = new fbp_graph();
    g->stream = (cudaStream_t)cuda_stream;
    if (alloc) {
        g->alloc = *alloc;
        g->has_alloc = true;
    }
    build_host_csr(n_vars, n_factors, factor_ptr, factor_vars, factor_type, factor_param, g->h);
    const HostCSR &h = g->h;
    g->prior.assign(prior_p1 ? prior_p1 : nullptr, prior_p1 ? prior_p1 + n_vars : nullptr);
    if (!prior_p1) g->prior.assign(n_vars, std::numeric_limits<float>::quiet_NaN());
    g->evidence.assign(evidence ? evidence : nullptr, evidence ? evidence + n_vars : nullptr);
    if (!evidence) g->evidence.assign(n_vars, (int8_t)-1);
    g->phi.resize(n_vars);
    parallel_for(n_vars, host_threads_all(), 1 << 16, [&](int64_t b, int64_t e) {
        for (int64_t v = b; v < e; ++v) g->phi[v] = phi_of(g->prior[v], g->evidence[v]);
    });

    int32_t *fptr32 = nullptr, *fvars = nullptr, *efac = nullptr, *vptr = nullptr, *vedge = nullptr;
    uint8_t *ftype = nullptr;
    float *fparam = nullptr, *phi = nullptr;
    std::vector<int32_t> fp32(h.fptr.begin(), h.fptr.end());
    if ((rc = upload(g, &fptr32, fp32.data(), fp32.size())) ||
        (rc = upload(g, &ftype, h.ftype.data(), h.ftype.size())) ||
        (rc = upload(g, &fparam, h.fparam.data(), h.fparam.size())) ||
        (rc = upload(g, &fvars, h.fvars.data(), h.fvars.size())) ||
        (rc = upload(g, &efac, h.efac.data(), h.efac.size())) ||
        (rc = upload(g, &vptr, h.vptr.data(), h.vptr.size())) ||
        (rc = upload(g, &vedge, h.vedge.data(), h.vedge.size())) ||
        (rc = upload(g, &phi, g->phi.data(), g->phi.size())) ||
        (rc = dalloc_n(g, &g->d_bar, 2)) ||
        (rc = dalloc_n(g, &g->d_out, 4)) ||
        (rc = dalloc_n(g, &g->a2v[0], (size_t)h.ne)) ||
        (rc = dalloc_n(g, &g->d_res, (size_t)kResSlots)) ||
        (rc = dalloc_n(g, &g->d_guards, 1))) {
        std::string keep = t_err;
        fbp_graph_destroy(g);
        t_err = keep;
        return rc;
    }
    g->d.nv = n_vars;
    g->d.na = n_factors;
    g->d.ne = h.ne;
    g->d.fptr = fptr32;
    g->d.ftype = ftype;
    g->d.fparam = fparam;
    g->d.fvars = fvars;
    g->d.efac = efac;
    g->d.vptr = vptr;
    g->d.vedge = vedge;
    g->d.phi = phi;
    launch_fill(g->a2v[0], 1.0f, h.ne, g->stream);  // uniform initial messages
    cudaError_t e = cudaMallocHost((void **)&g->h_res, sizeof(unsigned) * kResSlots);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&g->h_out, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = cudaEventCreate(&g->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&g->ev1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        fbp_graph_destroy(g);
        return fail(FBP_ERR_CUDA, "graph setup: %s", cudaGetErrorString(e));
    }
    LevelSet ls;
    ls.lp = {0, (int64_t)h.ne};
    if (h.ne == 0) ls.lp = {0};
    g->halves.push_back(std::move(ls));
    g->strategy = FBP_PARALL;
    for (int32_t a = 0; a < n_factors && !g->terms_needed; ++a) g->terms_needed = factor_type[a] == FBP_TERMS;
    *out = g;
    return FBP_OK;
}

extern "C" int fbp_set_factor_terms(fbp_graph *g, const int64_t *term_ptr, const int8_t *term_ind,
                                    const float *term_w)
{
    t_err.clear();
    if (!g || !term_ptr) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    const HostCSR &h = g->h;
    if (term_ptr[0] != 0) return fail(FBP_ERR_INVALID_ARG, "term_ptr[0] != 0");
    std::vector<int32_t> tptr(h.na + 1), tioff(std::max(h.na, 1));
    int64_t ioff = 0;
    for (int32_t a = 0; a < h.na; ++a) {
        const int64_t l = term_ptr[a + 1] - term_ptr[a];
        const int64_t b = h.fptr[a + 1] - h.fptr[a];
        if (l < 0) return fail(FBP_ERR_INVALID_ARG, "term_ptr decreases at factor %d", a);
        if (h.ftype[a] != FBP_TERMS && l != 0)
            return fail(FBP_ERR_INVALID_ARG, "factor %d is not generic but has terms", a);
        if (l > kTermsMaxTerms) return fail(FBP_ERR_INVALID_ARG, "factor %d has more than %d terms", a, kTermsMaxTerms);
        tptr[a] = (int32_t)term_ptr[a];
        tioff[a] = (int32_t)ioff;
        ioff += l * b;
        if (ioff >= ((int64_t)1 << 31)) return fail(FBP_ERR_INVALID_ARG, "term lists too large");
    }
    const int64_t nt = term_ptr[h.na];
    if (nt >= ((int64_t)1 << 31)) return fail(FBP_ERR_INVALID_ARG, "too many terms");
    tptr[h.na] = (int32_t)nt;
    if ((nt > 0 && !term_w) || (ioff > 0 && !term_ind)) return fail(FBP_ERR_INVALID_ARG, "NULL term arrays");
    for (int64_t k = 0; k < ioff; ++k)
        if (term_ind[k] < -1 || term_ind[k] > 1) return fail(FBP_ERR_INVALID_ARG, "indicator %lld not in {-1,0,1}", (long long)k);
    for (int64_t t = 0; t < nt; ++t)
        if (!(term_w[t] >= 0.f) || !std::isfinite(term_w[t])) return fail(FBP_ERR_INVALID_ARG, "term %lld: weight not finite and >= 0", (long long)t);
    if (g->d.tptr) {  // replacing earlier lists
        dfree(g, (void *)g->d.tptr);
        dfree(g, (void *)g->d.tioff);
        dfree(g, (void *)g->d.tind);
        dfree(g, (void *)g->d.tw);
        g->d.tptr = g->d.tioff = nullptr;
        g->d.tind = nullptr;
        g->d.tw = nullptr;
    }
    int32_t *d_tptr = nullptr, *d_tioff = nullptr;
    int8_t *d_tind = nullptr;
    float *d_tw = nullptr;
    int rc;
    if ((rc = upload(g, &d_tptr, tptr.data(), tptr.size())) || (rc = upload(g, &d_tioff, tioff.data(), tioff.size())))
        return rc;
    // empty lists still get a (never read) one-element buffer
    if ((rc = ioff > 0 ? upload(g, &d_tind, term_ind, (size_t)ioff) : dalloc_n(g, &d_tind, 1)) ||
        (rc = nt > 0 ? upload(g, &d_tw, term_w, (size_t)nt) : dalloc_n(g, &d_tw, 1)))
        return rc;
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    g->d.tptr = d_tptr;
    g->d.tioff = d_tioff;
    g->d.tind = d_tind;
    g->d.tw = d_tw;
    g->terms_set = true;
    flood_exec_drop(g);  // captured chunks hold the graph structure by value
    return FBP_OK;
}

extern "C" int fbp_schedule_set(fbp_graph *g, const fbp_schedule_spec *spec)
{
    t_err.clear();
    if (g) g->rs_levels_pending = false;
    if (!g || !spec) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    const HostCSR &h = g->h;
    std::vector<LevelSet> halves;
    int s = spec->strategy;
    if (s == FBP_RESIDUAL) {
        if (spec->residual_buckets != 0 && spec->residual_buckets != 3)
            return fail(FBP_ERR_INVALID_ARG, "residual_buckets must be 0 or 3");
        LevelSet ls;  // iteration 1 is PARALL
        ls.lp = {0, (int64_t)h.ne};
        if (h.ne == 0) ls.lp = {0};
        halves.push_back(std::move(ls));
    } else if (s == FBP_PARALL) {
        LevelSet ls;  // one class: Algorithm 2 cannot cut, every edge in one level
        ls.lp = {0, (int64_t)h.ne};
        if (h.ne == 0) ls.lp = {0};
        halves.push_back(std::move(ls));
    } else {
        const int nh = s == FBP_TOPO_FB ? 2 : 1;
        std::vector<int64_t> rank[2];
        int rc = build_ranks(h, *spec, 0, rank[0]);
        if (rc) return rc;
        if (nh == 2) backward_ranks(rank[0], rank[1]);
        halves.resize(nh);
        std::vector<LevelPack> packs(nh);
        const int max_fan = engine_max_fan();
        auto half_work = [&](int b) {
            dependency_levels(h, rank[b].data(), nullptr, h.ne, halves[b].lp, halves[b].le);
            pack_levels(h, g->fac_graph, halves[b].lp, halves[b].le, max_fan, packs[b]);
        };
        // the two halves of TOPO_FB are independent: the backward one on a
        // second host thread
        bool spawned_ok = true;
        std::thread second;
        if (nh == 2) {
            try {
                second = std::thread([&] {
                    try {
                        half_work(1);
                    } catch (...) {
                        spawned_ok = false;
                    }
                });
            } catch (...) {
                half_work(1);  // no thread to be had: run it here
            }
        }
        try {
            half_work(0);
        } catch (...) {
            if (second.joinable()) second.join();
            return fail(FBP_ERR_OOM, "host memory exhausted while building the schedule");
        }
        if (second.joinable()) second.join();
        if (!spawned_ok) return fail(FBP_ERR_OOM, "host memory exhausted while building the schedule");
        free_levels(g);
        g->halves = std::move(halves);
        g->strategy = s;
        for (int b = 0; b < nh; ++b)
            if ((rc = upload_levels(g, g->halves[b], &packs[b]))) return rc;
        if (!g->a2v[1] && dalloc_n(g, &g->a2v[1], (size_t)h.ne)) return FBP_ERR_OOM;
        return FBP_OK;
    }
    free_levels(g);
    g->halves = std::move(halves);
    g->strategy = s;
    if (s == FBP_RESIDUAL) {
        for (auto &ls : g->halves) {
            if (ls.le.empty() && h.ne) {  // PARALL list (RESIDUAL's first iteration)
                ls.le.resize(h.ne);
                for (int32_t e = 0; e < h.ne; ++e) ls.le[e] = e;
            }
            int rc = upload_levels(g, ls);
            if (rc) return rc;
        }
        if (!g->a2v[1] && dalloc_n(g, &g->a2v[1], (size_t)h.ne)) return FBP_ERR_OOM;
    }
    if (s == FBP_RESIDUAL) {
        if (!g->dres && dalloc_n(g, &g->dres, (size_t)h.ne)) return FBP_ERR_OOM;
        if (!g->d_act && dalloc_n(g, &g->d_act, (size_t)h.ne)) return FBP_ERR_OOM;
    }
    return FBP_OK;
}

extern "C" int fbp_schedule_build_host(int32_t n_vars, int32_t n_factors, const int64_t *factor_ptr,
                                       const int32_t *factor_vars, const fbp_schedule_spec *spec,
                                       int32_t backward, int32_t *n_levels, int64_t *level_ptr,
                                       int32_t *level_edges)
{
    t_err.clear();
    if (!spec || !n_levels) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    if (n_vars < 0 || n_factors < 0 || !factor_ptr || factor_ptr[0] != 0)
        return fail(FBP_ERR_INVALID_ARG, "bad CSR");
    for (int32_t a = 0; a < n_factors; ++a)
        if (factor_ptr[a + 1] < factor_ptr[a]) return fail(FBP_ERR_INVALID_ARG, "bad CSR");
    const int64_t E = factor_ptr[n_factors];
    if (E >= (int64_t)1 << 31) return fail(FBP_ERR_INVALID_ARG, "too many edges");
    for (int64_t e = 0; e < E; ++e)
        if (factor_vars[e] < 0 || factor_vars[e] >= n_vars) return fail(FBP_ERR_INVALID_ARG, "bad variable");
    if (spec->strategy == FBP_RESIDUAL) return fail(FBP_ERR_INVALID_ARG, "RESIDUAL levels are dynamic");
    HostCSR h;
    std::vector<uint8_t> t(n_factors, 0);
    std::vector<float> p(n_factors, 0.f);
    build_host_csr(n_vars, n_factors, factor_ptr, factor_vars, t.data(), p.data(), h);
    std::vector<int64_t> lp;
    std::vector<int32_t> le;
    if (spec->strategy == FBP_PARALL) {
        lp = {0, (int64_t)h.ne};
        if (h.ne == 0) lp = {0};
        le.resize(h.ne);
        std::iota(le.begin(), le.end(), 0);
    } else {
        std::vector<int64_t> rank;
        int rc = build_ranks(h, *spec, backward ? 1 : 0, rank);
        if (rc) return rc;
        dependency_levels(h, rank.data(), nullptr, h.ne, lp, le);
    }
    *n_levels = (int32_t)(lp.size() - 1);
    if (level_ptr) std::copy(lp.begin(), lp.end(), level_ptr);
    if (level_edges) std::copy(le.begin(), le.end(), level_edges);
    return FBP_OK;
}

extern "C" int fbp_schedule_levels(const fbp_graph *g, int32_t *n_levels, int64_t *level_ptr,
                                   int32_t *level_edges)
{
    t_err.clear();
    if (!g || !n_levels) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    if (g->rs_levels_pending && g->strategy == FBP_RESIDUAL) {  // the last device-scheduled RESIDUAL iteration's levels
        int rc = fetch_residual_levels(const_cast<fbp_graph *>(g));
        if (rc) return rc;
    }
    int32_t k = 0;
    for (auto &ls : g->halves) k += (int32_t)ls.lp.size() - 1;
    *n_levels = k;
    if (!level_ptr && !level_edges) return FBP_OK;
    int64_t base = 0;
    int32_t j = 0;
    if (level_ptr) level_ptr[0] = 0;
    for (auto &ls : g->halves) {
        for (size_t L = 1; L < ls.lp.size(); ++L) {
            if (level_ptr) level_ptr[++j] = base + ls.lp[L];
        }
        if (level_edges) {
            if (!ls.le.empty()) std::copy(ls.le.begin(), ls.le.end(), level_edges + base);
            else for (int32_t e = 0; e < g->h.ne; ++e) level_edges[base + e] = e;  // PARALL
        }
        base += ls.lp.back();
    }
    return FBP_OK;
}

// ---------------------------------------------------------------------------
// iteration driver
// ---------------------------------------------------------------------------
namespace fbp {

int read_residual(fbp_graph *g, double *res)
{
    CUDA_TRY(cudaMemcpyAsync(g->h_res, g->d_res, sizeof(unsigned) * kResSlots, cudaMemcpyDeviceToHost,
                             g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    unsigned m = 0;
    for (int i = 0; i < kResSlots; ++i) m = std::max(m, g->h_res[i]);
    float f;
    std::memcpy(&f, &m, sizeof f);
    *res = (double)f;
    return FBP_OK;
}

int ensure_res_cap(fbp_graph *g, int32_t n)
{
    if (n <= g->res_cap) return FBP_OK;
    dfree(g, g->d_res_it);
    g->d_res_it = nullptr;
    g->res_cap = 0;
    int32_t cap = std::max<int32_t>(n, 64);
    int rc = dalloc_n(g, &g->d_res_it, (size_t)cap);
    if (rc) return rc;
    g->res_cap = cap;
    return FBP_OK;
}

LevelPlanDev plan_of(const LevelSet &ls)
{
    LevelPlanDev p;
    p.lanes = ls.d_lanes;
    p.lrow = ls.d_lrow;
    p.lane_ptr = ls.d_lane_ptr;
    p.big = ls.d_big;
    p.big_ptr = ls.d_big_ptr;
    p.vel = ls.d_vel;
    p.n_levels = (int32_t)ls.lp.size() - 1;
    return p;
}

// Launch shape of the engine: one cluster (hardware barrier, the fastest
// level step) when the widest level fits the cluster's prefetched work items,
// otherwise a cooperative grid just wide enough for the widest level.
// Launch shape of the engine.  Default: a cooperative grid of one block per
// SM (a level's warps are spread round-robin over the blocks), grown if the
// widest level needs more lanes.  Cluster mode (one cluster, hardware
// barrier) only when asked for.
void engine_shape(const fbp_graph *g, int *grid, int *cluster)
{
    int32_t mx = 32;
    for (auto &ls : g->halves) mx = std::max(mx, ls.max_lanes);
    const int lanes_per_block = engine_block();
    *cluster = 0;
    if (g->engine_grid > 0) {
        *grid = g->engine_grid;
        return;
    }
    if (g->engine_cluster == 8 || g->engine_cluster == 16) {
        const int csize = engine_cluster_size();
        if (csize > 0) {
            *cluster = std::min(g->engine_cluster, csize);
            *grid = *cluster;
            return;
        }
    }
    // With the barrier engine, levels that average at most engine_solo lanes
    // (FBP_OPT_ENGINE_SOLO_LANES, default 128) run in one block, whose level
    // barrier is a block barrier (measured on GB300: 2.5 us per level against
    // 3.4-3.6 us with a grid barrier at 11-100 edges per level; wider levels
    // are faster spread over the grid).
    int64_t lanes = 0, levels = 0;
    for (auto &ls : g->halves) {
        lanes += ls.n_lanes;
        levels += (int64_t)ls.lp.size() - 1;
    }
    if (g->use_engine == 1 && levels > 0 && lanes <= (int64_t)g->engine_solo * levels) {
        *grid = 1;
        return;
    }
    const int need = (mx + lanes_per_block - 1) / lanes_per_block;
    *grid = std::min(std::max(need, num_sms()), engine_max_grid());
}

EngineArgs engine_args(fbp_graph *g)
{
    EngineArgs A;
    A.g = g->d;
    A.erow = g->erow;
    A.n_halves = (int32_t)g->halves.size();
    for (int h = 0; h < A.n_halves && h < 2; ++h) A.half[h] = plan_of(g->halves[h]);
    A.buf[0] = g->a2v[g->cur];
    A.buf[1] = g->a2v[g->cur ^ 1];
    A.guards = g->d_guards;
    A.bar = g->d_bar;
    A.out = g->d_out;
    A.spin_limit = g->spin_limit;
    for (auto &ls : g->halves) A.max_lanes = std::max(A.max_lanes, ls.max_lanes);
    A.dataflow = g->use_engine == 2;
    A.fuse_lanes = std::min(g->engine_fuse, engine_block());
    return A;
}

int engine_check(fbp_graph *g)
{
    CUDA_TRY(cudaMemcpyAsync(g->h_out, g->d_out, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (g->h_out[2]) return fail(FBP_ERR_TIMEOUT, "a device-side barrier wait expired (spin limit %lld cycles)",
                                 (long long)g->spin_limit);
    return FBP_OK;
}

int finish_run(fbp_graph *g, int32_t it, double res, int status, int32_t *iters_out, double *residual_out)
{
    CUDA_TRY(cudaEventRecord(g->ev1, g->stream));
    CUDA_TRY(cudaEventSynchronize(g->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev0, g->ev1);
    unsigned long long guards = 0;
    CUDA_TRY(cudaMemcpy(&guards, g->d_guards, sizeof guards, cudaMemcpyDeviceToHost));
    g->stats.iters = it;
    g->stats.residual = res;
    g->stats.run_ms = ms;
    g->stats.guards = (int64_t)guards;
    if (iters_out) *iters_out = it;
    if (residual_out) *residual_out = res;
    return status;
}

int marginals_launch(fbp_graph *g, float *dst, cudaStream_t s)
{
    if (g->n_marg_rows < 0) {
        std::vector<int32_t> rows;
        const int32_t cap = marginals_row_max();
        for (int32_t v = 0; v < g->h.nv; ++v)
            if (g->h.vptr[v + 1] - g->h.vptr[v] > cap) rows.push_back(v);
        int rc = upload(g, &g->marg_rows, rows.data(), rows.size());
        if (rc) return rc;
        g->n_marg_rows = (int32_t)rows.size();
    }
    launch_marginals(g->d, g->a2v[g->cur], dst, s);
    launch_marginals_long(g->d, g->a2v[g->cur], dst, g->marg_rows, g->n_marg_rows, s);
    CUDA_TRY(cudaGetLastError());
    return FBP_OK;
}

double residual_at(fbp_graph *g, int32_t it)
{
    if (it < 1) return 0.0;
    unsigned bits = 0;
    cudaMemcpy(&bits, g->d_res_it + (it - 1), sizeof bits, cudaMemcpyDeviceToHost);
    float f;
    std::memcpy(&f, &bits, sizeof f);
    return (double)f;
}

// Static strategy, persistent engine: the whole run in one launch.
int run_engine(fbp_graph *g, int32_t max_iters, double tol, int32_t *iters_out, double *residual_out)
{
    const HostCSR &h = g->h;
    int rc = ensure_res_cap(g, std::max(max_iters, 1));
    if (rc) return rc;
    CUDA_TRY(cudaMemsetAsync(g->d_res_it, 0, sizeof(unsigned) * std::max(max_iters, 1), g->stream));
    CUDA_TRY(cudaMemsetAsync(g->d_bar, 0, sizeof(unsigned) * 2, g->stream));
    CUDA_TRY(cudaMemsetAsync(g->d_out, 0, sizeof(int32_t) * 4, g->stream));
    EngineArgs A = engine_args(g);
    A.res = g->d_res_it;
    A.max_iters = max_iters;
    A.tol = (float)tol;
    if (max_iters == 0) return finish_run(g, 0, 0.0, FBP_NOT_CONVERGED, iters_out, residual_out);
    int grid = 1, cluster = 0;
    engine_shape(g, &grid, &cluster);
    CUDA_TRY(launch_engine(A, grid, cluster, g->stream));
    g->stats.kernel_launches += 1;
    rc = engine_check(g);
    if (rc) return rc;
    const int32_t it = g->h_out[0];
    const int status = g->h_out[1] == 0 ? FBP_OK : FBP_NOT_CONVERGED;
    g->cur ^= (it * A.n_halves) & 1;
    g->stats.updates += (int64_t)it * A.n_halves * h.ne;
    return finish_run(g, it, residual_at(g, it), status, iters_out, residual_out);
}

// Static strategy, one launch per level (the execution of Sec. 4.3.3).
int run_per_level(fbp_graph *g, int32_t max_iters, double tol, int32_t *iters_out, double *residual_out)
{
    const HostCSR &h = g->h;
    int rc = ensure_res_cap(g, std::max(max_iters, 1));
    if (rc) return rc;
    CUDA_TRY(cudaMemsetAsync(g->d_res_it, 0, sizeof(unsigned) * std::max(max_iters, 1), g->stream));
    CUDA_TRY(cudaMemsetAsync(g->d_out, 0, sizeof(int32_t) * 4, g->stream));  // result and error words
    int grid = 1, cluster = 0;
    engine_shape(g, &grid, &cluster);
    int32_t it = 0;
    double res = 0.0;
    int status = FBP_NOT_CONVERGED;
    for (it = 1; it <= max_iters; ++it) {
        for (auto &ls : g->halves) {
            LevelPlanDev full = plan_of(ls);
            for (int32_t L = 0; L < full.n_levels; ++L) {
                CUDA_TRY(cudaMemsetAsync(g->d_bar, 0, sizeof(unsigned) * 2, g->stream));
                EngineArgs A = engine_args(g);
                A.dataflow = 0;
                LevelPlanDev one = full;
                one.lane_ptr = full.lane_ptr + L;
                one.big_ptr = full.big_ptr + L;
                one.n_levels = 1;
                one.level_base = L;
                A.half[0] = one;
                A.n_halves = 1;
                A.res = g->d_res_it + (it - 1);
                A.max_iters = 1;
                A.tol = 0.f;
                CUDA_TRY(launch_engine(A, grid, cluster, g->stream));
                g->stats.kernel_launches += 1;
            }
            g->cur ^= 1;
            g->stats.updates += h.ne;
        }
        rc = engine_check(g);
        if (rc) return rc;
        res = residual_at(g, it);
        if (res < tol || h.ne == 0) {
            status = FBP_OK;
            break;
        }
    }
    if (it > max_iters) it = max_iters;
    return finish_run(g, it, res, status, iters_out, residual_out);
}

}  // namespace fbp

extern "C" int fbp_run(fbp_graph *g, int32_t max_iters, double tol, int32_t *iters_out,
                       double *residual_out)
{
    t_err.clear();
    if (!g || max_iters < 0 || !(tol >= 0.0)) return fail(FBP_ERR_INVALID_ARG, "bad argument");
    if (g->terms_needed && !g->terms_set)
        return fail(FBP_ERR_INVALID_ARG, "generic (FBP_TERMS) factors have no terms: call fbp_set_factor_terms");
    const HostCSR &h = g->h;
    g->stats = fbp_stats{};
    for (auto &ls : g->halves) g->stats.levels += (int32_t)ls.lp.size() - 1;
    CUDA_TRY(cudaMemsetAsync(g->d_guards, 0, sizeof(unsigned long long), g->stream));
    CUDA_TRY(cudaEventRecord(g->ev0, g->stream));
    if (g->strategy == FBP_RESIDUAL)
        return g->residual_device ? fbp_run_residual_device(g, max_iters, tol, iters_out, residual_out)
                                  : fbp_run_residual(g, max_iters, tol, iters_out, residual_out);
    if (g->strategy != FBP_PARALL) {
        if (g->use_engine == 3) return run_seq(g, max_iters, tol, iters_out, residual_out);
        return g->use_engine ? run_engine(g, max_iters, tol, iters_out, residual_out)
                             : run_per_level(g, max_iters, tol, iters_out, residual_out);
    }
    // flooding: a captured chunk of kFloodChunk iterations is replayed in
    // growing batches; the device counts iterations, marks the run done at
    // convergence or at the limit, and later kernels return at once
    if (!g->a2v_vm && dalloc_n(g, &g->a2v_vm, (size_t)h.ne)) return FBP_ERR_OOM;
    if (!g->flood_ready) {
        int rc = build_flood_plan(g);
        if (rc) return rc;
    }
    int rc = ensure_res_cap(g, std::max(max_iters, 1));
    if (rc) return rc;
    if (max_iters == 0) return finish_run(g, 0, 0.0, FBP_NOT_CONVERGED, iters_out, residual_out);
    cudaGraphExec_t exec = nullptr;
    if ((rc = flood_exec_for(g, g->flood, (float)tol, kFloodChunk, &exec))) return rc;
    flood_sync(g->d, g->a2v[g->cur], g->a2v_vm, g->stream);  // the messages may have changed since
    g->stats.kernel_launches += h.ne > 0;
    CUDA_TRY(cudaMemsetAsync(g->d_res, 0, sizeof(unsigned) * kResSlots, g->stream));
    g->h_out[0] = g->h_out[1] = g->h_out[2] = 0;
    g->h_out[3] = max_iters;
    CUDA_TRY(cudaMemcpyAsync(g->d_out, g->h_out, sizeof(int32_t) * 4, cudaMemcpyHostToDevice, g->stream));
    const int launches_per_iter = flood_launches(g->d, g->flood);
    int32_t queued = 0, reps = 1;
    while (queued < max_iters) {
        for (int32_t r = 0; r < reps && queued < max_iters; ++r) {
            CUDA_TRY(cudaGraphLaunch(exec, g->stream));
            queued += kFloodChunk;
            g->stats.kernel_launches += (int64_t)kFloodChunk * launches_per_iter;
        }
        CUDA_TRY(cudaMemcpyAsync(g->h_out, g->d_out, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, g->stream));
        CUDA_TRY(cudaStreamSynchronize(g->stream));
        if (g->h_out[0] != 0) break;
        reps = std::min(reps * 2, 8);
    }
    const int32_t it = g->h_out[1];
    g->stats.updates += (int64_t)it * h.ne;
    return finish_run(g, it, residual_at(g, it), g->h_out[0] == 1 ? FBP_OK : FBP_NOT_CONVERGED, iters_out,
                      residual_out);
}

int fbp::flood_exec_for(fbp_graph *g, const FloodPlanDev &F, float tol, int iters, cudaGraphExec_t *out)
{
    const void *key[3] = {g->a2v[g->cur], g->d_res_it, F.warps};
    if (g->flood_exec && g->flood_exec_iters == iters && g->flood_exec_tol == tol &&
        std::equal(key, key + 3, g->flood_exec_key)) {
        *out = g->flood_exec;
        return FBP_OK;
    }
    flood_exec_drop(g);
    IterCtl ctl{g->d_res, g->d_guards};
    CUDA_TRY(flood_capture(g->d, F, g->a2v[g->cur], g->a2v_vm, ctl, tol, g->d_res_it, g->d_out, iters, &g->flood_exec));
    g->flood_exec_iters = iters;
    g->flood_exec_tol = tol;
    std::copy(key, key + 3, g->flood_exec_key);
    *out = g->flood_exec;
    return FBP_OK;
}

void fbp::flood_exec_drop(fbp_graph *g)
{
    if (g->flood_exec) cudaGraphExecDestroy(g->flood_exec);
    g->flood_exec = nullptr;
    g->flood_exec_iters = 0;
}

// RESIDUAL strategy with the schedule on the device: iteration 1 is one
// flooding iteration; every later iteration derives the classes and the
// Algorithm 2 levels from the previous iteration's per-edge changes on the
// device (residual_schedule) and runs each level as a flooding step that
// writes only that level's edges (v->a messages from the level-start state,
// as the level execution prescribes).  Stops at the first iteration whose
// residual is below tol, or when no factor is active.
int fbp_run_residual_device(fbp_graph *g, int32_t max_iters, double tol, int32_t *iters_out,
                            double *residual_out)
{
    const HostCSR &h = g->h;
    int rc;
    if (!g->a2v_vm && (rc = dalloc_n(g, &g->a2v_vm, (size_t)h.ne))) return rc;
    if (!g->flood_ready && (rc = build_flood_plan(g))) return rc;
    if ((rc = ensure_res_cap(g, std::max(max_iters, 1)))) return rc;
    if (!g->dres && (rc = dalloc_n(g, &g->dres, (size_t)std::max(h.ne, 1)))) return rc;
    if (!g->rs.ctl) {
        if ((rc = dalloc_n(g, &g->rs.vres, (size_t)std::max(h.nv, 1))) || (rc = dalloc_n(g, &g->rs.cnt, (size_t)std::max(h.nv, 1))) ||
            (rc = dalloc_n(g, &g->rs.fcls, (size_t)std::max(h.na, 1))) ||
            (rc = dalloc_n(g, &g->rs.elev, (size_t)std::max(h.ne, 1))) || (rc = dalloc_n(g, &g->rs.ctl, 4)))
            return rc;
    }
    CUDA_TRY(cudaMemsetAsync(g->d_res_it, 0, sizeof(unsigned) * std::max(max_iters, 1), g->stream));
    if (max_iters == 0) return finish_run(g, 0, 0.0, FBP_NOT_CONVERGED, iters_out, residual_out);
    CUDA_TRY(cudaMemsetAsync(g->d_res, 0, sizeof(unsigned) * kResSlots, g->stream));
    g->h_out[0] = g->h_out[1] = g->h_out[2] = 0;
    g->h_out[3] = max_iters;
    CUDA_TRY(cudaMemcpyAsync(g->d_out, g->h_out, sizeof(int32_t) * 4, cudaMemcpyHostToDevice, g->stream));
    IterCtl ctl{g->d_res, g->d_guards};
    FloodPlanDev F = g->flood;
    F.dres = g->dres;
    const int per_level = flood_launches(g->d, g->flood) - 1;
    flood_sync(g->d, g->a2v[g->cur], g->a2v_vm, g->stream);
    g->stats.kernel_launches += h.ne > 0;
    int32_t it = 0, levels = 0;
    bool idle = false;  // no factor active
    int status = FBP_NOT_CONVERGED;
    for (it = 1; it <= max_iters; ++it) {
        int64_t active = h.ne;
        levels = 1;
        if (it == 1) {
            F.elevel = nullptr;
        } else {
            residual_schedule(g->d, g->dres, tol, g->rs, g->stream);
            g->stats.kernel_launches += 7;
            CUDA_TRY(cudaMemcpyAsync(g->h_res, g->rs.ctl, sizeof(int) * 4, cudaMemcpyDeviceToHost, g->stream));
            CUDA_TRY(cudaStreamSynchronize(g->stream));
            const int *c = reinterpret_cast<const int *>(g->h_res);
            active = c[kRsActive];
            levels = 1 + (c[kRsCut1] != INT_MAX) + (c[kRsCut2] != INT_MAX);
            g->rs_levels_pending = true;
            if (active == 0) {  // nothing changed by tol or more: the fixed point is reached
                idle = true;
                levels = 0;
                break;
            }
            F.elevel = g->rs.elev;
        }
        CUDA_TRY(cudaMemsetAsync(g->dres, 0, sizeof(float) * h.ne, g->stream));
        for (int32_t lv = 0; lv < levels; ++lv) {
            F.level = lv;
            flood_level(g->d, F, g->a2v[g->cur], g->a2v_vm, ctl, g->d_out, g->stream);
            g->stats.kernel_launches += per_level;
        }
        flood_check(ctl, (float)tol, g->d_res_it, g->d_out, g->stream);
        g->stats.kernel_launches += 1;
        g->stats.updates += active;
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(g->h_out, g->d_out, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, g->stream));
        CUDA_TRY(cudaStreamSynchronize(g->stream));
        if (g->h_out[0] != 0) break;
    }
    if (it > max_iters) it = max_iters;
    double res = 0.0;
    if (idle) {
        status = FBP_OK;
    } else {
        it = g->h_out[1];
        status = g->h_out[0] == 1 ? FBP_OK : FBP_NOT_CONVERGED;
        res = residual_at(g, it);
    }
    g->stats.levels = levels;
    return finish_run(g, it, res, status, iters_out, residual_out);
}

// The last device-scheduled RESIDUAL iteration's levels, on the host
// (canonical order: class, then edge id), for fbp_schedule_levels.
int fbp::fetch_residual_levels(fbp_graph *g)
{
    const HostCSR &h = g->h;
    std::vector<int8_t> fcls(h.na), elev(h.ne);
    CUDA_TRY(cudaMemcpyAsync(fcls.data(), g->rs.fcls, h.na, cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaMemcpyAsync(elev.data(), g->rs.elev, h.ne, cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    LevelSet &ls = g->halves[0];
    ls.le.clear();
    for (int c = 0; c <= 2; ++c)
        for (int32_t e = 0; e < h.ne; ++e)
            if (fcls[h.efac[e]] == c) ls.le.push_back(e);
    ls.lp.assign(1, 0);
    for (size_t i = 0; i < ls.le.size(); ++i)
        if (i > 0 && elev[ls.le[i]] != elev[ls.le[i - 1]]) ls.lp.push_back((int64_t)i);
    ls.lp.push_back((int64_t)ls.le.size());
    if (ls.le.empty()) ls.lp.assign(1, 0);
    g->rs_levels_pending = false;
    return FBP_OK;
}

// RESIDUAL strategy: the classes of the next iteration come from the previous
// iteration's per-edge changes, so its levels are rebuilt on the host every
// iteration and each iteration is one engine launch.
int fbp_run_residual(fbp_graph *g, int32_t max_iters, double tol, int32_t *iters_out,
                     double *residual_out)
{
    const HostCSR &h = g->h;
    int rc = ensure_res_cap(g, std::max(max_iters, 1));
    if (rc) return rc;
    CUDA_TRY(cudaMemsetAsync(g->d_res_it, 0, sizeof(unsigned) * std::max(max_iters, 1), g->stream));
    std::vector<float> dres(h.ne);
    std::vector<int64_t> rank(h.ne);
    std::vector<int32_t> act;
    int32_t it = 0;
    double res = 0.0;
    int status = FBP_NOT_CONVERGED;
    LevelSet &ls = g->halves[0];
    for (it = 1; it <= max_iters; ++it) {
        int64_t n;
        if (it == 1) {
            std::fill(rank.begin(), rank.end(), 0);
            act.resize(h.ne);
            for (int32_t e = 0; e < h.ne; ++e) act[e] = e;
            n = h.ne;
        } else {
            CUDA_TRY(cudaMemcpyAsync(dres.data(), g->dres, sizeof(float) * h.ne, cudaMemcpyDeviceToHost,
                                     g->stream));
            CUDA_TRY(cudaStreamSynchronize(g->stream));
            n = residual_classes(h, dres.data(), tol, rank.data(), act);
        }
        dependency_levels(h, rank.data(), act.data(), n, ls.lp, ls.le);
        rc = upload_levels(g, ls);
        if (rc) return rc;
        g->stats.levels = (int32_t)ls.lp.size() - 1;
        // inactive edges keep their value: start the other buffer as a copy
        CUDA_TRY(cudaMemcpyAsync(g->a2v[g->cur ^ 1], g->a2v[g->cur], sizeof(float) * h.ne,
                                 cudaMemcpyDeviceToDevice, g->stream));
        CUDA_TRY(cudaMemsetAsync(g->dres, 0, sizeof(float) * h.ne, g->stream));
        CUDA_TRY(cudaMemsetAsync(g->d_bar, 0, sizeof(unsigned) * 2, g->stream));
        CUDA_TRY(cudaMemsetAsync(g->d_out, 0, sizeof(int32_t) * 4, g->stream));  // result and error words
        EngineArgs A = engine_args(g);
        A.n_halves = 1;
        A.res = g->d_res_it + (it - 1);
        A.max_iters = 1;
        A.tol = 0.f;
        A.dres = g->dres;
        A.dataflow = 0;  // only the active edges are written
        if (n > 0) {
            int grid = 1, cluster = 0;
            engine_shape(g, &grid, &cluster);
            CUDA_TRY(launch_engine(A, grid, cluster, g->stream));
            g->stats.kernel_launches += 1;
        }
        g->cur ^= 1;
        g->stats.updates += n;
        rc = engine_check(g);
        if (rc) return rc;
        res = residual_at(g, it);
        if (res < tol || n == 0) {
            status = FBP_OK;
            break;
        }
    }
    if (it > max_iters) it = max_iters;
    return finish_run(g, it, res, status, iters_out, residual_out);
}

extern "C" int fbp_set_option(fbp_graph *g, int32_t option, int64_t value)
{
    t_err.clear();
    if (!g) return fail(FBP_ERR_INVALID_ARG, "NULL graph");
    switch (option) {
    case FBP_OPT_SPIN_LIMIT:
        if (value < 0) return fail(FBP_ERR_INVALID_ARG, "negative spin limit");
        g->spin_limit = value;
        return FBP_OK;
    case FBP_OPT_ENGINE_GRID:
        if (value < 0) return fail(FBP_ERR_INVALID_ARG, "negative grid");
        g->engine_grid = (int)std::min<int64_t>(value, engine_max_grid());
        return FBP_OK;
    case FBP_OPT_RESIDUAL_DEVICE:
        g->residual_device = value != 0;
        return FBP_OK;
    case FBP_OPT_ENGINE:
        if (value < 0 || value > 3) return fail(FBP_ERR_INVALID_ARG, "FBP_OPT_ENGINE must be 0, 1, 2 or 3");
        g->use_engine = (int)value;
        return FBP_OK;
    case FBP_OPT_FLOOD_HUB_MIN:
        if (value < kFloodSmallMax || value > kFloodMediumMax)
            return fail(FBP_ERR_INVALID_ARG, "hub threshold must be in [%d, %d]", kFloodSmallMax, kFloodMediumMax);
        g->flood_hub_min = (int)value;
        g->flood_ready = false;  // rebuilt at the next flooding run
        return FBP_OK;
    case FBP_OPT_FLOOD_CHUNK:
        if (value < kFloodChunkUnit || value > (1 << 16) || value % kFloodChunkUnit != 0)
            return fail(FBP_ERR_INVALID_ARG, "chunk must be a multiple of %d in [%d, 65536]", kFloodChunkUnit,
                        kFloodChunkUnit);
        g->flood_chunk = (int)value;
        g->flood_ready = false;
        return FBP_OK;
    case FBP_OPT_ENGINE_CLUSTER:
        if (value != 0 && value != 1 && value != 8 && value != 16)
            return fail(FBP_ERR_INVALID_ARG, "cluster option must be 0, 1, 8 or 16");
        g->engine_cluster = (int)value;
        return FBP_OK;
    case FBP_OPT_ENGINE_FUSE_LANES:
        if (value < 0 || value > engine_block())
            return fail(FBP_ERR_INVALID_ARG, "fuse threshold must be in [0, %d]", engine_block());
        g->engine_fuse = (int)value;
        return FBP_OK;
    case FBP_OPT_ENGINE_SOLO_LANES:
        if (value < 0 || value > (1 << 20)) return fail(FBP_ERR_INVALID_ARG, "one-block threshold must be in [0, 2^20]");
        g->engine_solo = (int)value;
        return FBP_OK;
    default:
        return fail(FBP_ERR_INVALID_ARG, "unknown option %d", option);
    }
}

extern "C" int fbp_marginals(const fbp_graph *gc, float *out_p1, int out_is_device)
{
    t_err.clear();
    fbp_graph *g = const_cast<fbp_graph *>(gc);
    if (!g || (!out_p1 && g->h.nv > 0)) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    if (g->h.nv == 0) return FBP_OK;
    float *dst = out_p1;
    if (!out_is_device) {
        if (!g->p1 && dalloc_n(g, &g->p1, (size_t)g->h.nv)) return FBP_ERR_OOM;
        dst = g->p1;
    }
    int rc = marginals_launch(g, dst, g->stream);
    if (rc) return rc;
    if (!out_is_device) {
        CUDA_TRY(cudaMemcpyAsync(out_p1, g->p1, sizeof(float) * g->h.nv, cudaMemcpyDeviceToHost, g->stream));
        CUDA_TRY(cudaStreamSynchronize(g->stream));
    }
    return FBP_OK;
}

extern "C" int fbp_set_evidence(fbp_graph *g, int32_t var, int8_t value)
{
    t_err.clear();
    if (!g || var < 0 || var >= g->h.nv || value < -1 || value > 1)
        return fail(FBP_ERR_INVALID_ARG, "bad argument");
    g->evidence[var] = value;
    g->phi[var] = phi_of(g->prior[var], value);
    CUDA_TRY(cudaMemcpyAsync(const_cast<float *>(g->d.phi) + var, &g->phi[var], sizeof(float),
                             cudaMemcpyHostToDevice, g->stream));
    return FBP_OK;
}

extern "C" int fbp_messages_export(const fbp_graph *gc, float *a2v)
{
    t_err.clear();
    fbp_graph *g = const_cast<fbp_graph *>(gc);
    if (!g || (!a2v && g->h.ne)) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    if (!g->h.ne) return FBP_OK;
    if (!g->pairs && dalloc_n(g, &g->pairs, 2 * (size_t)g->h.ne)) return FBP_ERR_OOM;
    launch_decode_pairs(g->a2v[g->cur], g->pairs, g->h.ne, g->stream);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(a2v, g->pairs, sizeof(float) * 2 * g->h.ne, cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    return FBP_OK;
}

extern "C" int fbp_messages_import(fbp_graph *g, const float *a2v)
{
    t_err.clear();
    if (!g || (!a2v && g->h.ne)) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    if (!g->h.ne) return FBP_OK;
    for (int64_t i = 0; i < 2 * (int64_t)g->h.ne; ++i)
        if (!(a2v[i] >= 0.f) || !std::isfinite(a2v[i])) return fail(FBP_ERR_INVALID_ARG, "message %lld invalid", (long long)i / 2);
    if (!g->pairs && dalloc_n(g, &g->pairs, 2 * (size_t)g->h.ne)) return FBP_ERR_OOM;
    CUDA_TRY(cudaMemcpyAsync(g->pairs, a2v, sizeof(float) * 2 * g->h.ne, cudaMemcpyHostToDevice, g->stream));
    launch_encode_pairs(g->pairs, g->a2v[g->cur], g->h.ne, g->stream);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    return FBP_OK;
}

extern "C" int fbp_messages_reset(fbp_graph *g)
{
    t_err.clear();
    if (!g) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    launch_fill(g->a2v[g->cur], 1.0f, g->h.ne, g->stream);
    CUDA_TRY(cudaGetLastError());
    return FBP_OK;
}

extern "C" int fbp_get_stats(const fbp_graph *g, fbp_stats *out)
{
    if (!g || !out) return fail(FBP_ERR_INVALID_ARG, "NULL argument");
    *out = g->stats;
    return FBP_OK;
}
