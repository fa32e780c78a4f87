// Belief-form sequential engine (sm_103a): a static schedule (SEQFIX, TOPO,
// TOPO_FB, CUSTOM) run level by level on graphs with high-degree variables
// (FBP_OPT_ENGINE = 3).
//
// The level engine forms each v->a message of a level by walking the
// variable's whole row (Eq. 1), which costs the row's length per message: on
// BINGO-shaped graphs most levels touch a hub of 1e4-1e5 entries.  Here every
// variable's belief b_v = phi_v prod_a mu_{a->v} is kept current instead, in
// the flooding kernels' record and grouping (csrc/fbp_flood.cu), and
// mu_{v->a} = b_v / mu_{a->v} (v2a_from_belief).  One level (Algorithm 2's
// S_l, whose updates are independent):
//   1. every new a->v message of the level from the messages as they stand
//      (all reads before any write, as the level's sequential order allows);
//   2. the writes, into the factor-major messages and the variable-major copy;
//   3. the beliefs of the level's variables again: a row of degree <= 8 from
//      its entries, a longer row's touched 32-entry sub-chunks;
//   4. the touched rows of several sub-chunks recombined (one thread per row
//      of 2..8 sub-chunks, the whole block per longer row).
// A message read in step 1 thus includes every update of the earlier levels,
// as in the in-place sequential execution of Sec. 4.3 (the oracle's
// run_levels).  Levels are short (about ten edges on BINGO-1M SEQFIX), so the
// whole run is one block of kFloodSlots threads and the levels are separated
// by block barriers; the per-level lists of step 3 and 4 are built on the host
// (each without repeats).
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "fbp_flood.h"
#include "fbp_flood_dev.cuh"
#include "fbp_graph_impl.h"
#include "fbp_msg.cuh"

namespace fbp {
namespace {

using namespace fdev;

struct SeqHalfDev {
    int32_t n_levels;
    const int32_t *lp, *le;
    const int4 *dp;
    const int32_t *dv, *dk, *dm, *dh;
};

struct SeqArgs {
    DevGraph g;
    FloodPlanDev F;
    float *a2v;                        // factor-major messages, updated in place
    float *a2v_vm;                     // variable-major copy
    float *tmp;                        // new messages of a level wider than the block
    SeqHalfDev half[2];
    int32_t n_halves;
    int32_t max_iters;
    float tol;
    unsigned *res;                     // [max_iters] residual bits of each iteration
    int32_t *out;                      // [4] iterations, 0 converged / 1 at the limit
    unsigned long long *guards;
};

// One warp's edge of a level, loaded ahead: the edge, its factor's row, type
// and parameter, and (lane j) the variable at the factor's position j.
struct EdgePre {
    int q = -1, lo = 0, n = 0, type = 0, var = 0, a = 0;
    float p = 0.f;
};

__device__ __forceinline__ EdgePre load_edge(const SeqArgs &S, int q)
{
    const DevGraph &g = S.g;
    EdgePre E;
    E.q = q;
    E.a = __ldg(g.efac + q);
    E.lo = __ldg(g.fptr + E.a);
    E.n = __ldg(g.fptr + E.a + 1) - E.lo;
    E.type = __ldg(g.ftype + E.a);
    E.p = __ldg(g.fparam + E.a);
    const int lane = threadIdx.x & 31;
    if (lane < E.n && E.n <= 32) E.var = __ldg(g.fvars + E.lo + lane);
    return E;
}

// The new a->v message of edge E.q from the current beliefs and messages, by
// a whole warp: lane j forms the v->a message of the factor's position j
// (belief / own message), and the closed form reads them by shuffle (every
// lane evaluates it; the result is the same in all).  A factor wider than a
// warp forms its messages one position at a time.  old = the edge's message
// now.
__device__ __forceinline__ float seq_message_warp(const SeqArgs &S, const EdgePre &E, float &old,
                                                  unsigned long long &ng)
{
    const DevGraph &g = S.g;
    const int lane = threadIdx.x & 31;
    const int lo = E.lo, n = E.n, pos = E.q - E.lo;
    P2 mu;
    if (n <= 32) {  // warp-uniform
        float x = 1.f;
        if (lane < n) x = v2a_from_belief(__ldcg(S.F.belief + E.var), __ldcg(S.a2v + lo + lane));
        auto getm = [&](int j) { return dec(__shfl_sync(0xffffffffu, x, j)); };
        mu = E.type == kTypeTERMS ? a2v_terms(g, E.a, n, pos, getm) : a2v_unified(E.type, E.p, n, pos, getm);
    } else {
        auto getm = [&](int j) {
            const int e = lo + j;
            return dec(v2a_from_belief(__ldcg(S.F.belief + __ldg(g.fvars + e)), __ldcg(S.a2v + e)));
        };
        mu = E.type == kTypeTERMS ? a2v_terms(g, E.a, n, pos, getm) : a2v_unified(E.type, E.p, n, pos, getm);
    }
    bool gd = false;
    const float r = enc_fast(mu, gd);
    if (lane == 0) ng += gd;
    old = __ldcg(S.a2v + E.q);
    return r;
}

// A sub-chunk's product (as sub_product_item: its entries multiplied in
// order), by a whole warp: one load per lane, then every lane multiplies the
// shuffled entries in order; lane 0 writes.
__device__ __forceinline__ void seq_sub_warp(const SeqArgs &S, const int4 sc)
{
    const int lane = threadIdx.x & 31;
    // sc = {variable, begin, end, agg slot or -1}
    const float x = sc.y + lane < sc.z ? __ldcg(S.a2v_vm + sc.y + lane) : 1.f;
    float xs[kFloodSub];  // every shuffle first, so the multiply chain does not wait on them
#pragma unroll
    for (int j = 0; j < kFloodSub; ++j) xs[j] = __shfl_sync(0xffffffffu, x, j);
    XP t = xp_one();
    const int len = sc.z - sc.y;
#pragma unroll
    for (int j = 0; j < kFloodSub; ++j)
        if (j < len) xmul(t, xs[j]);
    if (lane != 0) return;
    if (sc.w >= 0) {
        S.F.agg[sc.w] = t;
        return;
    }
    xmul(t, __ldg(S.g.phi + sc.x));
    S.F.belief[sc.x] = belief_pack(t);
}

__device__ __forceinline__ void seq_write(const SeqArgs &S, int q, float r)
{
    S.a2v[q] = r;
    S.a2v_vm[__ldg(S.F.vpos + q)] = r;
}

constexpr int kSeqWarps = kFloodSlots / 32;
constexpr int kSeqStage = 1024;  // new messages of a level staged in shared memory

// The whole run in one block of kFloodSlots threads.
__global__ void __launch_bounds__(kFloodSlots, 1) k_seq_belief(const SeqArgs S)
{
    __shared__ XP s_x[kFloodSlots];
    __shared__ float s_r[kSeqStage];
    __shared__ unsigned s_res[kSeqWarps];
    __shared__ int s_stop;
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    unsigned long long ng = 0;
    int it = 1, status = 1;
    for (; it <= S.max_iters; ++it) {
        float rmax = 0.f;
        for (int h = 0; h < S.n_halves; ++h) {
            const SeqHalfDev H = h == 0 ? S.half[0] : S.half[1];
            for (int L = 0; L < H.n_levels; ++L) {
                // 1: the level's new messages, one warp per edge, staged in
                // shared memory (a level wider than kSeqStage also in S.tmp)
                const int e0 = __ldg(H.lp + L), e1 = __ldg(H.lp + L + 1);
                for (int i = e0 + wp; i < e1; i += kSeqWarps) {  // warp-uniform
                    float old;
                    const float r = seq_message_warp(S, load_edge(S, __ldg(H.le + i)), old, ng);
                    if (lane == 0) {
                        rmax = fmaxf(rmax, delta_p1_fast(r, old));
                        if (i - e0 < kSeqStage) s_r[i - e0] = r;
                        else S.tmp[i - e0] = r;
                    }
                }
                __syncthreads();
                // 2: the writes
                for (int i = e0 + t; i < e1; i += kFloodSlots)
                    seq_write(S, __ldg(H.le + i), i - e0 < kSeqStage ? s_r[i - e0] : S.tmp[i - e0]);
                __syncthreads();
                // 3: short rows and touched sub-chunks
                const int4 d0 = __ldg(H.dp + L), d1 = __ldg(H.dp + L + 1);
                for (int i = d0.x + t; i < d1.x; i += kFloodSlots) {
                    const int v = __ldg(H.dv + i);
                    const int lo = __ldg(S.g.vptr + v);
                    belief_short_row<true>(S.F, S.a2v_vm, v, lo, __ldg(S.g.vptr + v + 1) - lo, __ldg(S.g.phi + v));
                }
                for (int i = d0.y + wp; i < d1.y; i += kSeqWarps)  // warp-uniform
                    seq_sub_warp(S, __ldg(S.F.subs + __ldg(H.dk + i)));
                // 4: touched rows of several sub-chunks
                if (d1.z > d0.z || d1.w > d0.w) {
                    __syncthreads();
                    for (int i = d0.z + t; i < d1.z; i += kFloodSlots)
                        belief_medium_row<true>(S.g, S.F, __ldg(S.F.medium + __ldg(H.dm + i)));
                    for (int i = d0.w; i < d1.w; ++i) belief_hub_block<true, 4>(S.g, S.F, __ldg(H.dh + i), s_x);
                }
                __syncthreads();
            }
        }
        // the iteration's residual; stop at the first below tol
        const unsigned bits = __reduce_max_sync(0xffffffffu, __float_as_uint(rmax));
        if ((t & 31) == 0) s_res[t >> 5] = bits;
        __syncthreads();
        if (t == 0) {
            unsigned m = 0;
            for (int w = 0; w < kSeqWarps; ++w) m = max(m, s_res[w]);
            S.res[it - 1] = m;
            s_stop = __uint_as_float(m) < S.tol;
        }
        __syncthreads();
        if (s_stop) {
            status = 0;
            break;
        }
    }
    if (ng) atomicAdd(S.guards, ng);
    if (t == 0) {
        S.out[0] = min(it, S.max_iters);
        S.out[1] = status;
    }
}

}  // namespace

#define SEQ_TRY(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return fail(FBP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

namespace {

// The plan of one level list: per level, its edges and, without repeats,
// the short rows, sub-chunks, medium rows and hub rows its writes touch.
int build_seq_half(fbp_graph *g, const LevelSet &ls, const std::vector<int32_t> &vpos,
                   const std::vector<int32_t> &sub0, const std::vector<int32_t> &row_of, SeqHalf &out)
{
    const HostCSR &h = g->h;
    const int32_t nl = ls.lp.empty() ? 0 : (int32_t)ls.lp.size() - 1;
    std::vector<int32_t> lp(nl + 1), dv, dk, dm, dh;
    std::vector<int4> dp(nl + 1);
    std::vector<int32_t> vst(h.nv, -1), kst(g->flood_subs_h.size(), -1);
    int32_t widest = 0;
    for (int32_t L = 0; L < nl; ++L) {
        lp[L] = (int32_t)ls.lp[L];
        dp[L] = make_int4((int)dv.size(), (int)dk.size(), (int)dm.size(), (int)dh.size());
        widest = std::max(widest, (int32_t)(ls.lp[L + 1] - ls.lp[L]));
        for (int64_t i = ls.lp[L]; i < ls.lp[L + 1]; ++i) {
            const int32_t q = ls.le[i], v = h.fvars[q];
            const int32_t lo = h.vptr[v], d = h.vptr[v + 1] - lo;
            if (d <= kFloodSmallMax) {
                if (vst[v] != L) dv.push_back(v);
                vst[v] = L;
                continue;
            }
            const int32_t k = sub0[v] + (vpos[q] - lo) / kFloodSub;
            if (kst[k] != L) dk.push_back(k);
            kst[k] = L;
            if (row_of[v] != -1 && vst[v] != L) (row_of[v] >= 0 ? dm : dh).push_back(row_of[v] >= 0 ? row_of[v] : -2 - row_of[v]);
            vst[v] = L;
        }
    }
    lp[nl] = nl > 0 ? (int32_t)ls.lp[nl] : 0;
    dp[nl] = make_int4((int)dv.size(), (int)dk.size(), (int)dm.size(), (int)dh.size());
    out.n_levels = nl;
    out.max_level = widest;
    int rc = upload(g, &out.lp, lp.data(), lp.size());
    if (!rc) rc = upload(g, &out.le, ls.le.data(), ls.le.size());
    if (!rc) rc = upload(g, &out.dp, dp.data(), dp.size());
    if (!rc) rc = upload(g, &out.dv, dv.data(), dv.size());
    if (!rc) rc = upload(g, &out.dk, dk.data(), dk.size());
    if (!rc) rc = upload(g, &out.dm, dm.data(), dm.size());
    if (!rc) rc = upload(g, &out.dh, dh.data(), dh.size());
    return rc;
}

int build_seq_plan(fbp_graph *g)
{
    const HostCSR &h = g->h;
    free_seq(g);
    // where each row's products live in the flooding plan
    std::vector<int32_t> vpos(h.ne), sub0(h.nv, -1), row_of(h.nv, -1);
    parallel_for(h.ne, host_threads(), 1 << 16, [&](int64_t b, int64_t e) {
        for (int64_t k = b; k < e; ++k) vpos[h.vedge[k]] = (int32_t)k;
    });
    for (size_t k = g->flood_subs_h.size(); k-- > 0;) sub0[g->flood_subs_h[k].x] = (int32_t)k;  // first sub-chunk
    for (size_t m = 0; m < g->flood_medium_h.size(); ++m) row_of[g->flood_medium_h[m].x] = (int32_t)m;
    for (size_t r = 0; r < g->flood_hub_h.size(); ++r) row_of[g->flood_hub_h[r].x] = -2 - (int32_t)r;
    g->seq.resize(g->halves.size());
    int64_t wide = 0;
    for (size_t k = 0; k < g->halves.size(); ++k) {
        int rc = build_seq_half(g, g->halves[k], vpos, sub0, row_of, g->seq[k]);
        if (rc) {
            free_seq(g);
            return rc;
        }
        wide = std::max<int64_t>(wide, g->seq[k].max_level);
    }
    if (wide > kSeqStage) {
        int rc = dalloc_n(g, &g->seq_tmp, (size_t)wide);
        if (rc) {
            free_seq(g);
            return rc;
        }
        g->seq_tmp_cap = wide;
    }
    return FBP_OK;
}

SeqHalfDev half_dev(const SeqHalf &s)
{
    return SeqHalfDev{s.n_levels, s.lp, s.le, s.dp, s.dv, s.dk, s.dm, s.dh};
}

}  // namespace

void free_seq(fbp_graph *g)
{
    for (auto &s : g->seq) {
        for (void *p : {(void *)s.lp, (void *)s.le, (void *)s.dp, (void *)s.dv, (void *)s.dk, (void *)s.dm, (void *)s.dh})
            dfree(g, p);
    }
    g->seq.clear();
    dfree(g, g->seq_tmp);
    g->seq_tmp = nullptr;
    g->seq_tmp_cap = 0;
}

int run_seq(fbp_graph *g, int32_t max_iters, double tol, int32_t *iters_out, double *residual_out)
{
    const HostCSR &h = g->h;
    if (g->halves.empty() || g->halves.size() > 2) return fail(FBP_ERR_INVALID_ARG, "no static schedule");
    int rc = ensure_res_cap(g, std::max(max_iters, 1));
    if (rc) return rc;
    if (!g->a2v_vm && (rc = dalloc_n(g, &g->a2v_vm, (size_t)h.ne))) return rc;
    if (!g->flood_ready && (rc = build_flood_plan(g))) return rc;
    if (g->seq.size() != g->halves.size() && (rc = build_seq_plan(g))) return rc;
    SEQ_TRY(cudaMemsetAsync(g->d_res_it, 0, sizeof(unsigned) * std::max(max_iters, 1), g->stream));
    SEQ_TRY(cudaMemsetAsync(g->d_out, 0, sizeof(int32_t) * 4, g->stream));
    if (max_iters == 0) return finish_run(g, 0, 0.0, FBP_NOT_CONVERGED, iters_out, residual_out);
    float *a2v = g->a2v[g->cur];
    // the beliefs of the current messages, as one flooding phase 1
    flood_sync(g->d, a2v, g->a2v_vm, g->stream);
    FloodPlanDev F = g->flood;
    F.done = g->d_out;  // 0 until the run below writes it
    flood_beliefs(g->d, F, g->a2v_vm, g->stream);
    SeqArgs S{};
    S.g = g->d;
    S.F = F;
    S.a2v = a2v;
    S.a2v_vm = g->a2v_vm;
    S.tmp = g->seq_tmp;
    S.half[0] = half_dev(g->seq[0]);
    S.half[1] = g->seq.size() > 1 ? half_dev(g->seq[1]) : SeqHalfDev{};
    S.n_halves = (int32_t)g->seq.size();
    S.max_iters = max_iters;
    S.tol = (float)tol;
    S.res = g->d_res_it;
    S.out = g->d_out;
    S.guards = g->d_guards;
    k_seq_belief<<<1, kFloodSlots, 0, g->stream>>>(S);
    SEQ_TRY(cudaGetLastError());
    g->stats.kernel_launches += 2 + (flood_launches(g->d, g->flood) > 3 ? 2 : 1);
    if ((rc = engine_check(g))) return rc;
    const int32_t it = g->h_out[0];
    const int status = g->h_out[1] == 0 ? FBP_OK : FBP_NOT_CONVERGED;
    int64_t per_iter = 0;
    for (auto &ls : g->halves) per_iter += (int64_t)ls.le.size();
    g->stats.updates += (int64_t)it * per_iter;
    return finish_run(g, it, residual_at(g, it), status, iters_out, residual_out);
}

}  // namespace fbp
